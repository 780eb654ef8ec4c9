// diag.cu -- variances diag(N^-1) by pruned, blocked sparse-RHS forward
// solves (paper Sec. 3.3.1 and Sec. 4.3):
//   (N^-1)_ii = sum_k z_k^2 / d_k,  z = L^-1 e_i,
// where z is nonzero only on the elimination-tree path i -> root (pruning),
// and the right-hand sides are processed in blocks of B consecutive pivots
// of the postorder, so that a block's paths share most of their supernodes.
//
// One CTA owns one block.  It walks the union of the block's paths upward
// (ascending supernode order is a topological order).  At supernode s it
// works only on the block's right-hand sides that lie in the subtree of s --
// a contiguous range [lo, hi) of the block, because subtrees are contiguous
// in postorder.  The panel of s (m x k, column-major) is consumed in block
// columns of 32: the 32 x nb slice of Z for those pivots is staged in shared
// memory and solved with the unit-lower diagonal block (one thread per
// right-hand side), its squares scaled by 1/d are added to the variances in
// FP64, and the rows below -- the rest of the supernode and, through the
// block's row map, its ancestors -- receive Z_rows -= L_rows,cols Z_cols from
// 64-row panel tiles staged in shared memory.
//
// The element type T is double (FP64 form) or float (mixed form: FP32 copy
// of L, FP32 Z, FP64 variance accumulation).
#include <cuda_runtime.h>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kThreads = 256;
constexpr int kRT = 64;  // panel rows per staged tile

struct DiagArgs {
    int32_t B;
    const int32_t *order, *blk_ptr, *uptr, *us, *ulo, *uhi, *uzoff, *rel, *rhs_out, *rhs_zrow;
    const int64_t *urel, *zbase;
    void* Z;
};

template <typename T>
size_t diag_smem_bytes(int B) {
    return sizeof(double) * (size_t)(B + kT) + sizeof(T) * (size_t)(kT * B + kT * (kT + 1) + kRT * (kT + 1));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_diag_inv(DevSym d, DiagArgs p, const T* __restrict__ L,
                                                       const double* __restrict__ D, double* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = p.B;
    double* var = reinterpret_cast<double*>(smem);
    double* dv = var + B;  // 1 / d of the current block column
    T* Zd = reinterpret_cast<T*>(dv + kT);  // [kT][B]
    T* Ld = Zd + kT * B;                    // [kT][kT+1]
    T* Lt = Ld + kT * (kT + 1);             // [kRT][kT+1]
    const int tid = threadIdx.x;
    const int b = p.order[blockIdx.x];
    T* Z = reinterpret_cast<T*>(p.Z) + p.zbase[b];
    const int64_t zsz = p.zbase[b + 1] - p.zbase[b];
    const int r0b = p.blk_ptr[b], nr = p.blk_ptr[b + 1] - r0b;
    for (int64_t i = tid; i < zsz; i += kThreads) Z[i] = T(0);
    for (int t = tid; t < B; t += kThreads) var[t] = 0.0;
    __syncthreads();
    for (int t = tid; t < nr; t += kThreads) Z[(int64_t)p.rhs_zrow[r0b + t] * B + t] = T(1);
    for (int u = p.uptr[b]; u < p.uptr[b + 1]; ++u) {
        const int s = p.us[u], lo = p.ulo[u], nb = p.uhi[u] - lo, zo = p.uzoff[u];
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
        const T* P = L + d.lptr[s];
        const int32_t* rel = p.rel + p.urel[u];
        for (int cb = 0; cb < k; cb += kT) {
            const int w = min(kT, k - cb);
            __syncthreads();
            for (int e = tid; e < kT * kT; e += kThreads) {
                const int i = e % kT, c = e / kT;
                Ld[i * (kT + 1) + c] = (i < w && c < i) ? P[(cb + i) + (int64_t)(cb + c) * m] : T(0);
            }
            if (tid < kT) dv[tid] = tid < w ? 1.0 / D[f + cb + tid] : 0.0;
            for (int e = tid; e < kT * nb; e += kThreads) {
                const int c = e / nb, t = e - c * nb;
                Zd[c * B + t] = c < w ? Z[(int64_t)(zo + cb + c) * B + lo + t] : T(0);
            }
            __syncthreads();
            for (int t = tid; t < nb; t += kThreads) {
                double v = 0.0;
                for (int c = 0; c < w; ++c) {
                    const T zc = Zd[c * B + t];
                    v += (double)zc * (double)zc * dv[c];
                    for (int r = c + 1; r < w; ++r) Zd[r * B + t] -= Ld[r * (kT + 1) + c] * zc;
                }
                var[lo + t] += v;
            }
            __syncthreads();
            for (int e = tid; e < w * nb; e += kThreads) {
                const int c = e / nb, t = e - c * nb;
                Z[(int64_t)(zo + cb + c) * B + lo + t] = Zd[c * B + t];
            }
            for (int64_t rb = cb + w; rb < m; rb += kRT) {
                const int nrow = (int)(m - rb < kRT ? m - rb : kRT);
                __syncthreads();
                for (int e = tid; e < kRT * kT; e += kThreads) {
                    const int i = e % kRT, c = e / kRT;
                    Lt[i * (kT + 1) + c] = (i < nrow && c < w) ? P[(rb + i) + (int64_t)(cb + c) * m] : T(0);
                }
                __syncthreads();
                for (int e = tid; e < nrow * nb; e += kThreads) {
                    const int i = e / nb, t = e - i * nb;
                    const T* lr = Lt + i * (kT + 1);
                    T acc = T(0);
#pragma unroll
                    for (int c = 0; c < kT; ++c) acc += lr[c] * Zd[c * B + t];
                    const int64_t row = rb + i;
                    const int64_t zr = row < k ? (int64_t)zo + row : (int64_t)rel[row - k];
                    Z[zr * B + lo + t] -= acc;
                }
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < nr; t += kThreads) out[p.rhs_out[r0b + t]] = var[t];
}

template <typename T>
void launch_t(const DevSym& d, const DevDiagPlan& p, const T* L, const double* D, double* out, cudaStream_t st) {
    DiagArgs a{p.B, p.order, p.blk_ptr, p.uptr, p.us, p.ulo, p.uhi, p.uzoff, p.rel, p.rhs_out, p.rhs_zrow,
               p.urel, p.zbase, p.Z};
    size_t sm = diag_smem_bytes<T>(p.B);
    k_diag_inv<T><<<p.nblocks, kThreads, sm, st>>>(d, a, L, D, out);
}

}  // namespace

cudaError_t diag_kernel_setup(int B) {
    cudaError_t e = cudaFuncSetAttribute(k_diag_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)diag_smem_bytes<double>(B));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_diag_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)diag_smem_bytes<float>(B));
}

void launch_diag_inverse(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D, double* out,
                         cudaStream_t st) {
    if (p.nblocks == 0) return;
    launch_t<double>(d, p, L, D, out, st);
}

void launch_diag_inverse_f32(const DevSym& d, const DevDiagPlan& p, const float* L, const double* D, double* out,
                             cudaStream_t st) {
    if (p.nblocks == 0) return;
    launch_t<float>(d, p, L, D, out, st);
}

}  // namespace spi
