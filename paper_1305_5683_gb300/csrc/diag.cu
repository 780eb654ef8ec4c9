// diag.cu -- variances diag(N^-1) by pruned, blocked sparse-RHS forward
// solves (paper Sec. 3.3.1 and Sec. 4.3):
//   (N^-1)_ii = sum_k z_k^2 / d_k,  z = L^-1 e_i,
// where z is nonzero only on the elimination-tree path i -> root (pruning),
// and the right-hand sides are processed in blocks of B consecutive pivots
// of the postorder, so that a block's paths share most of their supernodes.
// One CTA owns one block: it walks the union of the block's paths upward
// (ascending supernode order is a topological order), and at each supernode
// it works only on the block's right-hand sides that lie in the supernode's
// subtree -- a contiguous range of the block because subtrees are
// contiguous in postorder.
#include <cuda_runtime.h>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxB = 1024;

struct DiagArgs {
    int32_t B;
    const int32_t *order, *blk_ptr, *uptr, *us, *ulo, *uhi, *uzoff, *rel, *rhs_out, *rhs_zrow;
    const int64_t *urel, *zbase;
    double* Z;
};

__global__ void __launch_bounds__(kThreads) k_diag_inv(DevSym d, DiagArgs p, const double* __restrict__ L,
                                                       const double* __restrict__ D, double* __restrict__ out) {
    __shared__ double var[kMaxB];
    const int tid = threadIdx.x;
    const int b = p.order[blockIdx.x];
    const int B = p.B;
    double* Z = p.Z + p.zbase[b];
    const int64_t zsz = p.zbase[b + 1] - p.zbase[b];
    const int r0 = p.blk_ptr[b], nr = p.blk_ptr[b + 1] - r0;
    for (int64_t i = tid; i < zsz; i += kThreads) Z[i] = 0.0;
    for (int t = tid; t < B; t += kThreads) var[t] = 0.0;
    __syncthreads();
    for (int t = tid; t < nr; t += kThreads) Z[(int64_t)p.rhs_zrow[r0 + t] * B + t] = 1.0;
    __syncthreads();
    for (int u = p.uptr[b]; u < p.uptr[b + 1]; ++u) {
        const int s = p.us[u], lo = p.ulo[u], hi = p.uhi[u], zo = p.uzoff[u];
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
        const double* P = L + d.lptr[s];
        // unit-lower solve with L11 and the variance terms of the supernode's columns
        for (int t = lo + tid; t < hi; t += kThreads) {
            double v = 0.0;
            for (int c = 0; c < k; ++c) {
                const double zc = Z[(int64_t)(zo + c) * B + t];
                if (zc == 0.0) continue;
                v += zc * zc / D[f + c];
                for (int r = c + 1; r < k; ++r) Z[(int64_t)(zo + r) * B + t] -= P[r + (int64_t)c * m] * zc;
            }
            var[t] += v;
        }
        __syncthreads();
        // Z[below rows] -= L21 Z_s
        const int nb = hi - lo;
        const int64_t mb = m - k;
        const int32_t* rel = p.rel + p.urel[u];
        for (int64_t e = tid; e < mb * nb; e += kThreads) {
            const int64_t r = e / nb;
            const int t = lo + (int)(e - r * nb);
            double acc = 0.0;
            for (int c = 0; c < k; ++c) acc += P[k + r + (int64_t)c * m] * Z[(int64_t)(zo + c) * B + t];
            Z[(int64_t)rel[r] * B + t] -= acc;
        }
        __syncthreads();
    }
    for (int t = tid; t < nr; t += kThreads) out[p.rhs_out[r0 + t]] = var[t];
}

}  // namespace

void launch_diag_inverse(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D, double* out,
                         cudaStream_t st) {
    if (p.nblocks == 0) return;
    DiagArgs a{p.B, p.order, p.blk_ptr, p.uptr, p.us, p.ulo, p.uhi, p.uzoff, p.rel, p.rhs_out, p.rhs_zrow,
               p.urel, p.zbase, p.Z};
    k_diag_inv<<<p.nblocks, kThreads, 0, st>>>(d, a, L, D, out);
}

}  // namespace spi
