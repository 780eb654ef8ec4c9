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
// k_diag_inv<double> is the FP64 form; k_diag_inv_f32 the mixed form (FP32
// copy of L, FP32 Z, FP64 variance accumulation).  In the mixed form the large
// supernodes near the root (an upward-closed set, spi_options.diag_tc_min_pivots)
// are skipped here and taken afterwards by the tensor-core kernel of
// diag_tc.cu, which continues from the Z rows and partial variances this
// kernel leaves.
#include <cuda_runtime.h>

#include <algorithm>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kThreads = 256;
constexpr int kRT = 64;  // panel rows per staged tile

struct DiagArgs {
    int32_t B;
    const int32_t *order, *blk_ptr, *uptr, *us, *ulo, *uhi, *uzoff, *rel, *rhs_out, *rhs_zrow, *rhs_col;
    const int64_t *urel, *zbase;
    void* Z;
};

// Number of entries of the sorted pivots cols[lo .. lo+nb) below `limit`.
__device__ __forceinline__ int count_below(const int32_t* __restrict__ cols, int lo, int nb, int32_t limit) {
    int a = 0, b = nb;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (cols[lo + mid] < limit) a = mid + 1; else b = mid;
    }
    return a;
}

// The right-hand sides with a nonzero on the block columns [j0, j1] of a
// supernode are those in the union of the columns' subtrees, i.e. with pivot
// in [min fdesc(j0..j1), j1]; within the block's sorted active range
// [lo, lo + nb) that is the sub-range [lo + *a, lo + *b).
__device__ __forceinline__ void block_column_range(const DevSym& d, const int32_t* __restrict__ cols, int lo,
                                                   int nb, int32_t j0, int32_t j1, int* a, int* b) {
    int32_t first = j0;
    for (int32_t j = j0; j <= j1; ++j) first = min(first, d.fdesc[j]);
    *a = count_below(cols, lo, nb, first);
    *b = count_below(cols, lo, nb, j1 + 1);
}

template <typename T>
size_t diag_smem_bytes(int B) {
    return sizeof(double) * (size_t)(B + kT) + sizeof(T) * (size_t)(kT * B + kT * (kT + 1) + kRT * (kT + 1));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_diag_inv(DevSym d, DiagArgs p, const T* __restrict__ L,
                                                       const double* __restrict__ D, double* __restrict__ out,
                                                       Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    out += blockIdx.y * bs.out;
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = p.B;
    double* var = reinterpret_cast<double*>(smem);
    double* dv = var + B;  // 1 / d of the current block column
    T* Zd = reinterpret_cast<T*>(dv + kT);  // [kT][B]
    T* Ld = Zd + kT * B;                    // [kT][kT+1]
    T* Lt = Ld + kT * (kT + 1);             // [kRT][kT+1]
    __shared__ int rng[2];
    const int tid = threadIdx.x;
    const int b = p.order[blockIdx.x];
    T* Z = reinterpret_cast<T*>(p.Z) + blockIdx.y * bs.Z + p.zbase[b];
    const int64_t zsz = p.zbase[b + 1] - p.zbase[b];
    const int r0b = p.blk_ptr[b], nr = p.blk_ptr[b + 1] - r0b;
    for (int64_t i = tid; i < zsz; i += kThreads) Z[i] = T(0);
    for (int t = tid; t < B; t += kThreads) var[t] = 0.0;
    __syncthreads();
    for (int t = tid; t < nr; t += kThreads) Z[(int64_t)p.rhs_zrow[r0b + t] * B + t] = T(1);
    for (int u = p.uptr[b]; u < p.uptr[b + 1]; ++u) {
        const int s = p.us[u], lo0 = p.ulo[u], nbu = p.uhi[u] - lo0, zo = p.uzoff[u];
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
        const T* P = L + d.lptr[s];
        const int32_t* rel = p.rel + p.urel[u];
        for (int cb = 0; cb < k; cb += kT) {
            const int w = min(kT, k - cb);
            __syncthreads();
            if (tid == 0) block_column_range(d, p.rhs_col + r0b, lo0, nbu, f + cb, f + cb + w - 1, &rng[0], &rng[1]);
            for (int e = tid; e < kT * kT; e += kThreads) {
                const int i = e % kT, c = e / kT;
                Ld[i * (kT + 1) + c] = (i < w && c < i) ? P[(cb + i) + (int64_t)(cb + c) * m] : T(0);
            }
            __syncthreads();
            const int lo = lo0 + rng[0], nb = rng[1] - rng[0];
            if (tid < kT) dv[tid] = tid < w ? (d.dinv_a ? d.dinv_a[f + cb + tid] : 1.0 / D[f + cb + tid]) : 0.0;
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
                    if (d.dinv_a) {
                        // second pivot of a 2x2 block: the cross term 2 z_p z_c (D^-1)_pc with its
                        // partner p = c - 1, whose z is final (this block column or the last one)
                        const int j = f + cb + c;
                        if (d.pair[j] == j - 1) {
                            const T zp = c > 0 ? Zd[(c - 1) * B + t] : Z[(int64_t)(zo + cb - 1) * B + lo + t];
                            v += 2.0 * (double)zp * (double)zc * d.dinv_b[j];
                        }
                    }
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
                const int w4 = w & ~3;
                for (int e = tid; e < nrow * nb; e += kThreads) {
                    const int i = e / nb, t = e - i * nb;
                    const T* lr = Lt + i * (kT + 1);
                    const int64_t row = rb + i;
                    const int64_t zr = row < k ? (int64_t)zo + row : (int64_t)rel[row - k];
                    // start from the row's old value: every product is one FMA, no final subtraction
                    // (the FP64 pipe is the bound of this kernel)
                    T acc = Z[zr * B + lo + t];
                    int c = 0;
                    for (; c < w4; c += 4) {
                        acc -= lr[c] * Zd[c * B + t];
                        acc -= lr[c + 1] * Zd[(c + 1) * B + t];
                        acc -= lr[c + 2] * Zd[(c + 2) * B + t];
                        acc -= lr[c + 3] * Zd[(c + 3) * B + t];
                    }
                    for (; c < w; ++c) acc -= lr[c] * Zd[c * B + t];
                    Z[zr * B + lo + t] = acc;
                }
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < nr; t += kThreads) out[p.rhs_out[r0b + t]] = var[t];
}

// Mixed form: the same walk with an FP32 copy of L and FP32 Z (variance sums
// in FP64), in two phases per supernode s of the path:
//   A. its own k columns, 32 at a time: the unit-lower diagonal block solved
//      per right-hand side (thread per RHS), the squares scaled by 1/d added
//      to the variances in FP64, and the rows of s below the block (still
//      inside s) updated by a register-tiled SIMT GEMM;
//   B. the rows below s (its ancestors' pivots) updated once:
//      Z_below -= L(below, 0:k) Z_s, one GEMM with K = k, each 128-row tile
//      accumulated in registers over all of s's columns and added into Z at
//      the end.
// Phase B writes every Z row below s once per supernode instead of once per
// 32-column block, which is what the variance workspace's traffic (beyond L2
// at the benchmark sizes) is made of.  GEMM tiles: 128 threads, a 128-row x
// 64-RHS output tile, 8 x 8 outputs per thread; the panel tile is staged
// transposed (a thread's 8 rows are one pair of float4 loads), double-
// buffered with cp.async, and so is phase B's 32 x 64 chunk of Z_s.
constexpr int kFThreads = 128;
constexpr int kFRows = 128;
constexpr int kFCols = 64;

size_t diag_f32_smem_bytes(int B) {
    return sizeof(double) * (size_t)(B + kT) +
           sizeof(float) * (size_t)(kT * B + kT * (kT + 1) + 2 * kT * (kFRows + 4) + 2 * kT * kFCols);
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 writes a zero
// (nothing is read from src).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// 8 x 8 outer-product accumulation over `kw` K-columns of a transposed 128-row
// panel tile Lt ([K][kFRows + 4]) and a K x cols chunk Zc (leading dimension ldz).
__device__ __forceinline__ void gemm8x8(float (&acc)[8][8], const float* Lt, const float* Zc, int ldz, int kw,
                                        int ty, int tx) {
    const float* lcol = Lt + ty * 8;
    const float* zcol = Zc + tx * 8;
    for (int c = 0; c < kw; ++c) {
        const float4 a0 = *reinterpret_cast<const float4*>(lcol + c * (kFRows + 4));
        const float4 a1 = *reinterpret_cast<const float4*>(lcol + c * (kFRows + 4) + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(zcol + c * ldz);
        const float4 b1 = *reinterpret_cast<const float4*>(zcol + c * ldz + 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
}

__global__ void __launch_bounds__(kFThreads) k_diag_inv_f32(DevSym d, DiagArgs p, const float* __restrict__ L,
                                                             const double* __restrict__ D,
                                                             double* __restrict__ out, Strides bs,
                                                             const uint8_t* __restrict__ skip) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    out += blockIdx.y * bs.out;
    extern __shared__ __align__(16) unsigned char smem[];
    const int B = p.B;  // a multiple of 8 (padded RHS count)
    double* var = reinterpret_cast<double*>(smem);
    double* dv = var + B;
    float* Zd = reinterpret_cast<float*>(dv + kT);  // [kT][B]
    float* Ld = Zd + kT * B;                        // [kT][kT+1]
    float* Lt0 = Ld + kT * (kT + 1);                // [2][kT][kFRows+4], transposed panel tiles
    float* Lt1 = Lt0 + kT * (kFRows + 4);
    float* Zk0 = Lt1 + kT * (kFRows + 4);           // [2][kT][kFCols], phase B's chunks of Z_s
    float* Zk1 = Zk0 + kT * kFCols;
    __shared__ int rng[2];
    const int tid = threadIdx.x;
    const int tx = tid % 8, ty = tid / 8;
    const int b = p.order[blockIdx.x];
    float* Z = reinterpret_cast<float*>(p.Z) + blockIdx.y * bs.Z + p.zbase[b];
    const int64_t zsz = p.zbase[b + 1] - p.zbase[b];
    const int r0b = p.blk_ptr[b], nr = p.blk_ptr[b + 1] - r0b;
    for (int64_t i = tid; i < zsz; i += kFThreads) Z[i] = 0.f;
    for (int t = tid; t < B; t += kFThreads) var[t] = 0.0;
    __syncthreads();
    for (int t = tid; t < nr; t += kFThreads) Z[(int64_t)p.rhs_zrow[r0b + t] * B + t] = 1.f;
    for (int u = p.uptr[b]; u < p.uptr[b + 1]; ++u) {
        const int s = p.us[u], lo0 = p.ulo[u], nbu = p.uhi[u] - lo0, zo = p.uzoff[u];
        if (skip && skip[s]) continue;  // the tensor-core kernel's (it runs after this one)
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
        const float* P = L + d.lptr[s];
        const int32_t* rel = p.rel + p.urel[u];
        // ---- phase A: the supernode's own columns
        for (int cb = 0; cb < k; cb += kT) {
            const int w = min(kT, k - cb);
            __syncthreads();
            if (tid == 0) block_column_range(d, p.rhs_col + r0b, lo0, nbu, f + cb, f + cb + w - 1, &rng[0], &rng[1]);
            for (int e = tid; e < kT * kT; e += kFThreads) {
                const int i = e % kT, c = e / kT;
                Ld[i * (kT + 1) + c] = (i < w && c < i) ? P[(cb + i) + (int64_t)(cb + c) * m] : 0.f;
            }
            __syncthreads();
            const int lo = lo0 + rng[0], nb = rng[1] - rng[0];
            if (tid < kT) dv[tid] = tid < w ? 1.0 / D[f + cb + tid] : 0.0;
            for (int e = tid; e < kT * B; e += kFThreads) {
                const int c = e / B, t = e - c * B;
                Zd[e] = (c < w && t < nb) ? Z[(int64_t)(zo + cb + c) * B + lo + t] : 0.f;
            }
            __syncthreads();
            for (int t = tid; t < nb; t += kFThreads) {
                double v = 0.0;
                for (int c = 0; c < w; ++c) {
                    const float zc = Zd[c * B + t];
                    v += (double)zc * (double)zc * dv[c];
                    for (int r = c + 1; r < w; ++r) Zd[r * B + t] -= Ld[r * (kT + 1) + c] * zc;
                }
                var[lo + t] += v;
            }
            __syncthreads();
            for (int e = tid; e < w * nb; e += kFThreads) {
                const int c = e / nb, t = e - c * nb;
                Z[(int64_t)(zo + cb + c) * B + lo + t] = Zd[c * B + t];
            }
            // rows [cb + w, k) of the supernode, 128-row tiles double-buffered
            const int64_t rfirst = cb + w;
            const int ntiles = (int)((k - rfirst + kFRows - 1) / kFRows);
            auto issue = [&](int tt, float* dst) {
                const int64_t rb = rfirst + (int64_t)tt * kFRows;
                const int nrow = (int)(k - rb < kFRows ? k - rb : kFRows);
                for (int e = tid; e < kFRows * kT; e += kFThreads) {
                    const int i = e % kFRows, c = e / kFRows;
                    const bool ok = i < nrow && c < w;
                    cp_async4(dst + c * (kFRows + 4) + i, ok ? P + (rb + i) + (int64_t)(cb + c) * m : P, ok ? 4 : 0);
                }
                cp_async_commit();
            };
            if (ntiles > 0) issue(0, Lt0);
            const int w4 = (w + 3) & ~3;
            for (int tt = 0; tt < ntiles; ++tt) {
                const float* Lt = (tt & 1) ? Lt1 : Lt0;
                if (tt + 1 < ntiles) {
                    issue(tt + 1, (tt & 1) ? Lt0 : Lt1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                const int64_t rb = rfirst + (int64_t)tt * kFRows;
                const int nrow = (int)(k - rb < kFRows ? k - rb : kFRows);
                if (ty * 8 < nrow) {
                    for (int cbase = 0; cbase < nb; cbase += kFCols) {
                        if (cbase + tx * 8 >= nb) continue;
                        float acc[8][8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
                        gemm8x8(acc, Lt, Zd + cbase, B, w4, ty, tx);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int il = ty * 8 + i;
                            if (il >= nrow) break;
                            float* zrow = Z + (int64_t)(zo + rb + il) * B + lo + cbase + tx * 8;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                if (cbase + tx * 8 + j < nb) atomicAdd(zrow + j, -acc[i][j]);
                        }
                    }
                }
                __syncthreads();  // tile tt read by all before its buffer is refilled
            }
        }
        // ---- phase B: the rows below s, K = all k columns of s, RHS [lo0, lo0 + nbu)
        if (m > k) {
            const int nkc = (k + kT - 1) / kT;
            for (int64_t rb = k; rb < m; rb += kFRows) {
                const int nrow = (int)(m - rb < kFRows ? m - rb : kFRows);
                for (int cbase = 0; cbase < nbu; cbase += kFCols) {
                    const int ncol = min(kFCols, nbu - cbase);
                    auto issue = [&](int kc, float* lt, float* zk) {
                        const int c0 = kc * kT, w = min(kT, k - c0);
                        for (int e = tid; e < kFRows * kT; e += kFThreads) {
                            const int i = e % kFRows, c = e / kFRows;
                            const bool ok = i < nrow && c < w;
                            cp_async4(lt + c * (kFRows + 4) + i, ok ? P + (rb + i) + (int64_t)(c0 + c) * m : P, ok ? 4 : 0);
                        }
                        for (int e = tid; e < kT * kFCols; e += kFThreads) {
                            const int c = e / kFCols, t = e - c * kFCols;
                            const bool ok = c < w && t < ncol;
                            const float* src = Z + (int64_t)(zo + c0 + c) * B + lo0 + cbase + t;
                            cp_async4(zk + e, ok ? src : Z, ok ? 4 : 0);
                        }
                        cp_async_commit();
                    };
                    __syncthreads();  // the previous tile's buffers are free
                    issue(0, Lt0, Zk0);
                    float acc[8][8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
                    for (int kc = 0; kc < nkc; ++kc) {
                        const float* lt = (kc & 1) ? Lt1 : Lt0;
                        const float* zk = (kc & 1) ? Zk1 : Zk0;
                        if (kc + 1 < nkc) {
                            issue(kc + 1, (kc & 1) ? Lt0 : Lt1, (kc & 1) ? Zk0 : Zk1);
                            cp_async_wait<1>();
                        } else {
                            cp_async_wait<0>();
                        }
                        __syncthreads();
                        if (ty * 8 < nrow && tx * 8 < ncol) gemm8x8(acc, lt, zk, kFCols, min(kT, k - kc * kT + 3) & ~3, ty, tx);
                        __syncthreads();  // chunk kc read by all before its buffers are refilled
                    }
                    if (ty * 8 < nrow && tx * 8 < ncol) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int il = ty * 8 + i;
                            if (il >= nrow) break;
                            float* zrow = Z + (int64_t)rel[rb + il - k] * B + lo0 + cbase + tx * 8;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                if (tx * 8 + j < ncol) atomicAdd(zrow + j, -acc[i][j]);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < nr; t += kFThreads) out[p.rhs_out[r0b + t]] = var[t];
}

template <typename T>
void launch_t(const DevSym& d, const DevDiagPlan& p, const T* L, const double* D, double* out, int nb,
              const Strides& bs, size_t smem_min, cudaStream_t st) {
    DiagArgs a{p.B, p.order, p.blk_ptr, p.uptr, p.us, p.ulo, p.uhi, p.uzoff, p.rel, p.rhs_out, p.rhs_zrow,
               p.rhs_col, p.urel, p.zbase, p.Z};
    const size_t sm = std::max(diag_smem_bytes<T>(p.B), smem_min);
    k_diag_inv<T><<<dim3(p.nblocks, nb), kThreads, sm, st>>>(d, a, L, D, out, bs);
}

// Block of the inverse from one block's forward solves (paper Sec. 3.3.1:
// any set of entries of the inverse).  After k_diag_inv<double> has run on a
// single block, Z holds z_t = L^-1 e_(pivot of slot t) on the union of the
// block's paths, local row r belonging to pivot zpiv[r].  Since
// N^-1 = L^-T D^-1 L^-1, G_st = sum_r Z[r][s] Z[r][t] / d_zpiv[r].  One CTA
// per 32 x 32 tile of the lower triangle of G; rows in chunks of 32 staged in
// shared memory; thread (jj, i0) owns column jj and rows i0 + 4q of the tile.
// The result goes to out[rhs_out[s] * ldo + rhs_out[t]] and its mirror.
__global__ void __launch_bounds__(128) k_inverse_gram(const double* __restrict__ Z, int B, int64_t R,
                                                      const int32_t* __restrict__ zpiv,
                                                      const double* __restrict__ D,
                                                      const int32_t* __restrict__ rhs_out, double* __restrict__ out,
                                                      int64_t ldo) {
    __shared__ double Zs[kT][kT + 1];
    __shared__ double Zt[kT][kT + 1];
    __shared__ double w[kT];
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
    const int tj = (int)blockIdx.x - ti * (ti + 1) / 2;
    const int s0 = ti * kT, t0 = tj * kT;
    const int tid = threadIdx.x, jj = tid % kT, i0 = tid / kT;
    double acc[kT / 4];
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) acc[q] = 0.0;
    for (int64_t r0 = 0; r0 < R; r0 += kT) {
        __syncthreads();
        for (int e = tid; e < kT * kT; e += 128) {
            const int rr = e / kT, c = e % kT;
            const int64_t r = r0 + rr;
            Zs[rr][c] = (r < R && s0 + c < B) ? Z[r * B + s0 + c] : 0.0;
            Zt[rr][c] = (r < R && t0 + c < B) ? Z[r * B + t0 + c] : 0.0;
        }
        if (tid < kT) w[tid] = r0 + tid < R ? 1.0 / D[zpiv[r0 + tid]] : 0.0;
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kT; ++rr) {
            const double bt = Zt[rr][jj] * w[rr];
#pragma unroll
            for (int q = 0; q < kT / 4; ++q) acc[q] += Zs[rr][i0 + 4 * q] * bt;
        }
    }
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
        const int sl = s0 + i0 + 4 * q, tl = t0 + jj;
        if (sl < B && tl < B && tl <= sl) {
            const int64_t so = rhs_out[sl], to = rhs_out[tl];
            out[so * ldo + to] = acc[q];
            out[to * ldo + so] = acc[q];
        }
    }
}

// Gather every block's solved vectors into one matrix Zg (R rows = the union
// of all blocks' paths, one column per right-hand-side slot): block b's local
// row r is global row rowmap[zbase[b] / B + r]; rows off a block's paths stay 0.
__global__ void k_gather_blocks(const double* __restrict__ Z, int B, const int64_t* __restrict__ zbase,
                                const int32_t* __restrict__ blk_ptr, const int32_t* __restrict__ rowmap,
                                int64_t nslots, double* __restrict__ Zg) {
    const int b = blockIdx.x;
    const int64_t z0 = zbase[b], rows = (zbase[b + 1] - z0) / B;
    const int s0 = blk_ptr[b], nb = blk_ptr[b + 1] - s0;
    const int32_t* rm = rowmap + z0 / B;
    for (int64_t e = threadIdx.x; e < rows * nb; e += blockDim.x) {
        const int64_t r = e / nb;
        const int t = (int)(e - r * nb);
        Zg[(int64_t)rm[r] * nslots + s0 + t] = Z[z0 + r * B + t];
    }
}

}  // namespace

void launch_inverse_block(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D,
                          double* var_scratch, double* Zg, int64_t R, double* out, int64_t ldo, cudaStream_t st) {
    if (p.nblocks == 0 || p.nrhs == 0) return;
    Strides bs;
    bs.Z = p.zsize;
    bs.out = p.nrhs;
    cudaMemsetAsync(Zg, 0, (size_t)R * (size_t)p.nrhs * sizeof(double), st);
    launch_t<double>(d, p, L, D, var_scratch, 1, bs, 0, st);
    k_gather_blocks<<<p.nblocks, 256, 0, st>>>(p.Z, p.B, p.zbase, p.blk_ptr, p.rowmap, p.nrhs, Zg);
    const int nt = (int)((p.nrhs + kT - 1) / kT);
    k_inverse_gram<<<nt * (nt + 1) / 2, 128, 0, st>>>(Zg, (int)p.nrhs, R, p.zpiv, D, p.rhs_out, out, ldo);
}

namespace {
// out[dst[e]] = G[src[e]]: the requested entries of one block of the inverse
__global__ void k_pick_entries(const double* __restrict__ G, const int64_t* __restrict__ src,
                               const int64_t* __restrict__ dst, int64_t cnt, double* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
        out[dst[e]] = G[src[e]];
}
}  // namespace

void launch_pick_entries(const double* G, const int64_t* src, const int64_t* dst, int64_t cnt, double* out,
                         cudaStream_t st) {
    if (cnt <= 0) return;
    k_pick_entries<<<(int)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, st>>>(G, src, dst, cnt, out);
}

cudaError_t diag_kernel_setup(int B, size_t smem_min) {
    cudaError_t e = cudaFuncSetAttribute(k_diag_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max(diag_smem_bytes<double>(B), smem_min));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_diag_inv_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(diag_f32_smem_bytes((B + 7) & ~7), smem_min));
    // the largest shared-memory carveout, as the solve kernels that run beside them
    const int pref = (int)cudaSharedmemCarveoutMaxShared;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_inv<double>, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_diag_inv_f32, cudaFuncAttributePreferredSharedMemoryCarveout, pref);
    return e;
}

void launch_diag_inverse(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D, double* out,
                         int nb, const Strides& bs, size_t smem_min, cudaStream_t st) {
    if (p.nblocks == 0 || nb == 0) return;
    launch_t<double>(d, p, L, D, out, nb, bs, smem_min, st);
}

void launch_diag_inverse_f32(const DevSym& d, const DevDiagPlan& p, const float* L, const double* D, double* out,
                             int nb, const Strides& bs, size_t smem_min, const uint8_t* skip, cudaStream_t st) {
    if (p.nblocks == 0 || nb == 0) return;
    DiagArgs a{p.B, p.order, p.blk_ptr, p.uptr, p.us, p.ulo, p.uhi, p.uzoff, p.rel, p.rhs_out, p.rhs_zrow,
               p.rhs_col, p.urel, p.zbase, p.Z};
    k_diag_inv_f32<<<dim3(p.nblocks, nb), kFThreads, std::max(diag_f32_smem_bytes(p.B), smem_min), st>>>(
        d, a, L, D, out, bs, skip);
}

}  // namespace spi
