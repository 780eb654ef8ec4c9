// solve.cu -- solution phase (paper Sec. 3.2.3): forward substitution
// z = L^-1 P b bottom-up over the supernodal tree, then x = P^T L^-T D^-1 z
// top-down.  One launch per tree level; one CTA per supernode.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kThreads = 256;
constexpr int kFwdRows = 512;  // rows below the block per forward CTA
constexpr int kBwdCols = 256;  // columns per backward CTA
// In a batch of bands, a level runs each sweep in one launch, one CTA per
// (supernode, band) looping over the supernode's 32-column steps, when its
// largest supernode's work (k m - k^2 / 2 FMAs, on one SM) is below what the
// launch-per-step form spends on its chain of launches (about 10 us each,
// ~20,000 FMAs of one SM).  For a single problem the launch-per-step form
// measured faster at every level (its rows spread over more CTAs), so it
// keeps that form; so do the wide fronts near the root.
constexpr int64_t kFuseFmaPerStep = 20000;
constexpr int kAncRegs = 4;  // ancestor rows per thread whose updates are summed in registers

__global__ void k_permute_in(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ b,
                             double* __restrict__ w) {
    b += (int64_t)blockIdx.y * n;
    w += (int64_t)blockIdx.y * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        w[k] = b[perm[k]];
}

__global__ void k_permute_out(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ w,
                              double* __restrict__ x) {
    w += (int64_t)blockIdx.y * n;
    x += (int64_t)blockIdx.y * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        x[perm[k]] = w[k];
}

// (D^-1 z) at pivot j: z_j / d_j, or, for a symmetric indefinite factorization,
// D^-1 taken block by block (the 2x2 partner's z is final after the forward sweep).
__device__ __forceinline__ double dinv_z(const DevSym& d, const double* z, const double* D, int j) {
    if (!d.dinv_a) return z[j] / D[j];
    const int q = d.pair[j];
    return d.dinv_a[j] * z[j] + (q >= 0 ? d.dinv_b[j] * z[q] : 0.0);
}

// Rows of x gathered per pass of the backward first pass (x[rows[t]] for a chunk of
// rows t below the supernode): staged in shared memory by independent loads of the
// whole CTA, so that the column dot products read them from there instead of
// waiting on a dependent rows[t] -> x[rows[t]] pair of global loads per row.
constexpr int kXs = 2048;

template <bool kCg, typename TL>
__device__ __forceinline__ void gather_x(TL* xs, const double* x, const int32_t* rows, int64_t t0, int64_t t1) {
    for (int64_t t = t0 + threadIdx.x; t < t1; t += blockDim.x)
        xs[t - t0] = (TL)(kCg ? __ldcg(x + rows[t]) : x[rows[t]]);
}

// Backward diagonal block of a 32-column step: lane c (of warp 0) receives column c of
// L_bb below the diagonal (row r in lcol[r], r > c; rows past wb zero), staged through
// shared memory so that the panel is read a column at a time (lanes = rows).
template <typename TL>
__device__ __forceinline__ void bwd_block_cols(const TL* P, int64_t m, int cb, int wb, TL (*Lbb)[kT + 1],
                                               TL (&lcol)[kT], int lane) {
#pragma unroll 8
    for (int c = 0; c < kT; ++c)
        Lbb[lane][c] = (lane > c && lane < wb) ? P[(cb + lane) + (int64_t)(cb + c) * m] : TL(0);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kT; ++r) lcol[r] = Lbb[r][lane];
}

// y[a] -= sum_{r < wb} P[cb + r][a] xb[r] for the columns a in [a0, a1) of a panel P
// (column-major, leading dimension m; wb <= 32 kRowChunks): the backward sweep's update of
// a supernode's earlier columns by a solved block.  Warp w takes the groups of 32
// consecutive columns g = a0 + 32 (w + i nwarps); lane r loads row cb + r (+ 32 t) of each
// of the group's columns -- coalesced: the rows of a column are contiguous -- and
// lane_sums leaves column g + j's dot product in lane j.  kCg: y is read through L2
// (written by other CTAs of the same launch).
template <int kRowChunks, bool kCg, typename TL>
__device__ void bwd_update(const TL* P, int64_t m, int cb, int wb, const TL* xb, int a0, int a1, double* y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

    for (int g = a0 + 32 * warp; g < a1; g += 32 * nw) {
        TL v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = TL(0);
#pragma unroll
        for (int t = 0; t < kRowChunks; ++t) {
            const int r = 32 * t + lane;
            if (r < wb) {
                const TL xr = xb[r];
                const TL* p = P + (cb + r) + (int64_t)g * m;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (g + j < a1) v[j] += p[(int64_t)j * m] * xr;
            }
        }
        const TL sum = lane_sums(v, lane);
        if (g + lane < a1) {
            double* py = y + g + lane;
            *py = (kCg ? __ldcg(py) : *py) - (double)sum;
        }
    }
}

// Forward block step b of the supernodes of one level.  Item (s, chunk):
// every CTA of supernode s solves the 32 x 32 unit-lower diagonal block
// x_b = L_bb^-1 w_b in registers (lane r owns row r), the chunk-0 CTA stores
// x_b into z, and each CTA subtracts L(rows, block b) x_b from its own chunk
// of the rows below: the supernode's later pivots (plain stores: the rows of
// a chunk belong to one CTA) and its ancestors' rows (atomics: siblings of
// the level update the same ancestors).
template <typename TL>
__global__ void __launch_bounds__(kThreads) k_fwd_step(DevSym d, const int32_t* __restrict__ items, int b,
                                                       const TL* __restrict__ L, double* __restrict__ w,
                                                       double* __restrict__ z, Strides bs) {
    L += blockIdx.y * bs.L;
    w += blockIdx.y * bs.n;
    z += blockIdx.y * bs.n;
    __shared__ TL xb[kT];
    const int tid = threadIdx.x, lane = tid & 31;
    const int s = items[2 * blockIdx.x], chunk = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const TL* P = L + d.lptr[s];
    const int cb = b * kT, wb = min(kT, k - cb);
    if (tid < 32) {
        // lane r holds row r of the diagonal block: 32 independent loads first
        TL lrow[kT];
#pragma unroll
        for (int c = 0; c < kT; ++c)
            lrow[c] = (c < lane && lane < wb) ? P[(cb + lane) + (int64_t)(cb + c) * m] : 0.0;
        TL x = lane < wb ? (TL)w[f + cb + lane] : TL(0);
#pragma unroll
        for (int c = 0; c < kT - 1; ++c) {
            const TL xc = __shfl_sync(0xffffffffu, x, c);
            x -= lrow[c] * xc;
        }
        xb[lane] = x;
        if (chunk == 0 && lane < wb) z[f + cb + lane] = x;
    }
    __syncthreads();
    const int32_t* rows = d.srows + d.srowptr[s];
    const int64_t r0 = cb + wb + (int64_t)chunk * kFwdRows;
    const int64_t r1 = (m < r0 + kFwdRows) ? m : r0 + kFwdRows;
    for (int64_t r = r0 + tid; r < r1; r += kThreads) {
        TL acc = 0;
#pragma unroll 8
        for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
        if (r < k) w[f + r] -= acc;
        else atomicAdd(w + rows[r], -(double)acc);
    }
}

// Backward, first launch of a level: y_c = z_c / d_c - sum_{t >= k} L[t][c] x[rows[t]]
// for a chunk of 32 of the supernode's columns, stored into w.  Warp q takes
// the columns q, q + 8, q + 16, q + 24 of the chunk; its lanes run over the
// rows below (coalesced column reads, the gathered x shared by the four
// columns) and a shuffle reduction finishes each dot product.  Four partial
// sums per thread keep the kernel's registers low enough for several CTAs
// per SM.
template <typename TL>
__global__ void __launch_bounds__(kThreads) k_bwd_init(DevSym d, const int32_t* __restrict__ items,
                                                       const TL* __restrict__ L, const double* __restrict__ D,
                                                       const double* __restrict__ z, const double* __restrict__ x,
                                                       double* __restrict__ w, Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.Dn;
    z += blockIdx.y * bs.n;
    x += blockIdx.y * bs.n;
    w += blockIdx.y * bs.n;
    constexpr int kWarps = kThreads / 32, kPer = kT / kWarps;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = items[2 * blockIdx.x], chunk = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const TL* P = L + d.lptr[s];
    const int32_t* rows = d.srows + d.srowptr[s];
    const int c0 = chunk * kT, nc = min(kT, k - c0);
    __shared__ TL xs[kXs];
    TL acc[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) acc[q] = 0.0;
    for (int64_t t0 = k; t0 < m; t0 += kXs) {
        const int64_t t1 = m < t0 + kXs ? m : t0 + kXs;
        __syncthreads();
        gather_x<false>(xs, x, rows, t0, t1);
        __syncthreads();
#pragma unroll 4
        for (int64_t t = t0 + lane; t < t1; t += 32) {
            const TL xv = xs[t - t0];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int c = warp + kWarps * q;
                if (c < nc) acc[q] += P[t + (int64_t)(c0 + c) * m] * xv;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        TL v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int c = warp + kWarps * q;
        if (lane == 0 && c < nc) w[f + c0 + c] = dinv_z(d, z, D, f + c0 + c) - v;
    }
}

// Backward block step b (descending): every CTA solves L_bb^T x_b = y_b in
// registers, the chunk-0 CTA stores x_b, and each CTA updates its chunk of the
// earlier columns a < 32 b: y_a -= sum_r L[32b + r][a] x_b[r].
template <typename TL>
__global__ void __launch_bounds__(kThreads) k_bwd_step(DevSym d, const int32_t* __restrict__ items, int b,
                                                       const TL* __restrict__ L, double* __restrict__ w,
                                                       double* __restrict__ x, Strides bs) {
    L += blockIdx.y * bs.L;
    w += blockIdx.y * bs.n;
    x += blockIdx.y * bs.n;
    __shared__ TL xb[kT];
    __shared__ TL Lbb[kT][kT + 1];
    const int tid = threadIdx.x, lane = tid & 31;
    const int s = items[2 * blockIdx.x], chunk = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const TL* P = L + d.lptr[s];
    const int cb = b * kT, wb = min(kT, k - cb);
    if (tid < 32) {
        // lane c holds column c of the diagonal block (L_bb^T row c)
        TL lcol[kT];
        bwd_block_cols(P, m, cb, wb, Lbb, lcol, lane);
        TL y = lane < wb ? (TL)w[f + cb + lane] : TL(0);
#pragma unroll
        for (int r = kT - 1; r > 0; --r) {
            const TL xr = __shfl_sync(0xffffffffu, y, r);
            y -= lcol[r] * xr;
        }
        xb[lane] = y;
        if (chunk == 0 && lane < wb) x[f + cb + lane] = y;
    }
    __syncthreads();
    bwd_update<1, false>(P, m, cb, wb, xb, chunk * kBwdCols, min(cb, (chunk + 1) * kBwdCols), w + f);
}

// Forward sweep of one level in one launch: one CTA per (supernode, band)
// runs all of the supernode's 32-column steps.  Each step solves the diagonal
// block in warp 0 (lane r owns row r, as k_fwd_step) and updates the
// supernode's later pivots in place; the contributions to the ancestors' rows
// are summed over the steps in registers (thread t owns rows k + t + 256 j)
// and added once at the end, by atomics since siblings share ancestors.
template <typename TL>
__global__ void __launch_bounds__(kThreads) k_fwd_level(DevSym d, const int32_t* __restrict__ items,
                                                        const TL* __restrict__ L, double* __restrict__ w,
                                                        double* __restrict__ z, Strides bs) {
    L += blockIdx.y * bs.L;
    w += blockIdx.y * bs.n;
    z += blockIdx.y * bs.n;
    __shared__ TL xb[kT];
    const int tid = threadIdx.x, lane = tid & 31;
    const int s = items[2 * blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const TL* P = L + d.lptr[s];
    const int32_t* rows = d.srows + d.srowptr[s];
    const bool in_regs = m - k <= (int64_t)kAncRegs * kThreads;
    TL anc[kAncRegs];
#pragma unroll
    for (int j = 0; j < kAncRegs; ++j) anc[j] = 0.0;
    for (int cb = 0; cb < k; cb += kT) {
        const int wb = min(kT, k - cb);
        if (tid < 32) {
            TL lrow[kT];
#pragma unroll
            for (int c = 0; c < kT; ++c)
                lrow[c] = (c < lane && lane < wb) ? P[(cb + lane) + (int64_t)(cb + c) * m] : 0.0;
            TL x = lane < wb ? (TL)w[f + cb + lane] : TL(0);
#pragma unroll
            for (int c = 0; c < kT - 1; ++c) {
                const TL xc = __shfl_sync(0xffffffffu, x, c);
                x -= lrow[c] * xc;
            }
            xb[lane] = x;
            if (lane < wb) z[f + cb + lane] = x;
        }
        __syncthreads();
        for (int r = cb + wb + tid; r < k; r += kThreads) {  // the supernode's later pivots
            TL acc = 0;
            for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
            w[f + r] -= acc;
        }
        if (in_regs) {
#pragma unroll
            for (int j = 0; j < kAncRegs; ++j) {
                const int64_t r = k + tid + (int64_t)j * kThreads;
                if (r < m) {
                    TL acc = 0;
                    for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
                    anc[j] += acc;
                }
            }
        } else {
            for (int64_t r = k + tid; r < m; r += kThreads) {
                TL acc = 0;
                for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
                atomicAdd(w + rows[r], -(double)acc);
            }
        }
        __syncthreads();  // w of the next diagonal block, and xb, are rewritten
    }
    if (in_regs) {
#pragma unroll
        for (int j = 0; j < kAncRegs; ++j) {
            const int64_t r = k + tid + (int64_t)j * kThreads;
            if (r < m) atomicAdd(w + rows[r], -(double)anc[j]);
        }
    }
}

// Backward sweep of one level in one launch: one CTA per (supernode, band).
// First y_c = z_c / d_c - sum_{t >= k} L[t][c] x[rows[t]] for all of its
// columns (a warp per column, as k_bwd_init), then its 32-column steps in
// descending order (as k_bwd_step), each updating every earlier column.
template <typename TL>
__global__ void __launch_bounds__(kThreads) k_bwd_level(DevSym d, const int32_t* __restrict__ items,
                                                        const TL* __restrict__ L, const double* __restrict__ D,
                                                        const double* __restrict__ z, double* __restrict__ x,
                                                        double* __restrict__ w, Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.Dn;
    z += blockIdx.y * bs.n;
    x += blockIdx.y * bs.n;
    w += blockIdx.y * bs.n;
    constexpr int kWarps = kThreads / 32;
    __shared__ TL xb[kT];
    __shared__ TL xs[kXs];
    __shared__ TL Lbb[kT][kT + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s = items[2 * blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const TL* P = L + d.lptr[s];
    const int32_t* rows = d.srows + d.srowptr[s];
    // y_c = z_c / d_c - sum_{t >= k} L[t][c] x[rows[t]], a warp per column, the rows
    // below in passes of kXs whose x are gathered into shared memory first
    if (m == k)
        for (int c = tid; c < k; c += kThreads) w[f + c] = dinv_z(d, z, D, f + c);
    for (int64_t t0 = k; t0 < m; t0 += kXs) {
        const int64_t t1 = m < t0 + kXs ? m : t0 + kXs;
        __syncthreads();
        gather_x<false>(xs, x, rows, t0, t1);
        __syncthreads();
        for (int c = warp; c < k; c += kWarps) {
            TL acc = 0;
            for (int64_t t = t0 + lane; t < t1; t += 32) acc += P[t + (int64_t)c * m] * xs[t - t0];
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) w[f + c] = (t0 == k ? dinv_z(d, z, D, f + c) : w[f + c]) - acc;
        }
    }
    __syncthreads();
    for (int cb = ((k - 1) / kT) * kT; cb >= 0; cb -= kT) {
        const int wb = min(kT, k - cb);
        if (tid < 32) {
            TL lcol[kT];
            bwd_block_cols(P, m, cb, wb, Lbb, lcol, lane);
            TL y = lane < wb ? (TL)w[f + cb + lane] : TL(0);
#pragma unroll
            for (int r = kT - 1; r > 0; --r) {
                const TL xr = __shfl_sync(0xffffffffu, y, r);
                y -= lcol[r] * xr;
            }
            xb[lane] = y;
            if (lane < wb) x[f + cb + lane] = y;
        }
        __syncthreads();
        bwd_update<1, false>(P, m, cb, wb, xb, 0, cb, w + f);
        __syncthreads();
    }
}

// r -= N x for the symmetric N given by its lower CSC (caller numbering), one
// warp per column: the column's dot product for r_j, and the mirrored
// upper-triangle entries scattered into r_i.
__global__ void k_sym_residual(int32_t n, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                               const double* __restrict__ va, const double* __restrict__ x, double* __restrict__ r,
                               int64_t nnz) {
    va += blockIdx.y * nnz;
    x += (int64_t)blockIdx.y * n;
    r += (int64_t)blockIdx.y * n;
    const int lane = threadIdx.x & 31;
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const double xj = x[j];
        double acc = 0.0;
        for (int64_t p = cp[j] + lane; p < cp[j + 1]; p += 32) {
            const int32_t i = ri[p];
            const double a = va[p];
            acc += a * x[i];
            if (i != j) atomicAdd(r + i, -a * xj);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(r + j, -acc);
    }
}

// out[0] += sum a_i^2, out[1] += sum b_i^2
__global__ void k_norms2(int32_t n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
    a += (int64_t)blockIdx.y * n;
    if (b) b += (int64_t)blockIdx.y * n;
    out += 2 * blockIdx.y;
    double sa = 0.0, sb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        sa += a[i] * a[i];
        if (b) sb += b[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, sa);
        if (b) atomicAdd(out + 1, sb);
    }
}

__global__ void k_axpy(int32_t n, const double* __restrict__ dx, double* __restrict__ x) {
    dx += (int64_t)blockIdx.y * n;
    x += (int64_t)blockIdx.y * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += dx[i];
}

// w[t n + pos[t]] = 1 (w zeroed before): unit right-hand sides in pivot numbering
__global__ void k_set_units(int32_t n, const int32_t* __restrict__ pos, int R, double* __restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < R) w[(int64_t)t * n + pos[t]] = 1.0;
}

// out[t] = 2 v_t[idx_t] + sum_k v_t[k] r_t[k], with r_t = -N v_t: the variance
// 2 e^T v - v^T N v of an approximate v = F^-1 e (one CTA per right-hand side)
__global__ void k_refined_var(int32_t n, const double* __restrict__ v, const double* __restrict__ r,
                              const int32_t* __restrict__ idx, double* __restrict__ out) {
    __shared__ double part[kThreads / 32];
    const int t = blockIdx.x;
    v += (int64_t)t * n;
    r += (int64_t)t * n;
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += kThreads) s += v[k] * r[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) a += part[q];
        out[t] = 2.0 * v[idx[t]] + a;
    }
}

// out[t] = sum_k z_t[k]^2 dinv[k]: the variance from an unpruned forward solve
// (one CTA per right-hand side)
__global__ void k_zsq_var(int32_t n, const double* __restrict__ z, const double* __restrict__ dinv,
                          double* __restrict__ out) {
    __shared__ double part[kThreads / 32];
    const int t = blockIdx.x;
    z += (int64_t)t * n;
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += kThreads) s += z[k] * z[k] * dinv[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) a += part[q];
        out[t] = a;
    }
}

__global__ void k_reciprocal(int32_t n, const double* __restrict__ D, double* __restrict__ dinv) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        dinv[k] = 1.0 / D[k];
}

// ---------------------------------------------------------------------------
// Wide steps (mixed form): the supernodes whose variances run on the tensor
// cores have, per 128 of their columns, the inverse X_bb of the unit-lower
// diagonal block (prepared at the end of the factorization, FP32).  Their
// sweeps then take 128 columns per step: forward x_b = X_bb w_b and then
// w_below -= L(rows, block b) x_b; backward x_b = X_bb^T y_b and then
// y_a -= sum_r L[128 b + r][a] x_b[r] for the earlier columns a.  The same
// substitution in blocks of 128, a quarter of the 32-column steps on the chain.
constexpr int kW = 128;
constexpr int kFwdRowsW = 256;  // rows below per wide forward CTA
constexpr int kBwdColsW = 256;  // earlier columns per wide backward CTA

__global__ void __launch_bounds__(kThreads) k_fwd_wide(DevSym d, const int32_t* __restrict__ items, int b,
                                                       const float* __restrict__ L, WideArgs wa,
                                                       double* __restrict__ w, double* __restrict__ z, Strides bs) {
    const int band = blockIdx.y;
    L += band * bs.L;
    w += band * bs.n;
    z += band * bs.n;
    __shared__ float wv[kW], xb[kW];
    const int s = items[2 * blockIdx.x], chunk = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const float* P = L + d.lptr[s];
    const int32_t* rows = d.srows + d.srowptr[s];
    const int cb = b * kW, wb = min(kW, k - cb);
    const float* X = wa.xinv + band * wa.xband + (int64_t)(wa.xptr[s] + b) * (kW * kW);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kRowsPerWarp = kW / (kThreads / 32);
    // x_b[r] = sum_c X[r][c] w[c]: a warp per row (rows warp + 8 q), 16-byte loads of the
    // row, all of the warp's rows loaded before the reductions
    float4 xr[kRowsPerWarp];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q)
        xr[q] = *reinterpret_cast<const float4*>(X + (warp + (kThreads / 32) * q) * kW + 4 * lane);
    if (tid < kW) wv[tid] = tid < wb ? (float)w[f + cb + tid] : 0.f;
    __syncthreads();
    {
        const float w0 = wv[4 * lane], w1 = wv[4 * lane + 1], w2 = wv[4 * lane + 2], w3 = wv[4 * lane + 3];
#pragma unroll
        for (int q = 0; q < kRowsPerWarp; ++q) {
            float v = xr[q].x * w0 + xr[q].y * w1 + xr[q].z * w2 + xr[q].w * w3;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) xb[warp + (kThreads / 32) * q] = v;
        }
    }
    __syncthreads();
    if (chunk == 0 && tid < wb) z[f + cb + tid] = xb[tid];
    const int64_t r0 = cb + wb + (int64_t)chunk * kFwdRowsW;
    const int64_t r1 = m < r0 + kFwdRowsW ? m : r0 + kFwdRowsW;
    for (int64_t r = r0 + tid; r < r1; r += kThreads) {
        float acc = 0.f;
#pragma unroll 16
        for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
        if (r < k) w[f + r] -= acc;
        else atomicAdd(w + rows[r], -(double)acc);
    }
}

// (at most 128 registers: its CTAs must fit beside a variance kernel's on one SM, since
// the two run concurrently on two streams)
__global__ void __launch_bounds__(kThreads, 2) k_bwd_wide(DevSym d, const int32_t* __restrict__ items, int b,
                                                       const float* __restrict__ L, WideArgs wa,
                                                       double* __restrict__ w, double* __restrict__ x, Strides bs) {
    const int band = blockIdx.y;
    L += band * bs.L;
    w += band * bs.n;
    x += band * bs.n;
    __shared__ float yv[kW], xb[kW];
    const int s = items[2 * blockIdx.x], chunk = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const float* P = L + d.lptr[s];
    const int cb = b * kW, wb = min(kW, k - cb);
    const float* X = wa.xinv + band * wa.xband + (int64_t)(wa.xptr[s] + b) * (kW * kW);
    const int tid = threadIdx.x;
    __shared__ float part[kW];
    if (tid < kW) yv[tid] = tid < wb ? (float)w[f + cb + tid] : 0.f;
    __syncthreads();
    // x_b[c] = sum_r X[r][c] y[r] (X is zero above its diagonal): column c by threads c
    // (rows [0, 64)) and c + 128 (rows [64, 128)), coalesced over c, 16 loads in flight
    static_assert(kThreads == 2 * kW, "two threads per column of the diagonal tile");
    {
        const int c = tid % kW, h = tid / kW;
        float v = 0.f;
#pragma unroll 16
        for (int r = 64 * h; r < 64 * h + 64; ++r) v += X[r * kW + c] * yv[r];
        if (h == 1) part[c] = v;
        __syncthreads();
        if (h == 0) xb[c] = v + part[c];
    }
    __syncthreads();
    if (chunk == 0 && tid < wb) x[f + cb + tid] = xb[tid];
    bwd_update<kW / 32, false>(P, m, cb, wb, xb, chunk * kBwdColsW, min(cb, (chunk + 1) * kBwdColsW), w + f);
}

// ---------------------------------------------------------------------------
// Dependency-driven solve (one launch for both sweeps).
//
// The tasks -- forward step b of supernode s over a 512-row chunk of the rows
// below the step (kSolveFwd), the backward first pass over 32 of its columns
// (kSolveBwdInit), backward step b over 256 of its earlier columns
// (kSolveBwdStep) -- are listed forward sweep first, bottom-up level by level,
// then the backward sweep top-down, each level phase by phase across its
// supernodes, so that every task depends only on tasks before it.  A CTA takes
// the next task from a global counter, waits (bounded) until the counter it
// depends on reaches its value, runs it and counts it done: forward steps wait
// for the supernode's earlier steps, its first step for every forward task of
// its children (which in turn waited for theirs: all updates of the subtree
// into its rows are in); the backward pass of a supernode waits for every
// backward task of its parent (all ancestors' x are final), or, at a root, for
// its own forward sweep; backward steps wait for the supernode's earlier
// backward tasks.  Vectors written during the launch are read through L2.  As
// in the factorization, a wait that gives up raises FLAG_TIMEOUT and every CTA
// skips its remaining tasks.
constexpr uint32_t kSolveWaitLimit = 1u << 25;

__device__ __forceinline__ int sv_ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool sv_aborted(const DevStatus* status) {
    return (*reinterpret_cast<const volatile int*>(&status->flags) & FLAG_TIMEOUT) != 0;
}

__device__ bool sv_wait(const int* c, int need, const DevStatus* status, uint32_t limit) {
    if (limit == 0) return false;
    for (uint32_t it = 0;; ++it) {
        if (sv_ld_acquire(c) >= need) return true;
        if (it >= limit) return false;
        if ((it & 31) == 31 && sv_aborted(status)) return false;
        __nanosleep(100);
    }
}

template <typename TL>
__global__ void __launch_bounds__(kThreads) k_solve_dag(DevSym d, const DagTask* __restrict__ tasks, int ntasks,
                                                        int nb, int* cnt, int cstride, const TL* __restrict__ L,
                                                        const double* __restrict__ D, double* w, double* z, double* x,
                                                        DevStatus* status, Strides bs, uint32_t wait_limit) {
    // small shared memory: many CTAs of this kernel share an SM, each running short tasks
    constexpr int kXsDag = 512;
    __shared__ TL xb[kT];
    __shared__ TL xs[kXsDag];
    __shared__ int64_t s_t;
    __shared__ int s_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int* next = cnt + (int64_t)nb * cstride;
    const int64_t total = (int64_t)ntasks * nb;
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const int64_t t = (int64_t)(unsigned)atomicAdd(next, 1);
            int ok = 0;
            if (t < total) {
                const DagTask tk = tasks[t / nb];
                ok = !sv_aborted(status);
                if (ok && tk.wait_val > 0) {
                    ok = sv_wait(cnt + (t % nb) * cstride + tk.wait_idx, tk.wait_val, status, wait_limit);
                    if (!ok) atomicOr(&status->flags, FLAG_TIMEOUT);
                }
            }
            s_t = t;
            s_ok = ok;
        }
        __syncthreads();
        const int64_t t = s_t;
        if (t >= total) break;
        if (!s_ok) continue;
        const int band = (int)(t % nb);
        const DagTask tk = tasks[t / nb];
        const TL* Lb = L + band * bs.L;
        const double* Db = D + band * bs.Dn;
        double* wb_ = w + band * bs.n;
        double* zb = z + band * bs.n;
        double* xv = x + band * bs.n;
        const int s = tk.s;
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
        const TL* P = Lb + d.lptr[s];
        const int32_t* rows = d.srows + d.srowptr[s];
        if (tk.type == kSolveFwd) {
            const int cb = tk.a * kT, wb = min(kT, k - cb), chunk = tk.b;
            if (tid < 32) {
                TL lrow[kT];
#pragma unroll
                for (int c = 0; c < kT; ++c)
                    lrow[c] = (c < lane && lane < wb) ? P[(cb + lane) + (int64_t)(cb + c) * m] : 0.0;
                TL xx = lane < wb ? (TL)__ldcg(wb_ + f + cb + lane) : TL(0);
#pragma unroll
                for (int c = 0; c < kT - 1; ++c) {
                    const TL xc = __shfl_sync(0xffffffffu, xx, c);
                    xx -= lrow[c] * xc;
                }
                xb[lane] = xx;
                if (chunk == 0 && lane < wb) zb[f + cb + lane] = xx;
            }
            __syncthreads();
            const int64_t r0 = cb + wb + (int64_t)chunk * kFwdRows;
            const int64_t r1 = (m < r0 + kFwdRows) ? m : r0 + kFwdRows;
            for (int64_t r = r0 + tid; r < r1; r += kThreads) {
                TL acc = 0;
#pragma unroll 8
                for (int c = 0; c < wb; ++c) acc += P[r + (int64_t)(cb + c) * m] * xb[c];
                if (r < k) wb_[f + r] = __ldcg(wb_ + f + r) - acc;
                else atomicAdd(wb_ + rows[r], -(double)acc);
            }
        } else if (tk.type == kSolveBwdInit) {
            constexpr int kWarps = kThreads / 32, kPer = kT / kWarps;
            const int c0 = tk.b * kT, nc = min(kT, k - c0);
            TL acc[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) acc[q] = 0.0;
            for (int64_t t0 = k; t0 < m; t0 += kXsDag) {
                const int64_t t1 = m < t0 + kXsDag ? m : t0 + kXsDag;
                __syncthreads();
                gather_x<true>(xs, xv, rows, t0, t1);
                __syncthreads();
#pragma unroll 4
                for (int64_t r = t0 + lane; r < t1; r += 32) {
                    const TL xr = xs[r - t0];
#pragma unroll
                    for (int q = 0; q < kPer; ++q) {
                        const int c = warp + kWarps * q;
                        if (c < nc) acc[q] += P[r + (int64_t)(c0 + c) * m] * xr;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                TL v = acc[q];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                const int c = warp + kWarps * q;
                if (lane == 0 && c < nc) wb_[f + c0 + c] = __ldcg(zb + f + c0 + c) / Db[f + c0 + c] - v;
            }
        } else {
            const int cb = tk.a * kT, wb = min(kT, k - cb), chunk = tk.b;
            if (tid < 32) {
                TL lcol[kT];
#pragma unroll
                for (int r = 0; r < kT; ++r)
                    lcol[r] = (r > lane && r < wb) ? P[(cb + r) + (int64_t)(cb + lane) * m] : 0.0;
                TL y = lane < wb ? (TL)__ldcg(wb_ + f + cb + lane) : TL(0);
#pragma unroll
                for (int r = kT - 1; r > 0; --r) {
                    const TL xr = __shfl_sync(0xffffffffu, y, r);
                    y -= lcol[r] * xr;
                }
                xb[lane] = y;
                if (chunk == 0 && lane < wb) xv[f + cb + lane] = y;
            }
            __syncthreads();
            bwd_update<1, true>(P, m, cb, wb, xb, chunk * kBwdCols, min(cb, (chunk + 1) * kBwdCols), wb_ + f);
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            int* bc = cnt + band * cstride;
            atomicAdd(bc + tk.done_idx, 1);
            if (tk.pad >= 0) atomicAdd(bc + tk.pad, 1);
        }
    }
}

}  // namespace

void build_solve_dag(const Symbolic& S, SolvePlan& P) {
    P.dag.clear();
    const int32_t ns = S.ns;
    std::vector<int32_t> nfwd(ns, 0), nbwd(ns, 0), child_fwd(ns, 0);
    auto emit = [&](std::vector<std::vector<std::vector<DagTask>>>& ph) {
        size_t maxp = 0;
        for (auto& t : ph) maxp = std::max(maxp, t.size());
        for (size_t q = 0; q < maxp; ++q)
            for (auto& t : ph)
                if (q < t.size()) P.dag.insert(P.dag.end(), t[q].begin(), t[q].end());
    };
    // forward sweep, bottom-up
    for (int32_t l = 0; l < S.nlevels; ++l) {
        std::vector<std::vector<std::vector<DagTask>>> ph;
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p], k = S.k_of(s), m = S.m_of(s), par = S.sparent[s];
            std::vector<std::vector<DagTask>> t;
            int32_t done = 0;
            for (int32_t b = 0; b * kT < k; ++b) {
                const int32_t wb = std::min(kT, k - b * kT);
                const int64_t below = (int64_t)m - b * kT - wb;
                const int32_t nch = std::max<int32_t>(1, (int32_t)((below + kFwdRows - 1) / kFwdRows));
                std::vector<DagTask> step;
                for (int32_t c = 0; c < nch; ++c)
                    step.push_back(DagTask{kSolveFwd, s, b, c, b == 0 ? ns + s : s, b == 0 ? child_fwd[s] : done, s,
                                           par >= 0 ? ns + par : -1});
                done += nch;
                t.push_back(step);
            }
            nfwd[s] = done;
            if (par >= 0) child_fwd[par] += done;
            ph.push_back(std::move(t));
        }
        emit(ph);
    }
    // backward sweep, top-down
    for (int32_t l = S.nlevels - 1; l >= 0; --l) {
        std::vector<std::vector<std::vector<DagTask>>> ph;
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p], k = S.k_of(s), par = S.sparent[s];
            std::vector<std::vector<DagTask>> t;
            const int32_t nci = (k + kT - 1) / kT;
            std::vector<DagTask> init;
            for (int32_t c = 0; c < nci; ++c)
                init.push_back(DagTask{kSolveBwdInit, s, 0, c, par >= 0 ? 2 * ns + par : s,
                                       par >= 0 ? nbwd[par] : nfwd[s], 2 * ns + s, -1});
            t.push_back(init);
            int32_t done = nci;
            for (int32_t b = nci - 1; b >= 0; --b) {
                const int32_t ncb = std::max<int32_t>(1, (b * kT + kBwdCols - 1) / kBwdCols);
                std::vector<DagTask> step;
                for (int32_t c = 0; c < ncb; ++c) step.push_back(DagTask{kSolveBwdStep, s, b, c, 2 * ns + s, done, 2 * ns + s, -1});
                done += ncb;
                t.push_back(step);
            }
            nbwd[s] = done;
            ph.push_back(std::move(t));
        }
        emit(ph);
    }
}

void launch_solve_dag(const DevSym& d, const DagTask* tasks, int ntasks, int* counters, int cstride, const double* L,
                      const double* D, double* w, double* z, double* x, DevStatus* status, int nb, const Strides& bs,
                      int wait_limit, int grid, cudaStream_t st, const float* L32) {
    if (ntasks == 0 || nb == 0) return;
    const uint32_t lim = wait_limit > 0 ? (uint32_t)wait_limit : wait_limit < 0 ? 0u : kSolveWaitLimit;
    const int g = (int)std::min<int64_t>((int64_t)ntasks * nb, grid);
    if (L32)
        k_solve_dag<float><<<g, kThreads, 0, st>>>(d, tasks, ntasks, nb, counters, cstride, L32, D, w, z, x, status, bs,
                                                   lim);
    else
        k_solve_dag<double><<<g, kThreads, 0, st>>>(d, tasks, ntasks, nb, counters, cstride, L, D, w, z, x, status, bs,
                                                    lim);
}

// The solve runs on one stream while the variance kernels of the same factor run on
// another, and a variance CTA takes most of an SM's shared memory.  The solve kernels
// state the same (largest) shared-memory carveout preference as the variance kernels,
// so that an SM configured for a variance CTA can take theirs beside it (their shared
// memory and registers fit in what a variance CTA leaves).
cudaError_t solve_kernel_setup() {
    const int pref = (int)cudaSharedmemCarveoutMaxShared;
    const cudaFuncAttribute a = cudaFuncAttributePreferredSharedMemoryCarveout;
    const void* fns[] = {
        (const void*)k_fwd_step<float>,  (const void*)k_fwd_step<double>,  (const void*)k_bwd_init<float>,
        (const void*)k_bwd_init<double>, (const void*)k_bwd_step<float>,  (const void*)k_bwd_step<double>,
        (const void*)k_fwd_level<float>, (const void*)k_fwd_level<double>, (const void*)k_bwd_level<float>,
        (const void*)k_bwd_level<double>, (const void*)k_fwd_wide,       (const void*)k_bwd_wide,
        (const void*)k_solve_dag<float>, (const void*)k_solve_dag<double>, (const void*)k_sym_residual,
        (const void*)k_norms2,           (const void*)k_axpy,             (const void*)k_permute_in,
        (const void*)k_permute_out};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, a, pref);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t solve_dag_grid(int* grid) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_dag<double>, kThreads, 0);
    *grid = std::max(1, sms * per);
    return e;
}

void launch_zsq_var(int32_t n, const double* z, const double* dinv, int R, double* out, cudaStream_t st) {
    if (R <= 0) return;
    k_zsq_var<<<R, kThreads, 0, st>>>(n, z, dinv, out);
}

void launch_reciprocal(int32_t n, const double* D, double* dinv, cudaStream_t st) {
    if (n <= 0) return;
    k_reciprocal<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(n, D, dinv);
}

void launch_set_units(int32_t n, const int32_t* pos, int R, double* w, cudaStream_t st) {
    if (R <= 0) return;
    k_set_units<<<(R + 127) / 128, 128, 0, st>>>(n, pos, R, w);
}

void launch_refined_var(int32_t n, const double* v, const double* r, const int32_t* idx, int R, double* out,
                        cudaStream_t st) {
    if (R <= 0) return;
    k_refined_var<<<R, kThreads, 0, st>>>(n, v, r, idx, out);
}

void launch_sym_residual(int32_t n, const int64_t* cp, const int32_t* ri, const double* va, const double* x,
                         double* r, int nb, int64_t nnz, cudaStream_t st) {
    if (n == 0 || nb == 0) return;
    int grid = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, std::max(1, 152 * 8 / nb));
    k_sym_residual<<<dim3(grid, nb), 256, 0, st>>>(n, cp, ri, va, x, r, nnz);
}

void launch_norms2(int32_t n, const double* a, const double* b, double* out, int nb, cudaStream_t st) {
    if (n == 0 || nb == 0) return;
    k_norms2<<<dim3(std::min(1024, (n + 255) / 256), nb), 256, 0, st>>>(n, a, b, out);
}

void launch_axpy(int32_t n, const double* dx, double* x, int nb, cudaStream_t st) {
    if (n == 0 || nb == 0) return;
    k_axpy<<<dim3(std::min(1024, (n + 255) / 256), nb), 256, 0, st>>>(n, dx, x);
}

void launch_permute_in(int32_t n, const int32_t* perm, const double* b, double* w, int nb, cudaStream_t st) {
    if (n == 0 || nb == 0) return;
    k_permute_in<<<dim3(std::min(1024, (n + 255) / 256), nb), 256, 0, st>>>(n, perm, b, w);
}

void launch_permute_out(int32_t n, const int32_t* perm, const double* w, double* x, int nb, cudaStream_t st) {
    if (n == 0 || nb == 0) return;
    k_permute_out<<<dim3(std::min(1024, (n + 255) / 256), nb), 256, 0, st>>>(n, perm, w, x);
}

void build_solve_plan(const Symbolic& S, SolvePlan& P, int batch, const uint8_t* wide) {
    P = SolvePlan();
    for (int32_t l = 0; l < S.nlevels; ++l) {
        int32_t kmax = 0;
        int64_t work = 0;
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p];
            const int64_t k = S.k_of(s), m = S.m_of(s);
            kmax = std::max<int32_t>(kmax, (int32_t)k);
            work = std::max(work, k * m - k * k / 2);
        }
        if (batch > 1 && work <= (int64_t)((kmax + kT - 1) / kT) * kFuseFmaPerStep) {  // one launch per sweep
            Launch lf{10, 0, (int64_t)P.fwd_items.size() / 2, 0};
            Launch lb{11, 0, (int64_t)P.bwd_items.size() / 2, 0};
            for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
                const int32_t s = S.level_list[p];
                if (S.k_of(s) == 0) continue;
                P.fwd_items.push_back(s); P.fwd_items.push_back(0); lf.count++;
                P.bwd_items.push_back(s); P.bwd_items.push_back(0); lb.count++;
            }
            P.fwd_launches.push_back(lf);
            P.bwd_level_launches.push_back({lb});
            continue;
        }
        const int32_t nsteps = (kmax + kT - 1) / kT;
        std::vector<Launch> fw, bw;
        // wide steps of 128 columns for the flagged supernodes (kinds 15 and 16)
        for (int32_t b = 0; wide && b * kW < kmax; ++b) {
            Launch lf{15, b, (int64_t)P.fwd_items.size() / 2, 0};
            Launch lb{16, b, (int64_t)P.bwd_items.size() / 2, 0};
            for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
                const int32_t s = S.level_list[p], k = S.k_of(s), m = S.m_of(s);
                if (!wide[s] || k <= b * kW) continue;
                const int32_t wb = std::min(kW, k - b * kW);
                const int64_t below = (int64_t)m - b * kW - wb;
                const int32_t nch = std::max<int32_t>(1, (int32_t)((below + kFwdRowsW - 1) / kFwdRowsW));
                for (int32_t c = 0; c < nch; ++c) { P.fwd_items.push_back(s); P.fwd_items.push_back(c); lf.count++; }
                const int32_t ncb = std::max<int32_t>(1, (b * kW + kBwdColsW - 1) / kBwdColsW);
                for (int32_t c = 0; c < ncb; ++c) { P.bwd_items.push_back(s); P.bwd_items.push_back(c); lb.count++; }
            }
            if (lf.count) fw.push_back(lf);
            if (lb.count) bw.push_back(lb);
        }
        for (int32_t b = 0; b < nsteps; ++b) {
            Launch lf{4, b, (int64_t)P.fwd_items.size() / 2, 0};
            Launch lb{6, b, (int64_t)P.bwd_items.size() / 2, 0};
            for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
                const int32_t s = S.level_list[p], k = S.k_of(s), m = S.m_of(s);
                if (k <= b * kT || (wide && wide[s])) continue;
                const int32_t wb = std::min(kT, k - b * kT);
                const int64_t below = (int64_t)m - b * kT - wb;
                const int32_t nch = std::max<int32_t>(1, (int32_t)((below + kFwdRows - 1) / kFwdRows));
                for (int32_t c = 0; c < nch; ++c) { P.fwd_items.push_back(s); P.fwd_items.push_back(c); lf.count++; }
                const int32_t ncb = std::max<int32_t>(1, (b * kT + kBwdCols - 1) / kBwdCols);
                for (int32_t c = 0; c < ncb; ++c) { P.bwd_items.push_back(s); P.bwd_items.push_back(c); lb.count++; }
            }
            if (lf.count) fw.push_back(lf);
            if (lb.count) bw.push_back(lb);
        }
        Launch li{5, 0, (int64_t)P.bwd_items.size() / 2, 0};
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p], k = S.k_of(s);
            const int32_t nch = std::max<int32_t>(1, (k + kT - 1) / kT);
            for (int32_t c = 0; c < nch; ++c) { P.bwd_items.push_back(s); P.bwd_items.push_back(c); li.count++; }
        }
        P.fwd_launches.insert(P.fwd_launches.end(), fw.begin(), fw.end());
        // backward of level l: init, then the block steps in descending order
        std::vector<Launch> lvl;
        lvl.push_back(li);
        for (auto it = bw.rbegin(); it != bw.rend(); ++it) lvl.push_back(*it);
        P.bwd_level_launches.push_back(lvl);
    }
    // backward levels run top-down
    for (auto it = P.bwd_level_launches.rbegin(); it != P.bwd_level_launches.rend(); ++it)
        P.bwd_launches.insert(P.bwd_launches.end(), it->begin(), it->end());
    P.bwd_level_launches.clear();
}

template <typename TL>
void launch_solve_step_t(const DevSym& d, const Launch& l, const int32_t* fwd_items, const int32_t* bwd_items,
                         const TL* L, const double* D, double* w, double* z, double* x, int nb, const Strides& bs,
                         cudaStream_t st, const WideArgs* wa) {
    const dim3 g(l.count, nb);
    if constexpr (std::is_same<TL, float>::value) {
        if (l.kind == 15 && wa) {
            k_fwd_wide<<<g, kThreads, 0, st>>>(d, fwd_items + 2 * l.off, l.step, L, *wa, w, z, bs);
            return;
        }
        if (l.kind == 16 && wa) {
            k_bwd_wide<<<g, kThreads, 0, st>>>(d, bwd_items + 2 * l.off, l.step, L, *wa, w, x, bs);
            return;
        }
    }
    switch (l.kind) {
        case 4: k_fwd_step<TL><<<g, kThreads, 0, st>>>(d, fwd_items + 2 * l.off, l.step, L, w, z, bs); break;
        case 5: k_bwd_init<TL><<<g, kThreads, 0, st>>>(d, bwd_items + 2 * l.off, L, D, z, x, w, bs); break;
        case 10: k_fwd_level<TL><<<g, kThreads, 0, st>>>(d, fwd_items + 2 * l.off, L, w, z, bs); break;
        case 11: k_bwd_level<TL><<<g, kThreads, 0, st>>>(d, bwd_items + 2 * l.off, L, D, z, x, w, bs); break;
        default: k_bwd_step<TL><<<g, kThreads, 0, st>>>(d, bwd_items + 2 * l.off, l.step, L, w, x, bs); break;
    }
}

void launch_solve_step(const DevSym& d, const Launch& l, const int32_t* fwd_items, const int32_t* bwd_items,
                       const double* L, const double* D, double* w, double* z, double* x, int nb,
                       const Strides& bs, cudaStream_t st, const float* L32, const WideArgs* wa) {
    if (l.count == 0 || nb == 0) return;
    if (L32) launch_solve_step_t<float>(d, l, fwd_items, bwd_items, L32, D, w, z, x, nb, bs, st, wa);
    else launch_solve_step_t<double>(d, l, fwd_items, bwd_items, L, D, w, z, x, nb, bs, st, wa);
}

}  // namespace spi
