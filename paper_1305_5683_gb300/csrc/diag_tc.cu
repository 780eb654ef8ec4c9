// diag_tc.cu -- the mixed form's variances on the 5th-generation tensor cores
// for the large supernodes near the root (paper Sec. 3.3.1 and Sec. 4.3: the
// pruned forward solves z = L^-1 e_i, right-hand sides in blocks).
//
// The supernodes on the tensor cores are those with at least `min_k` pivots
// and all their ancestors (an upward-closed set T).  The SIMT kernel
// (k_diag_inv_f32) walks every block's paths below T first and leaves, in the
// block's workspace Z, the right-hand sides' values on T's rows; this kernel
// then walks the block's supernodes in T, one CTA per block of B <= 128
// right-hand sides, as dense products on the tensor cores.
//
// Supernode s (k pivots, m rows, unit-lower diagonal block L11, rows below
// L21) maps the incoming values of its own rows to z_own = L11^-1 z_in and
// then subtracts L21 z_own from the rows below.  The own rows are taken in
// tiles of 128: with X_ii the inverse of the 128 x 128 diagonal block of tile
// i (blocked forward substitution),
//     z_i = X_ii z_in_i + sum_{j<i} W_ij z_j,   W_ij = -X_ii L_ij,
// one product over K = 128 (i + 1) columns whose right operand is the block's
// Z rows 0 .. 128 (i + 1) of s (tiles j < i already final, tile i still the
// incoming values).  The rows below take z_below += (-L21) z_own over K = k.
// The left operands [X_ii, W_ij] and -L21 are prepared once per
// factorization (k_diag_tinv, k_diag_pack) as TF32 hi/lo pairs in 128 x 32
// tiles laid out exactly as the MMA reads them, and each tile pair reaches
// shared memory by one TMA tensor copy (cp.async.bulk.tensor).  The right
// operand (a 32-row chunk of Z, up to 128 right-hand sides) is split into hi
// and lo by the CTA's threads.  Products are 3 x TF32 (hi*hi, hi*lo, lo*hi)
// with FP32 accumulation in tensor memory, hi*hi restarted every kTcFlush
// chunks and added into a running sum with round-to-nearest (as in the
// Schur kernel).  Each own tile's z_i is written back to Z and its squares,
// scaled by 1/d, are summed over the tile's rows in FP32 (32 per warp, a
// butterfly across lanes) and added to the variances in FP64.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "spi_internal.cuh"
#include "tcgen05.cuh"

namespace spi {
namespace {

constexpr int kDtM = kDiagTcRows;       // rows of a tile (the MMA's M)
constexpr int kDtK = kDiagTcK;          // K columns of a tile
constexpr int kDtTile = kDtM * kDtK;    // floats of one TF32 plane of a tile (16 KB)
constexpr int kDtStage = 4 * kDtTile;   // A hi, A lo, B hi, B lo
constexpr int kDtThreads = 128;
// 3 stages, variances [128] (double), per-warp column sums [4][128], 6 mbarriers,
// the tensor-memory address and padding
constexpr size_t kDtSmem = 3 * kDtStage * sizeof(float) + 128 * sizeof(double) + 4 * 128 * sizeof(float) + 64;
constexpr size_t kTinvSmem = 2 * kDtM * (kDtM + 1) * sizeof(float);
constexpr size_t kPackSmem = (kDtM * (kDtM + 1) + kDtM * (kDtK + 1)) * sizeof(float);

struct DiagTcArgs {
    const uint8_t* tc;    // [ns] 1 = supernode on the tensor cores
    const int64_t* tptr;  // [ns] first packed tile of the supernode
    int64_t npt;          // packed tiles per band
};

// Inverse of the unit-lower 128 x 128 diagonal block of own row tile i of s
// (rows and columns [128 i, 128 i + w), zero beyond w): thread j computes column
// j by forward substitution, X[r][j] = -sum_{c=j}^{r-1} L[r][c] X[c][j].
__global__ void __launch_bounds__(kDtM) k_diag_tinv(DevSym d, const int32_t* __restrict__ dtiles, int64_t ndt,
                                                     const float* __restrict__ L, float* __restrict__ xinv,
                                                     int64_t bsL) {
    const int64_t t = blockIdx.x;
    L += blockIdx.y * bsL;
    xinv += ((int64_t)blockIdx.y * ndt + t) * (kDtM * kDtM);
    extern __shared__ float tsh[];
    float* Ls = tsh;                      // [128][129], row r, column c < r
    float* Xs = tsh + kDtM * (kDtM + 1);  // [128][129], X[r][j]
    const int s = dtiles[2 * t], i = dtiles[2 * t + 1];
    const int k = d.sfirst[s + 1] - d.sfirst[s];
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const float* P = L + d.lptr[s];
    const int r0 = i * kDtM, w = min(kDtM, k - r0);
    const int j = threadIdx.x;
    for (int c = 0; c < kDtM; ++c) {
        Ls[j * (kDtM + 1) + c] = (j < w && c < j) ? P[(r0 + j) + (int64_t)(r0 + c) * m] : 0.f;
        Xs[c * (kDtM + 1) + j] = (c == j && j < w) ? 1.f : 0.f;
    }
    __syncthreads();
    if (j < w) {
        for (int r = j + 1; r < w; ++r) {
            const float* lr = Ls + r * (kDtM + 1);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            int c = j;
            for (; c + 3 < r; c += 4) {
                a0 = fmaf(lr[c], Xs[c * (kDtM + 1) + j], a0);
                a1 = fmaf(lr[c + 1], Xs[(c + 1) * (kDtM + 1) + j], a1);
                a2 = fmaf(lr[c + 2], Xs[(c + 2) * (kDtM + 1) + j], a2);
                a3 = fmaf(lr[c + 3], Xs[(c + 3) * (kDtM + 1) + j], a3);
            }
            for (; c < r; ++c) a0 = fmaf(lr[c], Xs[c * (kDtM + 1) + j], a0);
            Xs[r * (kDtM + 1) + j] = -((a0 + a1) + (a2 + a3));
        }
    }
    __syncthreads();
    for (int r = 0; r < kDtM; ++r) xinv[r * kDtM + j] = Xs[r * (kDtM + 1) + j];
}

// a = hi + lo with two TF32 values
__device__ __forceinline__ void tc_split2(float a, float& hi, float& lo) {
    hi = tc_tf32(a);
    lo = tc_tf32(a - hi);
}

// One packed left-operand tile (supernode s, row tile rt, K chunk c): 128 rows x
// 32 columns as TF32 hi and lo planes in the K-major core-matrix layout:
//   own tiles (rt < T): columns [128 rt, 128 rt + 128) hold X_rt, columns below
//     128 rt hold W = -X_rt L[rows of rt][those columns];
//   tiles below (rt >= T): -L21 rows [128 (rt - T), +128), columns 32 c ...
__global__ void __launch_bounds__(kDtM) k_diag_pack(DevSym d, const int32_t* __restrict__ ptiles, int64_t npt,
                                                     const int32_t* __restrict__ xptr, int64_t ndt,
                                                     const float* __restrict__ L, const float* __restrict__ xinv,
                                                     float* __restrict__ pack, int64_t bsL) {
    const int64_t t = blockIdx.x;
    const int band = blockIdx.y;
    L += band * bsL;
    xinv += (int64_t)band * ndt * (kDtM * kDtM);
    float* dst = pack + ((int64_t)band * npt + t) * (2 * kDtTile);
    extern __shared__ float psh[];
    const int s = ptiles[4 * t], rt = ptiles[4 * t + 1], c = ptiles[4 * t + 2];
    const int k = d.sfirst[s + 1] - d.sfirst[s];
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const float* P = L + d.lptr[s];
    const int T = (k + kDtM - 1) / kDtM;
    const int tid = threadIdx.x;
    float v[kDtK];
    if (rt >= T) {
        const int64_t row = k + (int64_t)(rt - T) * kDtM + tid;
#pragma unroll
        for (int q = 0; q < kDtK; ++q) {
            const int col = c * kDtK + q;
            v[q] = (row < m && col < k) ? -P[row + (int64_t)col * m] : 0.f;
        }
    } else {
        const float* X = xinv + (int64_t)(xptr[s] + rt) * (kDtM * kDtM);
        float* Xs = psh;                       // [128][129]
        float* Lc = psh + kDtM * (kDtM + 1);   // [128][33]
        if (c >= 4 * rt) {
            const int c0 = (c - 4 * rt) * kDtK;
            for (int r = 0; r < kDtM; ++r)
                if (tid < kDtK) Xs[r * (kDtM + 1) + tid] = X[r * kDtM + c0 + tid];
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kDtK; ++q) v[q] = Xs[tid * (kDtM + 1) + q];
        } else {
            const int r0 = rt * kDtM, w = min(kDtM, k - r0);
            for (int r = 0; r < kDtM; ++r) Xs[r * (kDtM + 1) + tid] = X[r * kDtM + tid];
            for (int q = 0; q < kDtK; ++q)
                Lc[tid * (kDtK + 1) + q] = tid < w ? P[(r0 + tid) + (int64_t)(c * kDtK + q) * m] : 0.f;
            __syncthreads();
            float acc[kDtK];
#pragma unroll
            for (int q = 0; q < kDtK; ++q) acc[q] = 0.f;
            for (int p = 0; p < w; ++p) {
                const float x = Xs[tid * (kDtM + 1) + p];
#pragma unroll
                for (int q = 0; q < kDtK; ++q) acc[q] = fmaf(x, Lc[p * (kDtK + 1) + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < kDtK; ++q) v[q] = -acc[q];
        }
    }
#pragma unroll
    for (int q4 = 0; q4 < kDtK / 4; ++q4) {
        const int o = tc_kmajor_off(tid, 4 * q4) >> 2;
        float4 h, l;
        tc_split2(v[4 * q4 + 0], h.x, l.x);
        tc_split2(v[4 * q4 + 1], h.y, l.y);
        tc_split2(v[4 * q4 + 2], h.z, l.z);
        tc_split2(v[4 * q4 + 3], h.w, l.w);
        *reinterpret_cast<float4*>(dst + o) = h;
        *reinterpret_cast<float4*>(dst + kDtTile + o) = l;
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

// One tile pair (hi and lo planes, 32 KB) of the packed operands: the tensor map
// views them as [slices][256][4] floats, eight 4 KB slices per tile pair.
__device__ __forceinline__ void tma_tile_pair(uint32_t dst, const CUtensorMap* map, int32_t slice, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(0), "r"(slice), "r"(mbar)
        : "memory");
}

// Sum over the warp's 32 lanes of each of the 32 values v[0..31]; lane j returns
// the sum for index j (a butterfly: at each step a lane keeps half of its values
// and adds its partner's copy of that half).
__device__ __forceinline__ float lane_column_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool up = (lane & sft) != 0;
#pragma unroll
        for (int i = 0; i < sft; ++i) {
            const float send = up ? v[i] : v[i + sft];
            const float keep = up ? v[i + sft] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
        }
    }
    return v[0];
}

struct DiagArgsTc {
    int32_t B;
    const int32_t *order, *blk_ptr, *uptr, *us, *ulo, *uhi, *uzoff, *rel, *rhs_out;
    const int64_t *urel, *zbase;
    float* Z;
};

// Tensor memory of a CTA: two hi*hi accumulators A0, A1 taking the K chunks of
// a tile in groups of kTcFlush (group j in A_(j mod 2)), X the cross terms of
// the whole tile, S the running sum of the finished groups (an FP32
// round-to-nearest add on the CUDA cores while the next group accumulates in
// the other buffer).
constexpr uint32_t kDtA1 = 128, kDtX = 256, kDtS = 384;
constexpr int kDtStages = 3;

__device__ __forceinline__ void tc_add32(uint32_t (&r)[32], const uint32_t (&t)[32]) {
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(t[j]));
}

// Columns n0 .. n0 + 31 of one Z row (those below nbu): 16-byte accesses when the
// row segment is 16-byte aligned (lo0 a multiple of 4), else 4-byte ones.
__device__ __forceinline__ void z_store32(float* zr, const float (&v)[32], int n0, int nbu, bool vec) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int n = n0 + 4 * i;
        if (vec && n + 3 < nbu) {
            *reinterpret_cast<float4*>(zr + n) = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (n + e < nbu) zr[n + e] = v[4 * i + e];
        }
    }
}
__device__ __forceinline__ void z_load32(const float* zr, float (&v)[32], int n0, int nbu, bool vec) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int n = n0 + 4 * i;
        if (vec && n + 3 < nbu) {
            const float4 x = *reinterpret_cast<const float4*>(zr + n);
            v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) v[4 * i + e] = n + e < nbu ? zr[n + e] : 0.f;
        }
    }
}

// One CTA per block of right-hand sides.  The K chunks of all its tiles form one
// sequence (supernode by supernode, tile by tile), which is also the order of
// their packed left operands (consecutive within a supernode): chunk g uses
// stage g mod 3 of a 3-stage ring.  Thread 0 copies chunk g + 1's left operand
// while the CTA stages chunk g's right operand (split into TF32 hi and lo), then
// issues chunk g's 4 k-steps x 3 MMAs and commits them to the stage's mbarrier.
__global__ void __launch_bounds__(kDtThreads, 1)
    k_diag_inv_tc(DevSym d, DiagArgsTc p, DiagTcArgs ta, const double* __restrict__ D, double* __restrict__ out,
                  Strides bs, DevStatus* status, uint32_t wait_limit, const __grid_constant__ CUtensorMap tmap) {
    const int band = blockIdx.y;
    D += band * bs.n;
    out += band * bs.out;
    extern __shared__ __align__(1024) float dsm[];
    double* var = reinterpret_cast<double*>(dsm + kDtStages * kDtStage);  // [128]
    float* red = reinterpret_cast<float*>(var + 128);                      // [4][128]
    uint64_t* full = reinterpret_cast<uint64_t*>(red + 4 * 128);           // [3] operand copies
    uint64_t* done = full + kDtStages;                                     // [3] MMA commits
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + kDtStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int B = p.B;
    const int b = p.order[blockIdx.x];
    float* Z = p.Z + band * bs.Z + p.zbase[b];
    const int r0b = p.blk_ptr[b], nr = p.blk_ptr[b + 1] - r0b;
    const int64_t tile_band = (int64_t)band * ta.npt;
    const int u0 = p.uptr[b], u1 = p.uptr[b + 1];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem_u32(tmem_slot)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < 2 * kDtStages; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc_smem_u32(full + q)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int q = tid; q < 128; q += kDtThreads) var[q] = q < nr ? out[p.rhs_out[r0b + q]] : 0.0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    uint32_t g = 0;  // chunks whose MMAs were committed
    // ---- thread 0's operand copies, one chunk ahead of the MMAs
    uint32_t issued = 0;
    int pu = u0 - 1;
    int64_t pid = 0, pend = 0;
    auto issue_next = [&]() -> bool {
        while (pid == pend) {
            if (++pu >= u1) return true;  // nothing left to copy
            const int s = p.us[pu];
            if (!ta.tc[s]) continue;
            const int k = d.sfirst[s + 1] - d.sfirst[s];
            const int m = (int)(d.srowptr[s + 1] - d.srowptr[s]);
            const int T = (k + kDtM - 1) / kDtM, R = (m - k + kDtM - 1) / kDtM, nch = (k + kDtK - 1) / kDtK;
            pid = tile_band + ta.tptr[s];
            pend = pid + diag_tc_tile_offset(T, nch, T + R);
        }
        const uint32_t st = issued % kDtStages;
        // the stage's previous chunk (issued - 3) must have been read by its MMAs
        if (issued >= kDtStages && !tc_wait(done + st, ((issued - kDtStages) / kDtStages) & 1u, wait_limit)) return false;
        mbar_expect_tx(tc_smem_u32(full + st), 2 * kDtTile * sizeof(float));
        tma_tile_pair(tc_smem_u32(dsm + st * kDtStage), &tmap, (int32_t)(8 * pid), tc_smem_u32(full + st));
        ++pid;
        ++issued;
        return true;
    };
    if (tid == 0) ok = issue_next();
    for (int u = u0; u < u1; ++u) {
        if (__syncthreads_or(!ok)) { ok = false; break; }
        const int s = p.us[u];
        if (!ta.tc[s]) continue;
        const int lo0 = p.ulo[u], nbu = p.uhi[u] - lo0, zo = p.uzoff[u];
        const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
        const int m = (int)(d.srowptr[s + 1] - d.srowptr[s]);
        const int32_t* rel = p.rel + p.urel[u];
        const int N = (nbu + 31) & ~31;
        const bool vec = (lo0 & 3) == 0;
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(kDtM >> 4) << 24);
        const int T = (k + kDtM - 1) / kDtM, R = (m - k + kDtM - 1) / kDtM;
        const int nitems = N * (kDtK / 4);  // (right-hand side, 4-row group) pairs of one chunk
        float pre[8][4];                    // a chunk of Z (rows of s, right-hand sides [lo0, lo0 + N))
        auto fetch = [&](int c, int kext) {
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int item = tid + it * kDtThreads;
                const int n = item % N, kq = item / N;
                const int kr = c * kDtK + kq * 4;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    pre[it][e] = (item < nitems && n < nbu && kr + e < kext)
                                     ? Z[(int64_t)(zo + kr + e) * B + lo0 + n] : 0.f;
            }
        };
        bool prefetched = false;
        for (int tile = 0; tile < T + R && ok; ++tile) {
            const bool own = tile < T;
            const int rows0 = own ? tile * kDtM : k + (tile - T) * kDtM;
            const int nrow = min(kDtM, (own ? k : m) - rows0);
            const int kext = own ? min(kDtM * (tile + 1), k) : k;
            const int nck = (kext + kDtK - 1) / kDtK;
            if (!prefetched) fetch(0, kext);
            prefetched = false;
            for (int c = 0; c < nck; ++c) {
                const uint32_t gc = g, st = gc % kDtStages;
                float* A = dsm + st * kDtStage;
                float* Bh = A + 2 * kDtTile;
                float* Bl = Bh + kDtTile;
                // the stage's right operand buffers: free once chunk gc - 3's MMAs are done
                if (gc >= kDtStages) ok = tc_wait(done + st, ((gc - kDtStages) / kDtStages) & 1u, wait_limit) && ok;
                if (tid == 0 && ok && issued == gc + 1) ok = issue_next();
                if (__syncthreads_or(!ok)) { ok = false; break; }
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int item = tid + it * kDtThreads;
                    if (item < nitems) {
                        const int n = item % N, kq = item / N;
                        const int o = tc_kmajor_off(n, 4 * kq) >> 2;
                        float4 h, l;
                        tc_split2(pre[it][0], h.x, l.x);
                        tc_split2(pre[it][1], h.y, l.y);
                        tc_split2(pre[it][2], h.z, l.z);
                        tc_split2(pre[it][3], h.w, l.w);
                        *reinterpret_cast<float4*>(Bh + o) = h;
                        *reinterpret_cast<float4*>(Bl + o) = l;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                if (tid == 0) {
                    if (!tc_wait(full + st, (gc / kDtStages) & 1u, wait_limit)) {
                        ok = false;
                    } else {
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t acc = tmem + ((c >> 2) & 1 ? kDtA1 : 0u);
#pragma unroll
                        for (int kk = 0; kk < kDtK / 8; ++kk) {
                            const uint32_t ko = kk * 256;
                            const uint64_t ah = tc_desc(tc_smem_u32(A) + ko), al = tc_desc(tc_smem_u32(A + kDtTile) + ko);
                            const uint64_t bh = tc_desc(tc_smem_u32(Bh) + ko), bl = tc_desc(tc_smem_u32(Bl) + ko);
                            tc_mma(tmem + kDtX, ah, bl, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                            tc_mma(tmem + kDtX, al, bh, idesc, 1u);
                            tc_mma(acc, ah, bh, idesc, ((c & 3) > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    // the commit tracks every MMA issued before it, and arrives even if none was
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(tc_smem_u32(done + st)));
                }
                ++g;
                if ((c & 3) == 0 && c > 0) {
                    // group c/4 - 1 ended with chunk gc - 1: S (+)= its buffer while this group
                    // accumulates in the other one
                    const uint32_t gp = gc - 1;
                    if (ok) ok = tc_wait(done + gp % kDtStages, (gp / kDtStages) & 1u, wait_limit);
                    if (__syncthreads_or(!ok)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t row = (uint32_t)(warp * 32) << 16;
                    const uint32_t prev = ((c >> 2) - 1) & 1 ? kDtA1 : 0u;
                    for (int q = 0; q < N / 32; ++q) {
                        uint32_t a[32], sv[32];
                        tc_ld32(tmem + row + prev + q * 32, a);
                        if (c > 4) {
                            tc_ld32(tmem + row + kDtS + q * 32, sv);
                            tc_add32(a, sv);
                        }
                        tc_st32(tmem + row + kDtS + q * 32, a);
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;");
                }
                if (c + 1 < nck) {
                    fetch(c + 1, kext);
                } else if (!own && tile + 1 < T + R) {
                    fetch(0, kext);  // the next tile below takes the same right operand
                    prefetched = true;
                }
            }
            // thread 0 alone may have seen a wait run out (its operand copy): every exit is
            // decided collectively, so that all threads leave the loops together
            if (__syncthreads_or(!ok)) { ok = false; break; }
            const uint32_t gl = g - 1;
            ok = tc_wait(done + gl % kDtStages, (gl / kDtStages) & 1u, wait_limit);
            if (__syncthreads_or(!ok)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            // result = S (groups before the last) + the last group's buffer + X
            const int jl = (nck - 1) >> 2;
            const int row = warp * 32 + lane;
            const int lr = rows0 + row;
            const bool rv = row < nrow;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            const float dinv = (own && rv) ? (float)(1.0 / D[f + lr]) : 0.f;
            float* zrow = Z + (int64_t)(own ? zo + lr : (rv ? rel[lr - k] : 0)) * B + lo0;
            for (int q = 0; q < N / 32; ++q) {
                uint32_t r[32], t[32];
                tc_ld32(taddr + (jl & 1 ? kDtA1 : 0u) + q * 32, r);
                tc_ld32(taddr + kDtX + q * 32, t);
                tc_add32(r, t);
                if (jl > 0) {
                    tc_ld32(taddr + kDtS + q * 32, t);
                    tc_add32(r, t);
                }
                float v[32];
                if (own) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) v[jj] = __uint_as_float(r[jj]);
                    if (rv) z_store32(zrow, v, q * 32, nbu, vec);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) v[jj] = (rv && q * 32 + jj < nbu) ? v[jj] * v[jj] * dinv : 0.f;
                    red[warp * 128 + q * 32 + lane] = lane_column_sum(v, lane);
                } else if (rv) {
                    z_load32(zrow, v, q * 32, nbu, vec);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) v[jj] += __uint_as_float(r[jj]);
                    z_store32(zrow, v, q * 32, nbu, vec);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            if (own)
                for (int n = tid; n < nbu; n += kDtThreads)
                    var[lo0 + n] += ((double)red[n] + (double)red[128 + n]) + ((double)red[256 + n] + (double)red[384 + n]);
        }
        if (!ok) break;
    }
    if (!ok) {
        // a wait ran out: report it, let the copies and products in flight finish
        // (again bounded), then release tensor memory and leave the variances
        if (tid == 0) {
            atomicOr(&status->flags, FLAG_TIMEOUT);
            for (uint32_t q = issued > kDtStages ? issued - kDtStages : 0; q < issued; ++q)
                tc_wait(full + q % kDtStages, (q / kDtStages) & 1u);
            if (g > 0) tc_wait(done + (g - 1) % kDtStages, ((g - 1) / kDtStages) & 1u);
        }
    }
    __syncthreads();
    if (ok)
        for (int q = tid; q < nr; q += kDtThreads) out[p.rhs_out[r0b + q]] = var[q];
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

}  // namespace

cudaError_t diag_tc_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_diag_inv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDtSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_diag_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_diag_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPackSmem);
}

size_t diag_tc_pack_floats(int64_t npt) { return (size_t)npt * 2 * kDtTile; }
size_t diag_tc_xinv_floats(int64_t ndt) { return (size_t)ndt * kDtM * kDtM; }

// The tensor map over the packed tiles of `bands` bands: [slices][256][4]
// floats, 16-byte rows, 4 KB slices, eight slices per tile pair; one box is a
// whole tile pair (4 x 256 x 8).  cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query (no link against the driver library).
cudaError_t diag_tc_tensor_map(float* pack, int64_t npt, int bands, void* map_out) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const cuuint64_t dims[3] = {4, 256, (cuuint64_t)npt * bands * 8};
    const cuuint64_t strides[2] = {16, 4096};
    const cuuint32_t box[3] = {4, 256, 8};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, pack, dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

void launch_diag_tc_pack(const DevSym& d, const DevDiagTc& p, const float* L32, int nb, const Strides& bs,
                         cudaStream_t st) {
    if (p.ntc == 0 || nb == 0) return;
    k_diag_tinv<<<dim3((unsigned)p.ndt, nb), kDtM, kTinvSmem, st>>>(d, p.dtiles, p.ndt, L32, p.xinv, bs.L);
    k_diag_pack<<<dim3((unsigned)p.npt, nb), kDtM, kPackSmem, st>>>(d, p.ptiles, p.npt, p.xptr, p.ndt, L32, p.xinv,
                                                                     p.pack, bs.L);
}

void launch_diag_inv_tc(const DevSym& d, const DevDiagPlan& dp, const DevDiagTc& p, const double* D, double* out,
                        int nb, const Strides& bs, DevStatus* status, int wait_limit, cudaStream_t st) {
    if (p.ntc == 0 || dp.nblocks == 0 || nb == 0) return;
    const uint32_t lim = wait_limit > 0 ? (uint32_t)wait_limit : wait_limit < 0 ? 0u : kTcWaitLimit;
    DiagArgsTc a{dp.B, dp.order, dp.blk_ptr, dp.uptr, dp.us, dp.ulo, dp.uhi, dp.uzoff, dp.rel, dp.rhs_out,
                 dp.urel, dp.zbase, reinterpret_cast<float*>(dp.Z)};
    DiagTcArgs t{p.tc, p.tptr, p.npt};
    k_diag_inv_tc<<<dim3(dp.nblocks, nb), kDtThreads, kDtSmem, st>>>(
        d, a, t, D, out, bs, status, lim, *reinterpret_cast<const CUtensorMap*>(p.tmap));
}

}  // namespace spi
