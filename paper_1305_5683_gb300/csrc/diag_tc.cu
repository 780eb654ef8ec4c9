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
constexpr size_t kTinvSmem = (2 * kDtM * (kDtM + 1) + 3 * 32 * 33) * sizeof(float);
constexpr size_t kPackSmem = (kDtM * (kDtM + 1) + kDtM * (kDtK + 1)) * sizeof(float);

struct DiagTcArgs {
    const uint8_t* tc;    // [ns] 1 = supernode on the tensor cores
    const int64_t* tptr;  // [ns] first packed tile of the supernode
    int64_t npt;          // packed tiles per band
};

// acc[q] += sum_k A[r][k] B[k][c0 + 4 q] for the 32 x 32 blocks A, B in shared memory
// (row strides lda, ldb): thread t takes row r = t % 32 and the columns c0 + 4 q,
// c0 = t / 32 -- a warp reads one B entry at a time (broadcast) and A with lanes on rows.
__device__ __forceinline__ void mm32_acc(float (&acc)[8], const float* A, int lda, const float* B, int ldb) {
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
        const float a = A[r * lda + k];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fmaf(a, B[k * ldb + c0 + 4 * q], acc[q]);
    }
}

// Inverse X of the unit-lower 128 x 128 diagonal block of own row tile i of s (rows
// and columns [128 i, 128 i + w), zero beyond w), in 32 x 32 blocks: warp b inverts
// diagonal block b by forward substitution (lane j holds column j in registers),
// then the blocks below the diagonal follow by distance d = i - j,
// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj, as products of 32 x 32 blocks by all four
// warps (the blocks of one distance depend only on shorter distances).
constexpr int kTinvLd = kDtM + 1;
__global__ void __launch_bounds__(kDtM) k_diag_tinv(DevSym d, const int32_t* __restrict__ dtiles, int64_t ndt,
                                                     const float* __restrict__ L, float* __restrict__ xinv,
                                                     int64_t bsL) {
    const int64_t t = blockIdx.x;
    L += blockIdx.y * bsL;
    xinv += ((int64_t)blockIdx.y * ndt + t) * (kDtM * kDtM);
    extern __shared__ float tsh[];
    float* Ls = tsh;                     // [128][129], row r, column c < r
    float* Xs = tsh + kDtM * kTinvLd;    // [128][129], X[r][j]
    float* Tb = Xs + kDtM * kTinvLd;     // three [32][33] sums of one distance
    const int s = dtiles[2 * t], i = dtiles[2 * t + 1];
    const int k = d.sfirst[s + 1] - d.sfirst[s];
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const float* P = L + d.lptr[s];
    const int r0 = i * kDtM, w = min(kDtM, k - r0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c0 = 0; c0 < kDtM; c0 += 16) {  // thread = row, 16 loads in flight
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q] = (tid < w && c0 + q < tid) ? P[(r0 + tid) + (int64_t)(r0 + c0 + q) * m] : 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) Ls[tid * kTinvLd + c0 + q] = v[q];
    }
    for (int e = tid; e < kDtM * kTinvLd; e += kDtM) Xs[e] = 0.f;
    __syncthreads();
    {
        const int b = warp, gj = 32 * b + lane;
        const float* Lb = Ls + 32 * b * kTinvLd + 32 * b;
        float x[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            float acc = 0.f;
#pragma unroll
            for (int c = 0; c < r; ++c) acc = fmaf(Lb[r * kTinvLd + c], x[c], acc);
            x[r] = r < lane ? 0.f : (r == lane ? 1.f : -acc);
        }
        if (gj < w) {
#pragma unroll
            for (int r = 0; r < 32; ++r) Xs[(32 * b + r) * kTinvLd + gj] = x[r];
        }
    }
    __syncthreads();
    const int tr = tid & 31, tc = tid >> 5;
    for (int dd = 1; dd < 4; ++dd) {
        for (int ib = dd; ib < 4; ++ib) {
            const int jb = ib - dd;
            float acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.f;
            for (int kb = jb; kb < ib; ++kb)
                mm32_acc(acc, Ls + 32 * ib * kTinvLd + 32 * kb, kTinvLd, Xs + 32 * kb * kTinvLd + 32 * jb, kTinvLd);
            float* T = Tb + jb * 32 * 33;
#pragma unroll
            for (int q = 0; q < 8; ++q) T[tr * 33 + tc + 4 * q] = acc[q];
        }
        __syncthreads();
        for (int ib = dd; ib < 4; ++ib) {
            const int jb = ib - dd;
            float acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.f;
            mm32_acc(acc, Xs + 32 * ib * kTinvLd + 32 * ib, kTinvLd, Tb + jb * 32 * 33, 33);
#pragma unroll
            for (int q = 0; q < 8; ++q) Xs[(32 * ib + tr) * kTinvLd + 32 * jb + tc + 4 * q] = -acc[q];
        }
        __syncthreads();
    }
    for (int r = 0; r < kDtM; ++r) xinv[r * kDtM + tid] = Xs[r * kTinvLd + tid];
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
#pragma unroll 8
            for (int e = tid; e < kDtM * kDtK; e += kDtM) {
                const int r = e / kDtK, q = e % kDtK;
                Xs[r * (kDtM + 1) + q] = X[r * kDtM + c0 + q];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kDtK; ++q) v[q] = Xs[tid * (kDtM + 1) + q];
        } else {
            const int r0 = rt * kDtM, w = min(kDtM, k - r0);
            for (int r0x = 0; r0x < kDtM; r0x += 16) {  // 16 loads in flight per thread
                float xv[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) xv[q] = X[(r0x + q) * kDtM + tid];
#pragma unroll
                for (int q = 0; q < 16; ++q) Xs[(r0x + q) * (kDtM + 1) + tid] = xv[q];
            }
            float lv[kDtK];
#pragma unroll
            for (int q = 0; q < kDtK; ++q) lv[q] = tid < w ? P[(r0 + tid) + (int64_t)(c * kDtK + q) * m] : 0.f;
#pragma unroll
            for (int q = 0; q < kDtK; ++q) Lc[tid * (kDtK + 1) + q] = lv[q];
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

// Roles of the variance CTA (warp-specialized): warps 0-3 load chunks of Z
// (plain loads, one chunk ahead), split them into TF32 hi/lo, add finished
// hi*hi groups into S and run the tile epilogues (they own tensor-memory lanes
// 0-127); lane 0 of warp 4 copies the packed left operands (TMA tensor
// copies), lane 0 of warp 5 issues the MMAs.  They meet only at mbarriers.
// (The Z chunks went through a second TMA tensor map at first; when the
// kernel shared its SMs with the dependency-driven solve, those copies read
// rows that the previous tile's epilogue had written -- released to the
// copying thread through an mbarrier -- with stale values, while plain loads
// behind the same mbarrier read them right; so the workers load Z themselves.)
constexpr int kDtWork = 128;                       // threads of warps 0-3
constexpr int kDtRoles = kDtWork + 2 * 32;         // + warps 4, 5
constexpr int kDtAStages = 3, kDtBStages = 2;
constexpr int kDtRStages = 3;                      // raw Z chunks in flight (two ahead of the split)
constexpr int kDtRawCols = 132;                    // columns of a raw chunk: N + the 16-byte round-down
constexpr int kDtRaw = kDtK * kDtRawCols;          // floats of one raw chunk (32 rows)
constexpr int kDtOffB = kDtAStages * 2 * kDtTile;  // floats: A ring, split B ring, raw Z ring
constexpr int kDtOffRaw = kDtOffB + kDtBStages * 2 * kDtTile;
constexpr int kDtOffVar = kDtOffRaw + kDtRStages * kDtRaw;
// mbarriers: A full/empty, B full/empty, group full/empty, acc full/empty, z ready
enum : int { kBAF = 0, kBAE = 3, kBBF = 6, kBBE = 8, kBGF = 10, kBGE = 12, kBCF = 14, kBCE = 15, kBZR = 16,
             kDtBars = 17 };
constexpr size_t kDtSmem2 = (size_t)kDtOffVar * sizeof(float) + 128 * sizeof(double) + kDtBars * sizeof(uint64_t) + 16;

// 16-byte asynchronous copy global -> shared (L2 only); src_bytes 0 writes zeros
__device__ __forceinline__ void dt_cp16(uint32_t dst, const float* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void dt_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most n of this thread's copy groups are pending (n = 0 or 1)
__device__ __forceinline__ void dt_cp_wait(int n) {
    if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else asm volatile("cp.async.wait_group 1;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(tc_smem_u32(bar)) : "memory");
}
// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool dt_wait(uint64_t* bar, uint32_t parity, uint32_t limit, volatile int* abort) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(tc_smem_u32(bar)), "r"(parity));
        if (!done && *abort) return false;
    }
    return done != 0;
}

// The block's tensor-core supernodes in walk order and the shape of each.
struct DtNode {
    int s, lo0, nbu, zo, f, k, m, T, R, nch, N;
    int64_t urel;
};
__device__ __forceinline__ bool dt_next(const DevSym& d, const DiagArgsTc& p, const DiagTcArgs& ta, int& u, int u1,
                                        DtNode& x) {
    while (++u < u1) {
        const int s = p.us[u];
        if (!ta.tc[s]) continue;
        x.s = s;
        x.lo0 = p.ulo[u];
        x.nbu = p.uhi[u] - x.lo0;
        x.zo = p.uzoff[u];
        x.f = d.sfirst[s];
        x.k = d.sfirst[s + 1] - x.f;
        x.m = (int)(d.srowptr[s + 1] - d.srowptr[s]);
        x.T = (x.k + kDtM - 1) / kDtM;
        x.R = (x.m - x.k + kDtM - 1) / kDtM;
        x.nch = (x.k + kDtK - 1) / kDtK;
        x.N = (x.nbu + 31) & ~31;
        x.urel = p.urel[u];
        return true;
    }
    return false;
}
__device__ __forceinline__ int dt_chunks(const DtNode& x, int tile) {
    const int kext = tile < x.T ? min(kDtM * (tile + 1), x.k) : x.k;
    return (kext + kDtK - 1) / kDtK;
}

__global__ void __launch_bounds__(kDtRoles, 1)
    k_diag_inv_tc(DevSym d, DiagArgsTc p, DiagTcArgs ta, const double* __restrict__ D, double* __restrict__ out,
                  Strides bs, DevStatus* status, uint32_t wait_limit, const __grid_constant__ CUtensorMap tmap) {
    const int band = blockIdx.y;
    D += band * bs.n;
    out += band * bs.out;
    extern __shared__ __align__(1024) float dsm[];
    float* Aring = dsm;
    float* Bring = dsm + kDtOffB;
    float* Rring = dsm + kDtOffRaw;
    double* var = reinterpret_cast<double*>(dsm + kDtOffVar);  // [128]
    uint64_t* bar = reinterpret_cast<uint64_t*>(var + 128);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + kDtBars);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
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
    if (tid == kDtWork) {
        // arrivals per phase: one per worker warp for the barriers the worker warps arrive
        // on (B full, group empty, acc empty, z ready), else one (a copy's
        // expect-tx arrival or an MMA commit)
        for (int q = 0; q < kDtBars; ++q) {
            const bool workers = (q >= kBBF && q < kBBF + kDtBStages) || (q >= kBGE && q < kBGE + 2) || q == kBCE ||
                                 q == kBZR;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc_smem_u32(bar + q)),
                         "r"(workers ? kDtWork / 32 : 1));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort = 0;
    }
    for (int q = tid; q < 128; q += kDtRoles) var[q] = q < nr ? out[p.rhs_out[r0b + q]] : 0.0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t lim = wait_limit;
    // the last copies and commits of each role, drained below if a wait ran out
    uint32_t a_issued = 0, mma_chunks = 0;
    int mma_tiles = 0;
    if (warp == 4) {
        // ---- packed left operands: run ahead of the MMAs by up to 3 chunks
        if (lane == 0) {
            int u = u0 - 1;
            DtNode x;
            bool ok = true;
            while (ok && dt_next(d, p, ta, u, u1, x)) {
                const int64_t t0 = tile_band + ta.tptr[x.s];
                const int64_t nt = diag_tc_tile_offset(x.T, x.nch, x.T + x.R);
                for (int64_t t = 0; t < nt && ok; ++t) {
                    const uint32_t g = a_issued, st = g % kDtAStages;
                    if (g >= kDtAStages && !dt_wait(bar + kBAE + st, ((g - kDtAStages) / kDtAStages) & 1u, lim, abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(tc_smem_u32(bar + kBAF + st), 2 * kDtTile * sizeof(float));
                    tma_tile_pair(tc_smem_u32(Aring + st * 2 * kDtTile), &tmap, (int32_t)(8 * (t0 + t)),
                                  tc_smem_u32(bar + kBAF + st));
                    ++a_issued;
                }
            }
            if (!ok) *abort = 1;
        }
    } else if (warp == 5) {
        // ---- MMA issue: 4 k-steps x 3 products per chunk (hi*lo and lo*hi into X, hi*hi
        // into the group's buffer); commits free the stages, hand finished groups to
        // the flush and finished tiles to the epilogue
        if (lane == 0) {
            int u = u0 - 1;
            DtNode x;
            bool ok = true;
            uint32_t gcommit[2] = {0, 0};  // group commits per buffer so far
            uint32_t glast[2] = {0, 0};    // index of the last group commit on each buffer
            while (ok && dt_next(d, p, ta, u, u1, x)) {
                const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(x.N >> 3) << 17) |
                                       ((uint32_t)(kDtM >> 4) << 24);
                for (int tile = 0; tile < x.T + x.R && ok; ++tile) {
                    if (mma_tiles > 0 && !dt_wait(bar + kBCE, (uint32_t)(mma_tiles - 1) & 1u, lim, abort)) {
                        ok = false;
                        break;
                    }
                    const int nck = dt_chunks(x, tile);
                    for (int c = 0; c < nck && ok; ++c) {
                        const int j = c >> 2, buf = j & 1;
                        if ((c & 3) == 0 && j >= 2 && !dt_wait(bar + kBGE + buf, glast[buf] & 1u, lim, abort)) {
                            ok = false;
                            break;
                        }
                        const uint32_t g = mma_chunks, sa = g % kDtAStages, sb = g % kDtBStages;
                        if (!dt_wait(bar + kBAF + sa, (g / kDtAStages) & 1u, lim, abort) ||
                            !dt_wait(bar + kBBF + sb, (g / kDtBStages) & 1u, lim, abort)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const float* A = Aring + sa * 2 * kDtTile;
                        const float* Bh = Bring + sb * 2 * kDtTile;
                        const uint32_t acc = tmem + (buf ? kDtA1 : 0u);
#pragma unroll
                        for (int kk = 0; kk < kDtK / 8; ++kk) {
                            const uint32_t ko = kk * 256;
                            const uint64_t ah = tc_desc(tc_smem_u32(A) + ko), al = tc_desc(tc_smem_u32(A + kDtTile) + ko);
                            const uint64_t bh = tc_desc(tc_smem_u32(Bh) + ko), bl = tc_desc(tc_smem_u32(Bh + kDtTile) + ko);
                            tc_mma(tmem + kDtX, ah, bl, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                            tc_mma(tmem + kDtX, al, bh, idesc, 1u);
                            tc_mma(acc, ah, bh, idesc, ((c & 3) > 0 || kk > 0) ? 1u : 0u);
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     :: "r"(tc_smem_u32(bar + kBAE + sa)));
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     :: "r"(tc_smem_u32(bar + kBBE + sb)));
                        if ((c & 3) == 3 && c + 1 < nck) {  // a finished group that the flush takes
                            glast[buf] = gcommit[buf]++;
                            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                         :: "r"(tc_smem_u32(bar + kBGF + buf)));
                        }
                        ++mma_chunks;
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(tc_smem_u32(bar + kBCF)));
                    ++mma_tiles;
                }
            }
            if (!ok) *abort = 1;
        }
    } else {
        // ---- warps 0-3: split, flush, epilogue.  Each wait's outcome is made uniform
        // across the warp (a lane must not leave while the others reach __syncwarp);
        // the warps meet each other only at mbarriers, whose waits are all bounded.
        auto wwait = [&](uint64_t* br, uint32_t par) { return __all_sync(0xffffffffu, dt_wait(br, par, lim, abort)); };
        int u = u0 - 1, tiles = 0;
        uint32_t zwaits = 0;
        DtNode x;
        bool ok = true;
        uint32_t g = 0;                // chunks split
        uint32_t gwait[2] = {0, 0};    // group commits waited per buffer
        while (ok && dt_next(d, p, ta, u, u1, x)) {
            const int32_t* rel = p.rel + x.urel;
            const bool vec = (x.lo0 & 3) == 0;
            // Warp w stages rows [8 w, 8 w + 8) of every 32-row chunk: it copies them (16-byte
            // copies from the 16-byte-aligned column x0 at or below lo0, rows past kext and
            // columns past the workspace read as zeros) into the raw ring, and its lanes split
            // them (lane: right-hand sides lane + 32 v).  No other warp reads these rows.
            const int x0 = x.lo0 & ~3, sh = x.lo0 - x0;
            const int ngr = (sh + x.N + 3) / 4;  // 16-byte groups per row
            auto fetch = [&](int c, int kext, int rs) {
                float* raw = Rring + rs * kDtRaw;
                for (int e = lane; e < 8 * ngr; e += 32) {
                    const int r = 8 * warp + e / ngr, gq = e % ngr;
                    const int kr = c * kDtK + r, col = x0 + 4 * gq;
                    const bool on = kr < kext && col < B;
                    dt_cp16(tc_smem_u32(raw + r * kDtRawCols + 4 * gq), on ? Z + (int64_t)(x.zo + kr) * B + col : Z,
                            on ? 16 : 0);
                }
                dt_cp_commit();
            };
            for (int tile = 0; tile < x.T + x.R && ok; ++tile, ++tiles) {
                const bool own = tile < x.T;
                const int rows0 = own ? tile * kDtM : x.k + (tile - x.T) * kDtM;
                const int nrow = min(kDtM, (own ? x.k : x.m) - rows0);
                const int kext = own ? min(kDtM * (tile + 1), x.k) : x.k;
                const int nck = (kext + kDtK - 1) / kDtK;
                // the rows this tile reads were written by the previous tile's epilogue (an own
                // tile, or the first tile below) in all four warps: wait for their z-ready
                if (tiles > 0 && tile <= x.T && !wwait(bar + kBZR, zwaits++ & 1u)) { ok = false; break; }
                for (int c = 0; c < kDtRStages - 1 && c < nck; ++c) fetch(c, kext, c);
                for (int c = 0; c < nck && ok; ++c, ++g) {
                    const uint32_t sr = g % kDtBStages;
                    if (g >= kDtBStages && !wwait(bar + kBBE + sr, ((g - kDtBStages) / kDtBStages) & 1u)) {
                        ok = false;
                        break;
                    }
                    dt_cp_wait(c + 1 < nck ? 1 : 0);  // this warp's copies of chunk c have landed
                    __syncwarp();
                    const float* raw = Rring + (c % kDtRStages) * kDtRaw;
                    float* Bh = Bring + sr * 2 * kDtTile;
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int kq = 2 * warp + h2;
#pragma unroll
                        for (int vq = 0; vq < 4; ++vq) {
                            const int n = lane + 32 * vq;
                            if (n < x.N) {
                                const bool on = n < x.nbu;
                                float4 h, l;
                                tc_split2(on ? raw[(4 * kq + 0) * kDtRawCols + sh + n] : 0.f, h.x, l.x);
                                tc_split2(on ? raw[(4 * kq + 1) * kDtRawCols + sh + n] : 0.f, h.y, l.y);
                                tc_split2(on ? raw[(4 * kq + 2) * kDtRawCols + sh + n] : 0.f, h.z, l.z);
                                tc_split2(on ? raw[(4 * kq + 3) * kDtRawCols + sh + n] : 0.f, h.w, l.w);
                                const int o = tc_kmajor_off(n, 4 * kq) >> 2;
                                *reinterpret_cast<float4*>(Bh + o) = h;
                                *reinterpret_cast<float4*>(Bh + kDtTile + o) = l;
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;");
                    __syncwarp();  // this warp's reads of the raw stage are done before it is refilled
                    if (lane == 0) mbar_arrive(bar + kBBF + sr);
                    // the stage just read takes chunk c + 2 (still this tile: the next tile's rows may
                    // wait for this tile's epilogue)
                    if (c + kDtRStages - 1 < nck) fetch(c + kDtRStages - 1, kext, (c + kDtRStages - 1) % kDtRStages);
                    if ((c & 3) == 0 && c > 0) {
                        // S (+)= the buffer of group c/4 - 1 while this group accumulates in the other
                        const int pb = ((c >> 2) - 1) & 1;
                        if (!wwait(bar + kBGF + pb, gwait[pb]++ & 1u)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t row = (uint32_t)(warp * 32) << 16;
                        for (int q = 0; q < x.N / 32; ++q) {
                            uint32_t a[32], sv[32];
                            tc_ld32(tmem + row + (pb ? kDtA1 : 0u) + q * 32, a);
                            if (c > 4) {
                                tc_ld32(tmem + row + kDtS + q * 32, sv);
                                tc_add32(a, sv);
                            }
                            tc_st32(tmem + row + kDtS + q * 32, a);
                        }
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(bar + kBGE + pb);
                    }
                }
                if (!ok) break;
                // ---- epilogue of the tile: result = S (groups before the last) + last group + X
                if (!wwait(bar + kBCF, (uint32_t)tiles & 1u)) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int jl = (nck - 1) >> 2;
                const int row = warp * 32 + lane;
                const int lr = rows0 + row;
                const bool rv = row < nrow;
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
                const float dinv = (own && rv) ? (float)(1.0 / D[x.f + lr]) : 0.f;
                float* zrow = Z + (int64_t)(own ? x.zo + lr : (rv ? rel[lr - x.k] : 0)) * B + x.lo0;
                for (int q = 0; q < x.N / 32; ++q) {
                    uint32_t r[32], t[32];
                    tc_ld32(taddr + (jl & 1 ? kDtA1 : 0u) + q * 32, r);
                    tc_ld32(taddr + kDtX + q * 32, t);
                    tc_add32(r, t);
                    if (jl > 0) {
                        tc_ld32(taddr + kDtS + q * 32, t);
                        tc_add32(r, t);
                    }
                    float w[32];
                    if (own) {
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) w[jj] = __uint_as_float(r[jj]);
                        if (rv) z_store32(zrow, w, q * 32, x.nbu, vec);
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj)
                            w[jj] = (rv && q * 32 + jj < x.nbu) ? w[jj] * w[jj] * dinv : 0.f;
                        const float cs = lane_sums(w, lane);  // this warp's 32 rows of column q*32+lane
                        if (q * 32 + lane < x.nbu) atomicAdd(&var[x.lo0 + q * 32 + lane], (double)cs);
                    } else if (rv) {
                        z_load32(zrow, w, q * 32, x.nbu, vec);
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) w[jj] += __uint_as_float(r[jj]);
                        z_store32(zrow, w, q * 32, x.nbu, vec);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(bar + kBCE);
                    if (tile < x.T || tile + 1 == x.T + x.R) mbar_arrive(bar + kBZR);  // the tiles waited on
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy of this thread left in flight
        if (!ok) *abort = 1;
    }
    // ---- a wait ran out somewhere: let the copies and products in flight finish (again
    // bounded), report it, release tensor memory and leave the variances
    __syncthreads();
    const bool failed = *abort != 0;
    if (failed) {
        if (tid == kDtWork) {
            atomicOr(&status->flags, FLAG_TIMEOUT);
            for (uint32_t q = a_issued > kDtAStages ? a_issued - kDtAStages : 0; q < a_issued; ++q)
                tc_wait(bar + kBAF + q % kDtAStages, (q / kDtAStages) & 1u);
        }
        if (tid == kDtWork + 32 && mma_chunks > 0) {
            // one more commit tracks every MMA issued so far
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(tc_smem_u32(bar + kBCF)));
            tc_wait(bar + kBCF, (uint32_t)mma_tiles & 1u);
        }
    }
    __syncthreads();
    if (!failed)
        for (int q = tid; q < nr; q += kDtRoles) out[p.rhs_out[r0b + q]] = var[q];
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

}  // namespace

cudaError_t diag_tc_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_diag_inv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDtSmem2);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_diag_inv_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_diag_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_diag_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPackSmem);
}

size_t diag_tc_pack_floats(int64_t npt) { return (size_t)npt * 2 * kDtTile; }
size_t diag_tc_xinv_floats(int64_t ndt) { return (size_t)ndt * kDtM * kDtM; }

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query
// (no link against the driver library).
cudaError_t tensor_map_encoder(EncodeFn* out) {
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    *out = encode;
    return cudaSuccess;
}

// The tensor map over the packed tiles of `bands` bands: [slices][256][4]
// floats, 16-byte rows, 4 KB slices, eight slices per tile pair; one box is a
// whole tile pair (4 x 256 x 8).  cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query (no link against the driver library).
cudaError_t diag_tc_tensor_map(float* pack, int64_t npt, int bands, void* map_out) {
    EncodeFn encode = nullptr;
    cudaError_t e = tensor_map_encoder(&encode);
    if (e != cudaSuccess) return e;
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
    k_diag_inv_tc<<<dim3(dp.nblocks, nb), kDtRoles, kDtSmem2, st>>>(
        d, a, t, D, out, bs, status, lim, *reinterpret_cast<const CUtensorMap*>(p.tmap));
}

}  // namespace spi
