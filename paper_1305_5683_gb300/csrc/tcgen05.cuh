// tcgen05.cuh -- shared pieces of the kernels on the 5th-generation tensor
// cores (tcgen05.mma kind::tf32 with accumulators in tensor memory): shared-
// memory operand layout and descriptors, the split of FP32 values into TF32
// pieces, tensor-memory loads and stores, bounded mbarrier waits.
#pragma once
#include <cstdint>

namespace spi {
namespace {

constexpr uint32_t kTcWaitLimit = 1u << 20;
// Tensor memory of a tensor-core CTA: accumulator A (the hi*hi products) in
// columns [0, 128), B (the smaller cross products) in [128, 256), and S,
// the running sum of A, in [256, 384); 512 columns are allocated (a power of
// two).  The tensor cores do not round to nearest when they add into an
// accumulator, so a long accumulation drifts by about one unit in the last
// place per add: A is added into S (an FP32 round-to-nearest add on the CUDA
// cores) and restarted every kTcFlush K-chunks of 32 (128 columns), and the small terms,
// whose drift is relative to their own small size, go to B.
constexpr uint32_t kTcCols = 512, kAccB = 128, kAccS = 256;
constexpr int kTcFlush = 4;

__device__ __forceinline__ int tc_kmajor_off(int r, int c) {
    return (r >> 3) * 1024 + (c >> 2) * 128 + (r & 7) * 16 + (c & 3) * 4;
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle; leading (K) byte
// offset 128 between the two core matrices of a k-step, stride (M/N) byte
// offset 1024 between 8-row groups.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ float tc_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// a = hi + mid + lo, three TF32 values (the split of the split-precision products)
__device__ __forceinline__ void tc_split3(float a, float& hi, float& mid, float& lo) {
    hi = tc_tf32(a);
    const float r1 = a - hi;
    mid = tc_tf32(r1);
    lo = tc_tf32(r1 - mid);
}

// 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
}

// Store 32 consecutive accumulator columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
                    "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
                    "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]),
                    "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]),
                    "r"(r[31]));
    asm volatile("tcgen05.wait::st.sync.aligned;");
}

// The finished product for 32 columns of this warp's rows: (S + A) + B, or A + B
// if A was never added into S.
__device__ __forceinline__ void tc_acc32(uint32_t taddr, bool with_s, uint32_t (&r)[32]) {
    uint32_t t[32];
    tc_ld32(taddr, r);
    if (with_s) {
        tc_ld32(taddr + kAccS, t);
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(t[j]) + __uint_as_float(r[j]));
    }
    tc_ld32(taddr + kAccB, t);
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(t[j]));
}

__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = kTcWaitLimit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(tc_smem_u32(mbar)), "r"(parity));
    return done != 0;
}

}  // namespace
}  // namespace spi
