// peaks.cu -- measured throughput of the arithmetic units the kernels of this
// library are bound by, so that every roofline fraction the benchmark reports
// has a denominator measured on the device it runs on: FP64 FMA (the FP64
// form's factorization and variances), FP64 mma.sync (DMMA), FP32 FMA (the
// mixed form's SIMT kernels), and the 5th-generation tensor cores through
// tcgen05.mma with TF32 inputs (the mixed form's split-precision Schur
// updates) and BF16 inputs (checked against a cuBLAS BF16 figure).
//
// Every probe runs independent operations on every SM for a fixed number of
// iterations; the host times it with CUDA events and keeps the best of a few
// runs.  The results are written to a device buffer that the host never
// reads, so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "spi.h"

namespace {

constexpr int kFmaChains = 8;

__global__ void __launch_bounds__(256) k_peak_fma64(double a, double b, int iters, double* sink) {
    double acc[kFmaChains];
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) acc[q] = threadIdx.x * 1e-3 + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kFmaChains; ++q) acc[q] = fma(acc[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) s += acc[q];
    if (s == 12345.678) sink[threadIdx.x] = s;  // never true in practice; keeps the chains alive
}

__global__ void __launch_bounds__(256) k_peak_fma32(float a, float b, int iters, float* sink) {
    float acc[kFmaChains];
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) acc[q] = threadIdx.x * 1e-3f + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < kFmaChains; ++q) acc[q] = fmaf(acc[q], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kFmaChains; ++q) s += acc[q];
    if (s == 12345.678f) sink[threadIdx.x] = s;
}

// FP64 tensor path of mma.sync: m8n8k4, 4 independent accumulators per warp.
__global__ void __launch_bounds__(256) k_peak_dmma(double a0, double b0, int iters, double* sink) {
    double c[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) c[q][0] = c[q][1] = threadIdx.x * 1e-3;
    const double a = a0 + threadIdx.x * 1e-9, b = b0 - threadIdx.x * 1e-9;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(c[q][0]), "+d"(c[q][1]) : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) s += c[q][0] + c[q][1];
    if (s == 12345.678) sink[threadIdx.x] = s;
}

// tcgen05.mma, one CTA per SM: M = 128, N = 256, accumulator in tensor memory
// (256 columns), operands from a K-major no-swizzle shared-memory layout of
// 8-row core matrices (contents irrelevant: zeros).  One thread issues the
// MMAs; every 16 it commits to an mbarrier and waits (bounded) for the batch
// before the previous one to finish, so at most two batches are in flight.
constexpr int kPM = 128, kPN = 256;
constexpr int kPSmemA = kPM * 32 * 4, kPSmemB = kPN * 32 * 4;  // 32 K-columns of 4 bytes
constexpr uint32_t kPeakWait = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity));
    return done != 0;
}

template <int kKind>  // 0: kind::tf32 (K = 8 per MMA), 1: kind::f16 with BF16 inputs (K = 16)
__global__ void __launch_bounds__(128) k_peak_tcgen05(int batches, int* flag) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;
    unsigned char* B = sm + kPSmemA;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kPSmemA + kPSmemB);  // [2]
    uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (kPSmemA + kPSmemB) / 16; i += 128) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(slot)),
                     "r"(kPN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *slot;
    // instruction descriptor: FP32 accumulator; A and B TF32 (2) or BF16 (1); N >> 3, M >> 4
    const uint32_t ab = kKind == 0 ? 2u : 1u;
    const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(kPN >> 3) << 17) |
                           ((uint32_t)(kPM >> 4) << 24);
    bool ok = true;
    int last = -1;
    if (tid == 0) {
        for (int bt = 0; bt < batches && ok; ++bt) {
            if (bt >= 2) ok = mbar_wait(mbar + (bt & 1), (uint32_t)((bt - 2) >> 1) & 1u, kPeakWait);
            if (!ok) break;
            for (int q = 0; q < 16; ++q) {
                const uint32_t ko = (uint32_t)(q & 3) * 256;  // one of four 32-byte K steps
                const uint64_t da = kmajor_desc(smem_u32(A) + ko), db = kmajor_desc(smem_u32(B) + ko);
                const uint32_t acc = (bt > 0 || q > 0) ? 1u : 0u;
                if (kKind == 0)
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                else
                    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(mbar + (bt & 1))));
            last = bt;
        }
        // the last commit covers every MMA issued before it
        if (last >= 0 && !mbar_wait(mbar + (last & 1), (uint32_t)(last >> 1) & 1u, kPeakWait)) ok = false;
        if (!ok) atomicExch(flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kPN));
}

}  // namespace

extern "C" int spi_measure_peak(int unit, int reps, double* tflops) {
    if (!tflops || unit < 0 || unit > 4 || reps < 1) return SPI_ERR_ARG;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPI_ERR_CUDA;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 4096 * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return SPI_ERR_OOM; }
    int* flag = reinterpret_cast<int*>(static_cast<double*>(sink) + 2048);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // more shared memory than the probe uses, so that no SM runs two of its CTAs
    const size_t tc_smem = 116 * 1024;
    int rc = SPI_OK;
    if (unit >= 3) {
        cudaError_t e = cudaFuncSetAttribute(k_peak_tcgen05<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_peak_tcgen05<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem);
        if (e != cudaSuccess) rc = SPI_ERR_CUDA;
        if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess) rc = SPI_ERR_CUDA;
    }
    double best = 0.0;
    for (int r = 0; r <= reps && rc == SPI_OK; ++r) {  // run 0 warms up
        double flops = 0.0;
        cudaEventRecord(e0);
        switch (unit) {
            case 0: {
                const int iters = 1 << 14, grid = sms * 8;
                k_peak_fma64<<<grid, 256>>>(1.0000001, 1e-9, iters, static_cast<double*>(sink));
                flops = 2.0 * kFmaChains * iters * 256.0 * grid;
                break;
            }
            case 1: {
                const int iters = 1 << 12, grid = sms * 8;
                k_peak_dmma<<<grid, 256>>>(1.0000001, 1e-9, iters, static_cast<double*>(sink));
                flops = 4.0 * 512.0 * iters * (256.0 / 32.0) * grid;
                break;
            }
            case 2: {
                const int iters = 1 << 18, grid = sms * 8;
                k_peak_fma32<<<grid, 256>>>(1.0000001f, 1e-9f, iters, static_cast<float*>(sink));
                flops = 2.0 * kFmaChains * iters * 256.0 * grid;
                break;
            }
            default: {
                const int batches = 1 << 14;
                if (unit == 3) k_peak_tcgen05<0><<<sms, 128, tc_smem>>>(batches, flag);
                else k_peak_tcgen05<1><<<sms, 128, tc_smem>>>(batches, flag);
                flops = 2.0 * kPM * kPN * (unit == 3 ? 8.0 : 16.0) * 16.0 * batches * sms;
                break;
            }
        }
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) { rc = SPI_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    if (rc == SPI_OK && unit >= 3) {
        int f = 0;
        if (cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = SPI_ERR_CUDA;
        else if (f) rc = SPI_ERR_TIMEOUT;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc == SPI_OK) *tflops = best;
    return rc;
}
