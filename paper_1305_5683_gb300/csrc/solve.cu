// solve.cu -- solution phase (paper Sec. 3.2.3): forward substitution
// z = L^-1 P b bottom-up over the supernodal tree, then x = P^T L^-T D^-1 z
// top-down.  One launch per tree level; one CTA per supernode.
#include <cuda_runtime.h>

#include <algorithm>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kThreads = 256;

__global__ void k_permute_in(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ b,
                             double* __restrict__ w) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        w[k] = b[perm[k]];
}

__global__ void k_permute_out(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ w,
                              double* __restrict__ x) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        x[perm[k]] = w[k];
}

// Forward: x_s = L11^-1 w_s (unit lower), then w[rows below] -= L21 x_s.
__global__ void __launch_bounds__(kThreads) k_fwd(DevSym d, const int32_t* __restrict__ list,
                                                  const double* __restrict__ L, double* __restrict__ w) {
    extern __shared__ double xs[];
    const int tid = threadIdx.x;
    const int s = list[blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const double* P = L + d.lptr[s];
    for (int c = tid; c < k; c += kThreads) xs[c] = w[f + c];
    __syncthreads();
    for (int c = 0; c < k - 1; ++c) {
        const double xc = xs[c];
        for (int r = c + 1 + tid; r < k; r += kThreads) xs[r] -= P[r + (int64_t)c * m] * xc;
        __syncthreads();
    }
    for (int c = tid; c < k; c += kThreads) w[f + c] = xs[c];
    const int32_t* rows = d.srows + d.srowptr[s];
    for (int64_t t = k + tid; t < m; t += kThreads) {
        double acc = 0.0;
        for (int c = 0; c < k; ++c) acc += P[t + (int64_t)c * m] * xs[c];
        atomicAdd(w + rows[t], -acc);
    }
}

// Backward: y = D^-1 w_s - L21^T x_below, then x_s = L11^-T y (unit upper).
__global__ void __launch_bounds__(kThreads) k_bwd(DevSym d, const int32_t* __restrict__ list,
                                                  const double* __restrict__ L, const double* __restrict__ D,
                                                  double* __restrict__ w) {
    extern __shared__ double ys[];
    const int tid = threadIdx.x;
    const int s = list[blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const double* P = L + d.lptr[s];
    const int32_t* rows = d.srows + d.srowptr[s];
    const int lane = tid & 31, warp = tid >> 5;
    for (int c = warp; c < k; c += kThreads / 32) {
        double acc = 0.0;
        for (int64_t t = k + lane; t < m; t += 32) acc += P[t + (int64_t)c * m] * w[rows[t]];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) ys[c] = w[f + c] / D[f + c] - acc;
    }
    __syncthreads();
    for (int c = k - 1; c > 0; --c) {
        const double yc = ys[c];
        for (int r = tid; r < c; r += kThreads) ys[r] -= P[c + (int64_t)r * m] * yc;
        __syncthreads();
    }
    for (int c = tid; c < k; c += kThreads) w[f + c] = ys[c];
}

// r -= N x for the symmetric N given by its lower CSC (caller numbering), one
// warp per column: the column's dot product for r_j, and the mirrored
// upper-triangle entries scattered into r_i.
__global__ void k_sym_residual(int32_t n, const int64_t* __restrict__ cp, const int32_t* __restrict__ ri,
                               const double* __restrict__ va, const double* __restrict__ x, double* __restrict__ r) {
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
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += dx[i];
}

}  // namespace

void launch_sym_residual(int32_t n, const int64_t* cp, const int32_t* ri, const double* va, const double* x,
                         double* r, cudaStream_t st) {
    if (n == 0) return;
    int grid = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 152 * 8);
    k_sym_residual<<<grid, 256, 0, st>>>(n, cp, ri, va, x, r);
}

void launch_norms2(int32_t n, const double* a, const double* b, double* out, cudaStream_t st) {
    if (n == 0) return;
    k_norms2<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(n, a, b, out);
}

void launch_axpy(int32_t n, const double* dx, double* x, cudaStream_t st) {
    if (n == 0) return;
    k_axpy<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(n, dx, x);
}

void launch_permute_in(int32_t n, const int32_t* perm, const double* b, double* w, cudaStream_t st) {
    if (n == 0) return;
    k_permute_in<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(n, perm, b, w);
}

void launch_permute_out(int32_t n, const int32_t* perm, const double* w, double* x, cudaStream_t st) {
    if (n == 0) return;
    k_permute_out<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(n, perm, w, x);
}

cudaError_t solve_kernel_setup(int32_t kmax) {
    size_t bytes = (size_t)std::max(kmax, 1) * sizeof(double);
    if (bytes <= 48 * 1024) return cudaSuccess;
    if (bytes > 220 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_fwd_level(const DevSym& d, const int32_t* list, int32_t count, int32_t kmax, const double* L,
                      double* w, cudaStream_t st) {
    if (count == 0) return;
    k_fwd<<<count, kThreads, (size_t)std::max(kmax, 1) * sizeof(double), st>>>(d, list, L, w);
}

void launch_bwd_level(const DevSym& d, const int32_t* list, int32_t count, int32_t kmax, const double* L,
                      const double* D, double* w, cudaStream_t st) {
    if (count == 0) return;
    k_bwd<<<count, kThreads, (size_t)std::max(kmax, 1) * sizeof(double), st>>>(d, list, L, D, w);
}

}  // namespace spi
