// normal.cu -- the normal equations on the device (paper Sec. 4.1, Eq. 7):
// N = H^T W H (its lower triangle, on the pattern the context was analysed
// with) and b = H^T W y, from the design matrix H in CSR (rows =
// observations), and their update after the values of some columns of H
// changed (paper Table 3: recompute only what those columns touch).
//
// Rows are grouped on the host into runs of consecutive rows whose column
// sets nearly coincide (for SPI: the detectors of one pointing).  One CTA per
// group stages the group's rows densely over the union of their columns C
// (R rows x c columns in shared memory; a single long row is read in place),
// then each thread takes columns b of the union and walks a = b .. c-1,
// forming g_ab = sum_r w_r h_ra h_rb and adding it to N's entry
// (C[a], C[b]).  That entry's position is found by walking column C[b] of the
// pattern upward: the union and the pattern's rows are both ascending.
// Groups share entries of N, so the adds are FP64 atomics.  A product term
// with no place in the pattern sets an error flag.
#include <cuda_runtime.h>

#include "spi_internal.cuh"

namespace spi {
namespace {

constexpr int kNThreads = 256;

// kPass 0: the update's zero pass (entries and b of the marked columns set to
// 0); kPass 1: accumulate.  With mark == nullptr every pair is taken.
template <int kPass>
__global__ void __launch_bounds__(kNThreads) k_normal_group(NormalArgs a, const int32_t* __restrict__ groups,
                                                             const double* __restrict__ hv,
                                                             const double* __restrict__ w,
                                                             const double* __restrict__ y,
                                                             const uint8_t* __restrict__ mark,
                                                             double* __restrict__ nv, double* __restrict__ bv,
                                                             int* __restrict__ flag) {
    extern __shared__ __align__(16) double nsm[];
    const int g = groups[blockIdx.x];
    const int64_t r0 = a.grp_row[g], r1 = a.grp_row[g + 1];
    const int R = (int)(r1 - r0);
    const int64_t c0 = a.grp_colptr[g];
    const int c = (int)(a.grp_colptr[g + 1] - c0);
    const int32_t* C = a.grp_cols + c0;
    const int tid = threadIdx.x;
    // dense rows (R > 1): Hs[r * c + a]; a single row is read from hv directly
    const bool dense = R > 1;
    double* Hs = nsm;
    double* ws = nsm + (dense ? (size_t)R * c : 0);  // w_r and w_r y_r
    if (dense) {
        for (int e = tid; e < R * c; e += kNThreads) Hs[e] = 0.0;
        __syncthreads();
        for (int64_t e = a.rowptr[r0] + tid; e < a.rowptr[r1]; e += kNThreads) {
            int lo = 0, hi = R;  // the row of entry e
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (a.rowptr[r0 + mid] <= e) lo = mid; else hi = mid;
            }
            Hs[(size_t)lo * c + a.ent_pos[e]] = hv[e];
        }
    }
    for (int r = tid; r < R; r += kNThreads) {
        ws[2 * r] = w[r0 + r];
        ws[2 * r + 1] = w[r0 + r] * y[r0 + r];
    }
    __syncthreads();
    const double* h1 = hv + a.rowptr[r0];  // the single row's values, in union order
    auto H = [&](int r, int col) { return dense ? Hs[(size_t)r * c + col] : h1[col]; };
    for (int b = tid; b < c; b += kNThreads) {
        const int32_t j = C[b];
        const bool mb = mark ? mark[j] != 0 : true;
        // b_j = sum_r w_r y_r h_rj
        if (mark == nullptr || mb) {
            if (kPass == 0) {
                bv[j] = 0.0;
            } else {
                double s = 0.0;
                for (int r = 0; r < R; ++r) s += ws[2 * r + 1] * H(r, b);
                atomicAdd(bv + j, s);
            }
        }
        int64_t q = a.cp[j];
        const int64_t qend = a.cp[j + 1];
        for (int aa = b; aa < c; ++aa) {
            const int32_t i = C[aa];
            if (mark && !mb && !mark[i]) continue;
            while (q < qend && a.ri[q] < i) ++q;
            const bool found = q < qend && a.ri[q] == i;
            if (kPass == 0) {
                if (found) nv[q] = 0.0;
                continue;
            }
            double s = 0.0;
            for (int r = 0; r < R; ++r) s += ws[2 * r] * H(r, aa) * H(r, b);
            if (found) atomicAdd(nv + q, s);
            else if (s != 0.0) atomicOr(flag, 1);
        }
    }
}

}  // namespace

size_t normal_smem_bytes(int32_t max_dense_entries, int32_t max_rows) {
    return sizeof(double) * ((size_t)max_dense_entries + 2 * (size_t)max_rows);
}

cudaError_t normal_kernel_setup(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_normal_group<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_normal_group<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_normal(const NormalArgs& a, const int32_t* groups, int32_t ngroups, const double* hv, const double* w,
                   const double* y, const uint8_t* mark, bool zero_pass, double* nv, double* bv, int* flag,
                   size_t smem, cudaStream_t st) {
    if (ngroups == 0) return;
    if (zero_pass)
        k_normal_group<0><<<ngroups, kNThreads, smem, st>>>(a, groups, hv, w, y, mark, nv, bv, flag);
    else
        k_normal_group<1><<<ngroups, kNThreads, smem, st>>>(a, groups, hv, w, y, mark, nv, bv, flag);
}

}  // namespace spi
