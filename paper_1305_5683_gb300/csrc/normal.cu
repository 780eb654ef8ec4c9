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
// then takes the columns b of the union one at a time (u_r = w_r h_rb in
// shared memory) and spreads a = b .. c-1 over its threads, each forming
// g_ab = sum_r u_r h_ra and adding it to N's entry
// (C[a], C[b]).  That entry's position comes from a table the host builds at
// setup (pair (a, b) of group g at pairptr[g] + b c - b (b - 1) / 2 + a - b,
// -1 when the pattern has no such entry); when the table would be too large
// it is found by binary search in column C[b] of the pattern.  Groups share entries of N, so
// the adds are FP64 atomics.  A product term with no place in the pattern
// sets an error flag.
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
    // update: the group's marked columns, as a list of union indices (ascending)
    int32_t* ml = reinterpret_cast<int32_t*>(ws + 2 * R);
    double* us = ws + 2 * R;  // u_r = w_r h_rb of the current column b (after ml's space)
    __shared__ int nml;
    if (tid == 0) {
        int k = 0;
        if (mark)
            for (int aa = 0; aa < c; ++aa)
                if (mark[C[aa]]) ml[k++] = aa;
        nml = k;
    }
    __syncthreads();
    us += (nml + 1) / 2;  // doubles after the list (the list holds at most c ints)
    const double* h1 = hv + a.rowptr[r0];  // the single row's values, in union order
    auto H = [&](int r, int col) { return dense ? Hs[(size_t)r * c + col] : h1[col]; };
    // columns b one at a time across the CTA: g_ab = sum_r u_r h_ra for a = b .. c-1
    // (with a mark and an unmarked b: only the marked a)
    for (int b = 0; b < c; ++b) {
        const int32_t j = C[b];
        const bool mb = mark ? mark[j] != 0 : true;
        if (kPass == 1 && tid < R) us[tid] = ws[2 * tid] * H(tid, b);
        if (tid == kNThreads - 1 && mb) {  // b_j = sum_r w_r y_r h_rj
            if (kPass == 0) {
                bv[j] = 0.0;
            } else {
                double sb = 0.0;
                for (int r = 0; r < R; ++r) sb += ws[2 * r + 1] * H(r, b);
                atomicAdd(bv + j, sb);
            }
        }
        __syncthreads();
        const int32_t* pt = a.pairpos ? a.pairpos + a.pairptr[g] + (int64_t)b * c - (int64_t)b * (b - 1) / 2 - b
                                      : nullptr;
        int t0 = 0;
        if (!mb) {  // first marked a >= b
            int lo = 0, hi = nml;
            while (lo < hi) { const int mid = (lo + hi) >> 1; if (ml[mid] < b) lo = mid + 1; else hi = mid; }
            t0 = lo;
        }
        const int cnt = mb ? c - b : nml - t0;
        for (int t = tid; t < cnt; t += kNThreads) {
            const int aa = mb ? b + t : ml[t0 + t];
            const int32_t i = C[aa];
            int64_t q;
            bool found;
            if (pt) {
                const int32_t pos = pt[aa];
                found = pos >= 0;
                q = pos;
            } else {  // binary search of row i in column j of the pattern
                int64_t lo = a.cp[j], hi = a.cp[j + 1];
                while (lo < hi) { const int64_t mid = (lo + hi) >> 1; if (a.ri[mid] < i) lo = mid + 1; else hi = mid; }
                q = lo;
                found = q < a.cp[j + 1] && a.ri[q] == i;
            }
            if (kPass == 0) {
                if (found) nv[q] = 0.0;
                continue;
            }
            double sv = 0.0;
            if (dense) {
                const double* hc = Hs + aa;
                for (int r = 0; r < R; ++r) sv += us[r] * hc[(size_t)r * c];
            } else {
                sv = us[0] * h1[aa];
            }
            if (found) atomicAdd(nv + q, sv);
            else if (sv != 0.0) atomicOr(flag, 1);
        }
        __syncthreads();  // us is rewritten for the next column
    }
}

}  // namespace

size_t normal_smem_bytes(int32_t max_dense_entries, int32_t max_rows, int32_t max_cols) {
    return sizeof(double) * ((size_t)max_dense_entries + 3 * (size_t)max_rows + 1) +
           sizeof(int32_t) * (size_t)max_cols;
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
