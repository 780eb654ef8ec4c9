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

#include <algorithm>

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
                                                             const double* __restrict__ bw,
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
        ws[2 * r + 1] = bw ? bw[r0 + r] : w[r0 + r] * y[r0 + r];  // b_j = sum_r (w_r y_r or bw_r) h_rj
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
                   const double* y, const double* bw, const uint8_t* mark, bool zero_pass, double* nv, double* bv,
                   int* flag, size_t smem, cudaStream_t st) {
    if (ngroups == 0) return;
    if (zero_pass)
        k_normal_group<0><<<ngroups, kNThreads, smem, st>>>(a, groups, hv, w, y, bw, mark, nv, bv, flag);
    else
        k_normal_group<1><<<ngroups, kNThreads, smem, st>>>(a, groups, hv, w, y, bw, mark, nv, bv, flag);
}

// ---- Poisson maximum likelihood (the appendix on low-count fitting): the model
// e = H x, the Newton weights y/e^2, the gradient coefficients y/e - 1, and the
// Cash statistic C = sum (e - y ln e).

namespace {

// e = H x, one warp per row (H in CSR)
__global__ void k_spmv_rows(int64_t nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            const double* __restrict__ hv, const double* __restrict__ x, double* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < nrows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double s = 0.0;
        for (int64_t p = rowptr[r] + lane; p < rowptr[r + 1]; p += 32) s += hv[p] * x[colind[p]];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) e[r] = s;
    }
}

// acc[0] += sum (e - y ln e); acc[1] += number of rows with e <= 0; with w != null
// also w = y / e^2 and v = y / e - 1
__global__ void k_mle_rows(int64_t nrows, const double* __restrict__ e, const double* __restrict__ y,
                           double* __restrict__ w, double* __restrict__ v, double* __restrict__ acc) {
    double c = 0.0, bad = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const double er = e[r], yr = y[r];
        if (!(er > 0.0)) { bad += 1.0; continue; }
        c += yr > 0.0 ? er - yr * log(er) : er;
        if (w) {
            const double q = yr / er;
            w[r] = q / er;
            v[r] = q - 1.0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, c);
        if (bad != 0.0) atomicAdd(acc + 1, bad);
    }
}

// xt = x + t dx
__global__ void k_step(int32_t n, const double* __restrict__ x, const double* __restrict__ dx, double t,
                       double* __restrict__ xt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xt[i] = x[i] + t * dx[i];
}

}  // namespace

void launch_spmv_rows(int64_t nrows, const int64_t* rowptr, const int32_t* colind, const double* hv, const double* x,
                      double* e, cudaStream_t st) {
    if (nrows == 0) return;
    const int grid = (int)std::min<int64_t>((nrows * 32 + 255) / 256, 152 * 16);
    k_spmv_rows<<<grid, 256, 0, st>>>(nrows, rowptr, colind, hv, x, e);
}

void launch_mle_rows(int64_t nrows, const double* e, const double* y, double* w, double* v, double* acc,
                     cudaStream_t st) {
    if (nrows == 0) return;
    const int grid = (int)std::min<int64_t>((nrows + 255) / 256, 152 * 8);
    k_mle_rows<<<grid, 256, 0, st>>>(nrows, e, y, w, v, acc);
}

void launch_step(int32_t n, const double* x, const double* dx, double t, double* xt, cudaStream_t st) {
    if (n == 0) return;
    k_step<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(n, x, dx, t, xt);
}


// ---- Algorithm 1 of the appendix on the "empty-field" pattern: the background
// entry of row i (its one entry in the first k0 columns, the pointing's
// normalisation I_p^bg) holds U[upat_i] t_i; with x known the pattern is
// re-estimated from y^S (the counts of the other columns) and a_i = t_i x_c(i).

namespace {

constexpr int kBgThreads = 256;

// bgpos[i]: the position in H's values of row i's entry in the first k0 columns,
// -1 if it has none; flag set when a row has two such entries, or when its
// pattern index does not match (an entry needs 0 <= upat < npat, none needs -1)
__global__ void k_bg_locate(int64_t nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                            int32_t k0, const int32_t* __restrict__ upat, int32_t npat, int64_t* __restrict__ bgpos,
                            int* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t pos = -1;
        int cnt = 0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (colind[p] < k0) { pos = p; ++cnt; }
        const int32_t u = upat[i];
        const bool bad = cnt > 1 || (cnt == 1) != (u >= 0) || u >= npat;
        if (bad) atomicOr(flag, 1);
        bgpos[i] = bad ? -1 : pos;
    }
}

// hv[bgpos_i] = U[upat_i] t_i
__global__ void k_bg_write(int64_t nrows, const int64_t* __restrict__ bgpos, const int32_t* __restrict__ upat,
                           const double* __restrict__ t, const double* __restrict__ U, double* __restrict__ hv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = bgpos[i];
        if (p >= 0) hv[p] = U[upat[i]] * t[i];
    }
}

// One warp per row: y^S_i, a_i = t_i x_c(i), r_i = y_i - y^S_i and e_i = y^S_i + h_bg x_c(i).
// sums[k] / sums[npat + k]: the numerator / denominator of U_k,
//   least squares (kMle 0): r a w / a^2 w;  likelihood (kMle 1): r / a,
// accumulated per CTA in shared memory; acc[0] += the statistic at (U, x):
// w (y - e)^2, or e - y ln e; acc[1] += the rows with e <= 0 (likelihood).
template <int kMle>
__global__ void __launch_bounds__(kBgThreads) k_bg_sums(int64_t nrows, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ colind,
                                                        const double* __restrict__ hv, const double* __restrict__ x,
                                                        int32_t k0, const int64_t* __restrict__ bgpos,
                                                        const int32_t* __restrict__ upat,
                                                        const double* __restrict__ t, const double* __restrict__ y,
                                                        const double* __restrict__ w, int32_t npat,
                                                        double* __restrict__ sums, double* __restrict__ acc) {
    extern __shared__ double bsm[];  // [2 npat]
    for (int k = threadIdx.x; k < 2 * npat; k += kBgThreads) bsm[k] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double stat = 0.0, bad = 0.0;
    for (int64_t i = ((int64_t)blockIdx.x * kBgThreads + threadIdx.x) >> 5; i < nrows;
         i += ((int64_t)gridDim.x * kBgThreads) >> 5) {
        double s = 0.0;
        for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
            const int32_t j = colind[p];
            if (j >= k0) s += hv[p] * x[j];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const int64_t p = bgpos[i];
            double e = s, a = 0.0;
            if (p >= 0) {
                const double xc = x[colind[p]];
                a = t[i] * xc;
                e += hv[p] * xc;
            }
            const double yi = y[i];
            if (kMle) {
                if (e > 0.0) stat += yi > 0.0 ? e - yi * log(e) : e;
                else bad += 1.0;
            } else {
                const double d = yi - e;
                stat += w[i] * d * d;
            }
            if (p >= 0) {
                const int32_t k = upat[i];
                const double r = yi - s;
                if (kMle) {
                    atomicAdd(bsm + k, r);
                    atomicAdd(bsm + npat + k, a);
                } else {
                    const double wa = w[i] * a;
                    atomicAdd(bsm + k, r * wa);
                    atomicAdd(bsm + npat + k, a * wa);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        stat += __shfl_down_sync(0xffffffffu, stat, o);
        bad += __shfl_down_sync(0xffffffffu, bad, o);
    }
    if (lane == 0) {
        if (stat != 0.0) atomicAdd(acc, stat);
        if (bad != 0.0) atomicAdd(acc + 1, bad);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * npat; k += kBgThreads)
        if (bsm[k] != 0.0) atomicAdd(sums + k, bsm[k]);
}

// U_k = numerator / denominator where the denominator is positive
__global__ void k_bg_pattern(int32_t npat, const double* __restrict__ sums, double* __restrict__ U) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npat; k += gridDim.x * blockDim.x) {
        const double den = sums[npat + k];
        if (den > 0.0) U[k] = sums[k] / den;
    }
}

int bg_grid(int64_t nrows, int per_cta) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((nrows + per_cta - 1) / per_cta, 152 * 8));
}

}  // namespace

void launch_bg_locate(int64_t nrows, const int64_t* rowptr, const int32_t* colind, int32_t k0, const int32_t* upat,
                      int32_t npat, int64_t* bgpos, int* flag, cudaStream_t st) {
    if (nrows == 0) return;
    k_bg_locate<<<bg_grid(nrows, 256), 256, 0, st>>>(nrows, rowptr, colind, k0, upat, npat, bgpos, flag);
}

void launch_bg_write(int64_t nrows, const int64_t* bgpos, const int32_t* upat, const double* t, const double* U,
                     double* hv, cudaStream_t st) {
    if (nrows == 0) return;
    k_bg_write<<<bg_grid(nrows, 256), 256, 0, st>>>(nrows, bgpos, upat, t, U, hv);
}

void launch_bg_sums(bool mle, int64_t nrows, const int64_t* rowptr, const int32_t* colind, const double* hv,
                    const double* x, int32_t k0, const int64_t* bgpos, const int32_t* upat, const double* t,
                    const double* y, const double* w, int32_t npat, double* sums, double* acc, cudaStream_t st) {
    if (nrows == 0) return;
    const int grid = bg_grid(nrows, kBgThreads / 32);
    const size_t smem = 2 * (size_t)npat * sizeof(double);
    if (mle)
        k_bg_sums<1><<<grid, kBgThreads, smem, st>>>(nrows, rowptr, colind, hv, x, k0, bgpos, upat, t, y, w, npat,
                                                     sums, acc);
    else
        k_bg_sums<0><<<grid, kBgThreads, smem, st>>>(nrows, rowptr, colind, hv, x, k0, bgpos, upat, t, y, w, npat,
                                                     sums, acc);
}

void launch_bg_pattern(int32_t npat, const double* sums, double* U, cudaStream_t st) {
    if (npat == 0) return;
    k_bg_pattern<<<(npat + 255) / 256, 256, 0, st>>>(npat, sums, U);
}

}  // namespace spi
