// diag_tc_plan.cpp -- host plan of the tensor-core variance kernel
// (diag_tc.cu): which supernodes it takes, and the numbering of the packed
// left-operand tiles that both the packing kernel and the variance kernel use.
#include "diag_tc_plan.h"

namespace spi {

// Host plan: T = the supernodes with at least min_k pivots and all their
// ancestors (ascending postorder: children before parents, so one pass
// carries a mark to the root); their packed tiles in the order of
// k_diag_inv_tc's tile numbering; the diagonal tiles to invert.
void build_diag_tc(const Symbolic& S, int min_k, DiagTcHost& h) {
    h = DiagTcHost();
    h.tc.assign(S.ns, 0);
    h.tptr.assign(S.ns, -1);
    h.xptr.assign(S.ns, -1);
    if (min_k <= 0) return;
    for (int32_t s = 0; s < S.ns; ++s)
        if (S.k_of(s) >= min_k) h.tc[s] = 1;
    for (int32_t s = 0; s < S.ns; ++s)
        if (h.tc[s] && S.sparent[s] >= 0) h.tc[S.sparent[s]] = 1;
    int64_t npt = 0;
    int32_t ndt = 0;
    for (int32_t s = 0; s < S.ns; ++s) {
        if (!h.tc[s]) continue;
        ++h.ntc;
        const int32_t k = S.k_of(s), m = S.m_of(s);
        const int32_t T = (k + kDiagTcRows - 1) / kDiagTcRows, R = (m - k + kDiagTcRows - 1) / kDiagTcRows, nch = (k + kDiagTcK - 1) / kDiagTcK;
        h.tptr[s] = npt;
        h.xptr[s] = ndt;
        for (int32_t rt = 0; rt < T + R; ++rt) {
            const int32_t nck = diag_tc_row_chunks(T, nch, rt);
            for (int32_t c = 0; c < nck; ++c) {
                h.ptiles.insert(h.ptiles.end(), {s, rt, c, 0});
                ++npt;
            }
        }
        for (int32_t rt = 0; rt < T; ++rt) {
            h.dtiles.insert(h.dtiles.end(), {s, rt});
            ++ndt;
        }
    }
    h.npt = npt;
    h.ndt = ndt;
}

// TF32 MMA flops (3 products per output, the padded tile shapes) of one pass of
// k_diag_inv_tc over a plan's blocks, from the union list of every block.
double diag_tc_mma_flops(const Symbolic& S, const DiagTcHost& h, const DiagPlan& dp) {
    double fl = 0;
    for (int32_t b = 0; b < dp.nblocks; ++b)
        for (int32_t u = dp.uptr[b]; u < dp.uptr[b + 1]; ++u) {
            const int32_t s = dp.us[u];
            if (!h.tc[s]) continue;
            const int32_t k = S.k_of(s), m = S.m_of(s), nbu = dp.uhi[u] - dp.ulo[u];
            const double N = (double)((nbu + 31) & ~31);
            const int32_t T = (k + kDiagTcRows - 1) / kDiagTcRows, R = (m - k + kDiagTcRows - 1) / kDiagTcRows, nch = (k + kDiagTcK - 1) / kDiagTcK;
            double chunks = (double)R * nch;
            for (int32_t rt = 0; rt < T; ++rt) chunks += diag_tc_row_chunks(T, nch, rt);
            fl += chunks * 3.0 * 2.0 * kDiagTcRows * kDiagTcK * N;
        }
    return fl;
}
}  // namespace spi
