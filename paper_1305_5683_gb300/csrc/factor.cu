// factor.cu -- numerical factorization (paper Sec. 3.2.2): multifrontal
// LDL^T over the supernodal elimination tree, bottom-up level by level.
//
// Every front of supernode s is an m x m dense matrix whose first k columns
// (the panel, column-major, leading dimension m) hold the supernode's
// columns of N plus the contributions of its children, and whose trailing
// (m-k) x (m-k) part (F22, present only when s has children) accumulates the
// children's contribution blocks.  Per front:
//   F11 = L11 D1 L11^T, L21 = F21 L11^-T D1^-1: right-looking over block
//       columns of 32 -- the row tiles below the pivot tile (one CTA each),
//       then the rank-32 update of the trailing panel columns (one CTA per
//       32 x 32 tile), whose first tile is the next pivot tile: that CTA
//       factors it (FP64) right after its update;
//   C   = F22 - L21 D1 L21^T    (Schur complement tiles)
// and C is added into the parent's front through the parent-relative index
// map (the extend-add of the multifrontal method), with FP64 atomics because
// siblings of one level add into the same parent concurrently.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

#include "spi_internal.cuh"
#include "tcgen05.cuh"

namespace spi {

// Trailing blocks at least this tall go to the tensor-core Schur kernel in
// mixed precision.  Smaller fronts leave much of a 128 x 128 tile empty and
// run as fast on the SIMT kernel, whose FP32 accumulation is also a little
// more accurate than the tensor cores' (which truncate when aligning addends).
constexpr int32_t kTcMinRows = 2048;
// Trailing blocks this tall or taller may be given to the tensor cores by the
// autotuner (a smaller block leaves most of a 128 x 128 tile empty).
constexpr int32_t kTcMinLegal = 256;
// Wide fronts (mixed precision, more than kOuter pivots, at least kTcMinRows
// rows) are blocked twice: the 32-column steps update only the columns of
// their own kOuter-column block, and after every kOuter columns one
// tensor-core launch applies the rank-kOuter update to all remaining panel
// columns (kind 9); the next pivot tile is then factored by a kind-0 launch.
constexpr int32_t kOuter = 128;
constexpr int32_t kInner = kOuter / kT;
// tensor-core output tile (rows x columns) and K chunk; one thread per tile row
constexpr int kTcM = 128, kTcN = 128, kTcK = 32;
constexpr int kThreads = 128;  // threads of the SIMT front kernels
static_assert(kTcM == 128 && kTcN == 128, "the tensor-core kernels give thread t row t of both operand tiles");

int32_t ilog2_floor(int64_t v) {
    int32_t r = 0;
    while (v > 1) { v >>= 1; ++r; }
    return r;
}

int32_t panel_bucket(int64_t m, int64_t k) { return ilog2_floor(std::max<int64_t>(m, 1)) * 32 + ilog2_floor(std::max<int64_t>(k, 1)); }
int32_t schur_bucket(int64_t m, int64_t k) {
    return ilog2_floor(std::max<int64_t>(m - k, 1)) * 32 + ilog2_floor(std::max<int64_t>(k, 1));
}

bool wide_front(bool tensor_cores, int64_t m, int64_t k) { return tensor_cores && k > kOuter && m >= kTcMinRows; }
bool schur_tc_legal(bool tensor_cores, int64_t m, int64_t k) { return tensor_cores && m - k >= kTcMinLegal && k >= 32; }
// A panel may run in one CTA of the per-level kernel when its work is bounded
// (about m k^2 / 2 multiply-adds on one SM).
bool fused_legal(int64_t m, int64_t k) { return m * k * k <= ((int64_t)1 << 26) && k <= 512; }

// Built-in rules, used for buckets the autotuner has not timed: the panel of a
// front runs in one CTA when its work (about m k^2 / 2 multiply-adds plus the
// chain of ceil(k / 32) block steps) is small; the Schur complement goes to
// the tensor cores from kTcMinRows trailing rows on.
bool rule_fused(int64_t m, int64_t k) { return m * k * k <= (int64_t)1 << 22 && k <= 256; }
bool rule_schur_tc(int64_t m, int64_t k) { return m - k >= kTcMinRows; }

namespace {

// The panel work of a front (for ordering the persistent kernel's items).
int64_t panel_cost(const Symbolic& S, int32_t s) {
    const int64_t k = S.k_of(s), m = S.m_of(s);
    return S.sdiag[s] ? m * k : m * k * k / 2 + k * 1024;
}

// One launch of the persistent per-level panel kernel (kind 12) over `fronts`,
// heaviest first (diagonal-pivot fronts are encoded as ~s).
void append_fused(const Symbolic& S, FactorPlan& F, std::vector<int32_t> fronts) {
    if (fronts.empty()) return;
    std::stable_sort(fronts.begin(), fronts.end(),
                     [&](int32_t a, int32_t b) { return panel_cost(S, a) > panel_cost(S, b); });
    Launch l{12, 0, (int64_t)F.fused_items.size(), (int32_t)fronts.size()};
    for (int32_t s : fronts) F.fused_items.push_back(S.sdiag[s] ? ~s : s);
    F.launches.push_back(l);
}

// The block-step chain of `fronts` (none with a diagonal pivot block): per
// 32-column step, the pivot tiles that start an outer block, the row tiles of
// the panel solve, the trailing panel update (whose first tile factors the
// next pivot tile) and, for wide fronts in mixed precision, the rank-kOuter
// tensor-core update at the end of each outer block.
void append_tiled(const Symbolic& S, FactorPlan& F, const std::vector<int32_t>& fronts, bool tensor_cores) {
    int32_t kmax = 0;
    for (int32_t s : fronts) kmax = std::max(kmax, S.k_of(s));
    const int32_t nsteps = (kmax + kT - 1) / kT;
    for (int32_t b = 0; b < nsteps; ++b) {
        Launch ld{0, b, (int64_t)F.diag_items.size(), 0};
        Launch lt{1, b, (int64_t)F.trsm_items.size() / 2, 0};
        Launch lu{3, b, (int64_t)F.update_items.size() / 3, 0};
        Launch lw{9, b, (int64_t)F.panel_tc_items.size() / 3, 0};
        for (int32_t s : fronts) {
            const int32_t k = S.k_of(s), m = S.m_of(s);
            if (k <= b * kT) continue;
            const bool wide = wide_front(tensor_cores, m, k);
            if (b == 0 || (wide && b % kInner == 0)) {
                F.diag_items.push_back(s);
                ld.count++;
            }
            const int32_t w = std::min(kT, k - b * kT), r0 = b * kT + w;
            for (int32_t rt = 0; r0 + rt * kT < m; ++rt) {
                F.trsm_items.push_back(s);
                F.trsm_items.push_back(rt);
                lt.count++;
            }
            // trailing panel columns [r0, kend): lower tiles of rows [cj, m)
            const int32_t kend = wide ? std::min(k, kOuter * (b / kInner + 1)) : k;
            for (int32_t tj = 0; r0 + tj * kT < kend; ++tj) {
                const int32_t cj = r0 + tj * kT;
                for (int32_t ti = 0; cj + ti * kT < m; ++ti) {
                    F.update_items.push_back(s);
                    F.update_items.push_back(ti);
                    F.update_items.push_back(tj);
                    lu.count++;
                }
            }
            // end of an outer block: rank-kOuter update of panel columns [r0, k)
            if (wide && r0 == kend && r0 < k) {
                for (int32_t ti = 0; r0 + ti * kTcM < m; ++ti)
                    for (int32_t tj = 0; r0 + tj * kTcN < k && tj * kTcN <= ti * kTcM + kTcM - 1; ++tj) {
                        F.panel_tc_items.push_back(s);
                        F.panel_tc_items.push_back(ti);
                        F.panel_tc_items.push_back(tj);
                        lw.count++;
                    }
            }
        }
        if (ld.count) F.launches.push_back(ld);
        if (lt.count) F.launches.push_back(lt);
        if (lu.count) F.launches.push_back(lu);
        if (lw.count) F.launches.push_back(lw);
    }
}

// Schur complements of `simt` (32 x 32 tiles, kind 2) and `tc` (128 x 128
// tensor-core tiles, kind 7), each added into its parent's front.
void append_schur(const Symbolic& S, FactorPlan& F, const std::vector<int32_t>& simt, const std::vector<int32_t>& tc) {
    Launch ls{2, 0, (int64_t)F.schur_items.size() / 3, 0};
    for (int32_t s : simt) {
        const int32_t k = S.k_of(s), m = S.m_of(s);
        const int32_t nt = (m - k + kT - 1) / kT;
        for (int32_t ti = 0; ti < nt; ++ti)
            for (int32_t tj = 0; tj <= ti; ++tj) {
                F.schur_items.push_back(s);
                F.schur_items.push_back(ti);
                F.schur_items.push_back(tj);
                ls.count++;
            }
    }
    Launch lc{7, 0, (int64_t)F.schur_tc_items.size() / 3, 0};
    for (int32_t s : tc) {
        const int32_t k = S.k_of(s), m = S.m_of(s);
        for (int32_t ti = 0; ti * kTcM < m - k; ++ti)
            for (int32_t tj = 0; tj * kTcN < m - k && tj * kTcN <= ti * kTcM + kTcM - 1; ++tj) {
                F.schur_tc_items.push_back(s);
                F.schur_tc_items.push_back(ti);
                F.schur_tc_items.push_back(tj);
                lc.count++;
            }
    }
    if (ls.count) F.launches.push_back(ls);
    if (lc.count) F.launches.push_back(lc);
}

}  // namespace

bool FactorChoice::fused(int64_t m, int64_t k) const {
    if (force_panel == 1) return false;
    if (force_panel == 2) return true;
    auto it = panel.find(panel_bucket(m, k));
    return it != panel.end() ? it->second != 0 : rule_fused(m, k);
}

bool FactorChoice::schur_tc(int64_t m, int64_t k) const {
    if (force_schur == 1) return false;
    if (force_schur == 2) return true;
    auto it = schur.find(schur_bucket(m, k));
    return it != schur.end() ? it->second != 0 : rule_schur_tc(m, k);
}

namespace {

// The tasks of the dependency-driven kernel for levels [0, nlev): per level,
// phase by phase across the level's fronts (a front's Schur tiles at the phase
// after its last), so that the order is topological (see k_factor_dag).
void build_dag(const Symbolic& S, FactorPlan& F, int32_t nlev, const std::vector<uint8_t>& fused) {
    const int32_t ns = S.ns;
    std::vector<int32_t> child_tiles(ns, 0);  // Schur tiles the children of each front add in
    for (int32_t l = 0; l < nlev; ++l) {
        std::vector<std::vector<std::vector<DagTask>>> ph;  // [front of the level][phase] tasks
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p];
            const int32_t k = S.k_of(s), m = S.m_of(s);
            std::vector<std::vector<DagTask>> t;
            auto task = [&](int32_t type, int32_t a, int32_t b) { return DagTask{type, s, a, b, 0, 0, s, 0}; };
            if (S.sdiag[s]) t.push_back({task(kDagDiagFront, 0, 0)});
            else if (fused[s]) t.push_back({task(kDagFused, 0, 0)});
            else {
                t.push_back({task(kDagPivot, 0, 0)});
                for (int32_t b = 0; b * kT < k; ++b) {
                    const int32_t w = std::min(kT, k - b * kT), r0 = b * kT + w;
                    std::vector<DagTask> tr, up;
                    for (int32_t c = 0; r0 + (int64_t)c * kThreads < m; ++c) tr.push_back(task(kDagTrsm, b, c));
                    for (int32_t tj = 0; r0 + tj * kT < k; ++tj)
                        for (int32_t ti = 0; r0 + tj * kT + ti * kT < m; ++ti) up.push_back(task(kDagUpdate, b, (ti << 16) | tj));
                    if (!tr.empty()) t.push_back(tr);
                    if (!up.empty()) t.push_back(up);
                }
            }
            // waits: the first phase on the children's Schur tiles, later phases on the
            // front's own earlier tasks
            int32_t done = 0;
            for (size_t q = 0; q < t.size(); ++q) {
                for (DagTask& x : t[q]) {
                    x.wait_idx = q == 0 ? ns + s : s;
                    x.wait_val = q == 0 ? child_tiles[s] : done;
                }
                done += (int32_t)t[q].size();
            }
            std::vector<DagTask> sc;
            const int32_t par = S.sparent[s];
            if (par != -1 && m > k) {
                const int32_t nt = (m - k + kT - 1) / kT;
                for (int32_t ti = 0; ti < nt; ++ti)
                    for (int32_t tj = 0; tj <= ti; ++tj) sc.push_back(DagTask{kDagSchur, s, ti, tj, s, done, ns + par, 0});
                child_tiles[par] += (int32_t)sc.size();
            }
            if (!sc.empty()) t.push_back(sc);
            ph.push_back(std::move(t));
        }
        size_t maxp = 0;
        for (auto& t : ph) maxp = std::max(maxp, t.size());
        for (size_t q = 0; q < maxp; ++q)
            for (auto& t : ph)
                if (q < t.size()) F.dag.insert(F.dag.end(), t[q].begin(), t[q].end());
    }
}

}  // namespace

void build_factor_plan(const Symbolic& S, FactorPlan& F, bool tensor_cores_allowed, const FactorChoice& ch,
                       bool markers) {
    F = FactorPlan();
    const bool tensor_cores = tensor_cores_allowed && ch.force_schur != 1;  // 1: no tensor-core launch at all
    if (ch.dag && !markers) {
        // the levels before the first one with a tensor-core launch run as one dependency-driven launch
        int32_t nlev = S.nlevels;
        std::vector<uint8_t> fused(S.ns, 0);
        for (int32_t l = 0; l < S.nlevels && nlev == S.nlevels; ++l)
            for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
                const int32_t s = S.level_list[p];
                const int32_t k = S.k_of(s), m = S.m_of(s);
                const bool tc_schur = S.sparent[s] != -1 && m > k && schur_tc_legal(tensor_cores, m, k) && ch.schur_tc(m, k);
                if (tc_schur || (!S.sdiag[s] && wide_front(tensor_cores, m, k))) { nlev = l; break; }
                fused[s] = !S.sdiag[s] && fused_legal(m, k) && ch.force_panel != 1 && ch.fused(m, k);
            }
        build_dag(S, F, nlev, fused);
        F.dag_levels = nlev;
        if (!F.dag.empty()) F.launches.push_back(Launch{13, 0, 0, (int32_t)F.dag.size()});
    }
    F.level_launch_ptr.push_back(0);
    auto marker = [&](int kind, int32_t bucket) {
        F.launches.push_back(Launch{-1, (int)F.groups.size(), 0, 0});
        F.groups.push_back(FactorPlan::Group{kind, bucket});
    };
    for (int32_t l = F.dag_levels; l < S.nlevels; ++l) {
        // panels: fronts with a diagonal pivot block always run in the persistent
        // kernel; wide fronts of the mixed form always run the tiled chain (their
        // tensor-core trailing updates); the rest as chosen per bucket
        std::map<int32_t, std::vector<int32_t>> fused_by, tiled_by;
        std::vector<int32_t> diag_fronts;
        std::map<int32_t, std::vector<int32_t>> simt_by, tc_by;
        for (int32_t p = S.level_ptr[l]; p < S.level_ptr[l + 1]; ++p) {
            const int32_t s = S.level_list[p];
            const int32_t k = S.k_of(s), m = S.m_of(s);
            if (S.sdiag[s]) diag_fronts.push_back(s);
            else if (!wide_front(tensor_cores, m, k) && fused_legal(m, k) && ch.fused(m, k))
                fused_by[panel_bucket(m, k)].push_back(s);
            else tiled_by[panel_bucket(m, k)].push_back(s);
            if (S.sparent[s] == -1 || m <= k) continue;
            if (schur_tc_legal(tensor_cores, m, k) && ch.schur_tc(m, k)) tc_by[schur_bucket(m, k)].push_back(s);
            else simt_by[schur_bucket(m, k)].push_back(s);
        }
        if (ch.force_panel == 1 && !diag_fronts.empty()) {
            // every panel on the block-step kernels: diagonal-pivot fronts one CTA each (kind 8)
            if (markers) marker(FactorPlan::kDiagFronts, -1);
            F.launches.push_back(Launch{8, 0, (int64_t)F.dfront_items.size(), (int32_t)diag_fronts.size()});
            F.dfront_items.insert(F.dfront_items.end(), diag_fronts.begin(), diag_fronts.end());
            diag_fronts.clear();
        }
        if (markers) {
            // one timed group per (kind, bucket) of the level, launched on its own
            if (!diag_fronts.empty()) { marker(FactorPlan::kDiagFronts, -1); append_fused(S, F, diag_fronts); }
            for (auto& kv : fused_by) { marker(FactorPlan::kPanel, kv.first); append_fused(S, F, kv.second); }
            for (auto& kv : tiled_by) { marker(FactorPlan::kPanel, kv.first); append_tiled(S, F, kv.second, tensor_cores); }
            for (auto& kv : simt_by) { marker(FactorPlan::kSchur, kv.first); append_schur(S, F, kv.second, {}); }
            for (auto& kv : tc_by) { marker(FactorPlan::kSchur, kv.first); append_schur(S, F, {}, kv.second); }
        } else {
            std::vector<int32_t> fused(diag_fronts), tiled, simt, tc;
            for (auto& kv : fused_by) fused.insert(fused.end(), kv.second.begin(), kv.second.end());
            for (auto& kv : tiled_by) tiled.insert(tiled.end(), kv.second.begin(), kv.second.end());
            for (auto& kv : simt_by) simt.insert(simt.end(), kv.second.begin(), kv.second.end());
            for (auto& kv : tc_by) tc.insert(tc.end(), kv.second.begin(), kv.second.end());
            std::sort(tiled.begin(), tiled.end());
            std::sort(simt.begin(), simt.end());
            std::sort(tc.begin(), tc.end());
            append_fused(S, F, fused);
            append_tiled(S, F, tiled, tensor_cores);
            append_schur(S, F, simt, tc);
        }
        F.level_launch_ptr.push_back((int32_t)F.launches.size());
    }
    if (markers) marker(FactorPlan::kEnd, -1);
    for (const Launch& la : F.launches) {
        if (la.kind == 12) F.n_fused_launches++;
        if (la.kind == 7 || la.kind == 9) { F.n_tc_launches++; F.n_tc_tiles += la.count; }
        if (la.kind >= 0) F.n_kernel_launches++;
    }
    // flops the SIMT kernels execute (full 32 x 32 tiles, explicit zeros included;
    // a multiply-add counts 2), against the algorithmic count from exact column counts
    auto w_of = [&](int32_t s, int32_t b) { return (double)std::min(kT, S.k_of(s) - b * kT); };
    for (const Launch& la : F.launches) {
        if (la.kind == 0)
            for (int32_t q = 0; q < la.count; ++q) F.work_flops += 2.0 * std::pow(w_of(F.diag_items[la.off + q], la.step), 3) / 3.0;
        if (la.kind == 1)
            for (int32_t q = 0; q < la.count; ++q) {
                const double w = w_of(F.trsm_items[2 * (la.off + q)], la.step);
                F.work_flops += kT * w * w;
            }
        if (la.kind == 3)
            for (int32_t q = 0; q < la.count; ++q) {
                const double w = w_of(F.update_items[3 * (la.off + q)], la.step);
                F.work_flops += 2.0 * kT * kT * w + (F.update_items[3 * (la.off + q) + 1] == 0 &&
                                                     F.update_items[3 * (la.off + q) + 2] == 0 ? 2.0 * kT * kT * kT / 3.0 : 0.0);
            }
        if (la.kind == 2)
            for (int32_t q = 0; q < la.count; ++q) F.work_flops += 2.0 * kT * kT * S.k_of(F.schur_items[3 * (la.off + q)]);
        if (la.kind == 13)
            for (const DagTask& t : F.dag) {
                const double k = S.k_of(t.s), m = S.m_of(t.s);
                if (t.type == kDagFused) F.work_flops += m * k * k - 2.0 * k * k * k / 3.0;
                if (t.type == kDagPivot) F.work_flops += 2.0 * std::pow(std::min<double>(kT, k), 3) / 3.0;
                if (t.type == kDagTrsm) F.work_flops += kThreads * std::pow(std::min<double>(kT, k - t.a * kT), 2);
                if (t.type == kDagUpdate) F.work_flops += 2.0 * kT * kT * std::min<double>(kT, k - t.a * kT);
                if (t.type == kDagSchur) F.work_flops += 2.0 * kT * kT * k;
            }
        if (la.kind == 12)
            for (int32_t q = 0; q < la.count; ++q) {
                const int32_t code = F.fused_items[la.off + q];
                if (code < 0) continue;
                const double k = S.k_of(code), m = S.m_of(code);
                F.work_flops += m * k * k - 2.0 * k * k * k / 3.0;  // the panel's LDL^T part of the front
            }
    }
    // tensor-core work: per tile, K rounded up to the 32-wide chunk, 6 MMAs per product
    for (size_t t = 0; t < F.schur_tc_items.size(); t += 3)
        F.tc_flops += 2.0 * kTcM * kTcN * (double)((S.k_of(F.schur_tc_items[t]) + kTcK - 1) / kTcK * kTcK) * 6.0;
    F.tc_flops += 2.0 * kTcM * kTcN * (double)kOuter * 6.0 * (double)(F.panel_tc_items.size() / 3);
}

namespace {

template <typename S>
__global__ void k_assemble(const int64_t* __restrict__ amap, const double* __restrict__ vals, int64_t nnz,
                           S* __restrict__ L, const int32_t* __restrict__ diag_src, int32_t n,
                           double* __restrict__ adiag, Strides bs) {
    vals += blockIdx.y * bs.nnz;
    L += blockIdx.y * bs.L;
    adiag += blockIdx.y * bs.n;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = i; p < nnz; p += stride) L[amap[p]] = (S)vals[p];
    for (int64_t j = i; j < n; j += stride) adiag[j] = vals[diag_src[j]];
}

// A load of data that another CTA of the same launch may have written (the
// dependency-driven kernel): through L2 only (ld.global.cg), never from an L1
// line this SM cached before that CTA's store.  Plain loads otherwise.
template <bool kCg, typename T>
__device__ __forceinline__ T ldx(const T* p) {
    if constexpr (kCg) return __ldcg(p);
    else return *p;
}

// 1/d in FP64 with three FP64 operations on the dependency chain (a dependent FP64
// operation costs about 64 cycles on this GPU; a division or a conversion to and from
// single precision costs several).  d = m 2^(ex - 1023) with m in [1, 2): a single-
// precision seed r0 ~ 1/m is formed from m's top 23 mantissa bits by bit operations and
// one __frcp_rn, then refined by one step of the third-order reciprocal iteration (the
// Newton-Raphson iteration for 1/m carried one term further: 1/m = r0 / (1 - e) =
// r0 (1 + e + e^2 + ...), e = 1 - m r0), r0 (1 + e + e^2); |e| < 2^-22, so the dropped
// e^3 term is below FP64 rounding and the result is within 2 ulp of the correctly
// rounded 1/m (measured against 1.0 / d over 2^22 values spanning 2^-60 .. 2^60:
// at most 1.93 ulp).  The exponent is restored by integer arithmetic.  Zero,
// subnormal, huge or non-finite d divide.
__device__ __forceinline__ double recip_fp64(double d) {
    const long long b = __double_as_longlong(d);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex < 4 || ex > 2042) return 1.0 / d;
    const double m = __longlong_as_double((b & 0x800FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
    const float mf = __int_as_float((int)((b >> 29) & 0x7FFFFF) | 0x3F800000 | (int)((b >> 32) & 0x80000000LL));
    const int rb = __float_as_int(__frcp_rn(mf));  // in (0.5, 1]
    const double r0 = __longlong_as_double(((long long)(rb & 0x80000000) << 32) |
                                           ((long long)(((rb >> 23) & 0xff) - 127 + 1023) << 52) |
                                           ((long long)(rb & 0x7FFFFF) << 29));
    const double e = fma(-m, r0, 1.0);
    const double r = fma(r0, fma(e, e, e), r0);
    return __longlong_as_double(__double_as_longlong(r) - ((long long)(ex - 1023) << 52));
}

// Entries of the lower triangle of order kT - 2, row by row: entry e is (e >> 8, e & 255).
constexpr int kTri = (kT - 2) * (kT - 1) / 2;

// Unblocked LDL^T, in FP64, of the w x w pivot tile whose first pivot is
// column c0 of supernode s (panel P of storage type S, leading dimension m),
// by the CTA's 128 threads; writes L (unit lower, d on the diagonal) back into
// P, d into D (FP64) and into DS (the storage type's copy used for scaling).
// The tile is bound by its column-to-column dependency chain, not by FP64
// throughput, so the work is split by that chain.  Per column c, one barrier
// apart: warp 3 forms column c + 1 -- its last update, the pivot
// d_{c+1} = a_{c+1,c+1} - a_{c+1,c} l_{c+1,c} and 1/d_{c+1} (every lane
// computes them: one lane costs as much as 32), then l_{j,c+1} = a_{j,c+1} / d_{c+1}
// -- while warps 0-2 apply column c to the rest of the triangle,
// a_ij -= a_ic l_jc for c + 2 <= j <= i (from a table of the triangle's
// entries).  The scaled columns of L wait in the tile's unused upper triangle
// until the end; the pivots are checked there, all at once.
template <typename S, bool kCg = false>
__device__ void factor_pivot_tile(double (*A)[kT + 1], double* dv, S* P, int64_t m, int c0, int w,
                                  int f, double* D, S* DS, const double* __restrict__ adiag, DevStatus* status,
                                  int band_base) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ double lc[2][kT];    // l_{j,c} of the column being applied, alternating
    __shared__ uint16_t tri[kTri];
    static_assert(kThreads == 128 && kT == 32, "three update warps and one pivot warp over a 32 x 32 tile");
    for (int e = tid; e < kT * kT; e += kThreads) {
        const int i = e % kT, j = e / kT;
        if (i < w && j <= i) A[i][j] = (double)ldx<kCg>(P + (c0 + i) + (int64_t)(c0 + j) * m);
    }
    for (int e = tid; e < kTri; e += kThreads) {
        int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        if ((i + 1) * (i + 2) / 2 <= e) ++i;
        if (i * (i + 1) / 2 > e) --i;
        tri[e] = (uint16_t)((i << 8) | (e - i * (i + 1) / 2));
    }
    __syncthreads();
    if (warp == 3) {  // column 0
        const double d = A[0][0];
        const double inv = recip_fp64(d);
        if (lane == 0) dv[0] = d;
        if (lane > 0 && lane < w) {
            const double l = A[lane][0] * inv;
            lc[0][lane] = l;
            A[0][lane] = l;
        }
    }
    __syncthreads();
    for (int c = 0; c + 1 < w; ++c) {
        const double* l = lc[c & 1];
        if (warp == 3) {
            const int j = lane;
            const double lcc = l[c + 1];
            const double d = fma(-A[c + 1][c], lcc, A[c + 1][c + 1]);
            double a = 0.0;
            if (j > c + 1 && j < w) a = fma(-A[j][c], lcc, A[j][c + 1]);
            const double inv = recip_fp64(d);
            if (j == c + 1) dv[c + 1] = d;
            if (j > c + 1 && j < w) {
                const double lj = a * inv;
                A[j][c + 1] = a;
                lc[(c + 1) & 1][j] = lj;
                A[c + 1][j] = lj;
            }
        } else {
            const int n = w - 2 - c, N = n * (n + 1) / 2;
            for (int e = tid; e < N; e += 2 * 96) {
                const int e2 = e + 96;
                const int t = tri[e], t2 = tri[e2 < N ? e2 : e];
                const int gi = c + 2 + (t >> 8), gj = c + 2 + (t & 255);
                const int gi2 = c + 2 + (t2 >> 8), gj2 = c + 2 + (t2 & 255);
                const double v = fma(-A[gi][c], l[gj], A[gi][gj]);
                const double v2 = fma(-A[gi2][c], l[gj2], A[gi2][gj2]);
                A[gi][gj] = v;
                if (e2 < N) A[gi2][gj2] = v2;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < kT * kT; e += kThreads) {
        const int i = e % kT, j = e / kT;
        if (i < w && j <= i) P[(c0 + i) + (int64_t)(c0 + j) * m] = (S)(i == j ? dv[i] : A[j][i]);
    }
    if (tid < w) {
        const double dc = dv[tid];
        if (!(dc > 0.0) || dc <= 1e-14 * adiag[f + c0 + tid]) {
            atomicOr(&status->flags, FLAG_NOT_SPD);
            atomicMin(&status->bad_pivot, band_base + f + c0 + tid);
        }
        D[f + c0 + tid] = dc;
        DS[f + c0 + tid] = (S)dc;
    }
}

// Pivot tile of block column 0 of every supernode of a level (the pivot
// tiles of later block columns are factored by the trailing-update CTA that
// writes them last, k_panel_update).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_diag_tile(DevSym d, const int32_t* __restrict__ items, int b,
                                                        S* __restrict__ L, double* __restrict__ D, S* __restrict__ DS,
                                                        const double* __restrict__ adiag, DevStatus* status,
                                                        Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    DS += blockIdx.y * bs.n;
    adiag += blockIdx.y * bs.n;
    __shared__ double A[kT][kT + 1];
    __shared__ double dv[kT];
    const int s = items[blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const int c0 = b * kT;
    factor_pivot_tile(A, dv, L + d.lptr[s], m, c0, min(kT, k - c0), f, D, DS, adiag, status,
                      (int)(blockIdx.y * bs.n));
}

// Front with a diagonal pivot block (independent leaf columns grouped into
// one front, no children): d_c is the input diagonal entry (kept in FP64 in
// adiag) and L21(:, c) = F21(:, c) / d_c.
template <typename S, bool kCg = false>
__device__ void diag_front_body(const DevSym& d, int s, S* L, double* D, S* DS, const double* __restrict__ adiag,
                                DevStatus* status, int band_base) {
    const int tid = threadIdx.x;
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    S* P = L + d.lptr[s];
    for (int c = tid; c < k; c += kThreads) {
        const double dc = adiag[f + c];
        if (!(dc > 0.0)) {
            atomicOr(&status->flags, FLAG_NOT_SPD);
            atomicMin(&status->bad_pivot, band_base + f + c);
        }
        D[f + c] = dc;
        DS[f + c] = (S)dc;
        P[c + (int64_t)c * m] = (S)dc;
    }
    // one reciprocal per column (uniform across the CTA), then scale its rows
    for (int c = 0; c < k; ++c) {
        const S rc = (S)(1.0 / adiag[f + c]);
        for (int64_t r = k + tid; r < m; r += kThreads) P[r + (int64_t)c * m] = ldx<kCg>(P + r + (int64_t)c * m) * rc;
    }
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_diag_front(DevSym d, const int32_t* __restrict__ items,
                                                         S* __restrict__ L, double* __restrict__ D, S* __restrict__ DS,
                                                         const double* __restrict__ adiag, DevStatus* status,
                                                         Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    DS += blockIdx.y * bs.n;
    adiag += blockIdx.y * bs.n;
    diag_front_body(d, items[blockIdx.x], L, D, DS, adiag, status, (int)(blockIdx.y * bs.n));
}

// Shared memory of the per-level panel kernel; the three phases of a block
// step use it in turn.
template <typename C>
union FrontPanelSmem {
    struct {
        double A[kT][kT + 1];
        double dv[kT];
    } piv;                      // the FP64 pivot tile
    struct {
        C Bd[kT][kT + 1];       // strictly lower part of the factored pivot tile
        C rd[kT];               // 1 / d of its pivots
        C X[kThreads][kT + 1];  // one row of the panel solve per thread
    } trsm;
    struct {
        C Li[kT][kT + 1];       // 32 rows of the block column
        C Lj[kT][kT + 1];       // 32 rows of the block column scaled by d
    } upd;
};

// A whole front's panel by one CTA: per 32-column block step, the FP64 pivot
// tile, the panel solve of every row below it (one thread per row), then the
// rank-32 update of the remaining panel columns in 32 x 32 tiles.  The Schur
// complement is left to the Schur tiles.
template <typename C, bool kCg>
__device__ void front_panel_body(const DevSym& d, int s, C* Lb, double* Db, C* DSb, const double* ab,
                                 DevStatus* status, int base, FrontPanelSmem<C>& sm) {
    const int tid = threadIdx.x;
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    C* P = Lb + d.lptr[s];
    for (int c0 = 0; c0 < k; c0 += kT) {
        const int w = min(kT, k - c0);
        __syncthreads();
        factor_pivot_tile<C, kCg>(sm.piv.A, sm.piv.dv, P, m, c0, w, f, Db, DSb, ab, status, base);
        __syncthreads();
        // L21 = X L11^-T D^-1 for the rows below the pivot tile
        for (int e = tid; e < kT * kT; e += kThreads) {
            const int i = e % kT, j = e / kT;
            sm.trsm.Bd[i][j] = (i < w && j < i) ? ldx<kCg>(P + (c0 + i) + (int64_t)(c0 + j) * m) : C(0);
        }
        if (tid < kT) sm.trsm.rd[tid] = tid < w ? (C)(1.0 / ldx<kCg>(Db + f + c0 + tid)) : C(0);
        __syncthreads();
        C* xr = sm.trsm.X[tid];
        for (int64_t r = c0 + w + tid; r < m; r += kThreads) {
            for (int c = 0; c < w; ++c) xr[c] = ldx<kCg>(P + r + (int64_t)(c0 + c) * m);
            for (int c = 1; c < w; ++c) {
                C y = xr[c];
                for (int cp = 0; cp < c; ++cp) y -= xr[cp] * sm.trsm.Bd[c][cp];
                xr[c] = y;
            }
            for (int c = 0; c < w; ++c) P[r + (int64_t)(c0 + c) * m] = xr[c] * sm.trsm.rd[c];
        }
        // rank-w update of panel columns [c0 + w, k), rows i >= j, in 32 x 32 tiles:
        // P[i][j] -= sum_c L[i][c] d_c L[j][c]; thread (ii, j0) owns row ii, columns j0 + 4 q
        const int ii = tid % kT, j0 = tid / kT;
        for (int cj = c0 + w; cj < k; cj += kT) {
            const int nj = min(kT, k - cj);
            __syncthreads();  // the panel solve (or the previous column tile) is done
            for (int e = tid; e < kT * kT; e += kThreads) {
                const int i = e % kT, c = e / kT;
                sm.upd.Lj[i][c] = (i < nj && c < w)
                                      ? ldx<kCg>(P + (cj + i) + (int64_t)(c0 + c) * m) * ldx<kCg>(DSb + f + c0 + c)
                                      : C(0);
            }
            for (int64_t ri = cj; ri < m; ri += kT) {
                const int ni = (int)(m - ri < kT ? m - ri : kT);
                __syncthreads();
                for (int e = tid; e < kT * kT; e += kThreads) {
                    const int i = e % kT, c = e / kT;
                    sm.upd.Li[i][c] = (i < ni && c < w) ? ldx<kCg>(P + (ri + i) + (int64_t)(c0 + c) * m) : C(0);
                }
                __syncthreads();
                if (ii < ni) {
                    C acc[kT / 4];
#pragma unroll
                    for (int q = 0; q < kT / 4; ++q) acc[q] = C(0);
#pragma unroll 4
                    for (int c = 0; c < w; ++c) {
                        const C ai = sm.upd.Li[ii][c];
#pragma unroll
                        for (int q = 0; q < kT / 4; ++q) acc[q] += ai * sm.upd.Lj[j0 + 4 * q][c];
                    }
                    C old[kT / 4];
#pragma unroll
                    for (int q = 0; q < kT / 4; ++q) {
                        const int jj = j0 + 4 * q;
                        old[q] = (jj < nj && ri + ii >= cj + jj) ? ldx<kCg>(P + (ri + ii) + (int64_t)(cj + jj) * m)
                                                                   : C(0);
                    }
#pragma unroll
                    for (int q = 0; q < kT / 4; ++q) {
                        const int jj = j0 + 4 * q;
                        if (jj < nj && ri + ii >= cj + jj) P[(ri + ii) + (int64_t)(cj + jj) * m] = old[q] - acc[q];
                    }
                }
            }
        }
    }
}

// Persistent per-level panel kernel (kind 12): the CTAs walk the level's list
// of fronts (heaviest first, in steps of the grid; item t is front
// items[t / nb] of band t % nb) and each processes a whole front's panel on
// its own, so a small front costs one launch per level instead of three or
// more per 32-column block step.  A front with a diagonal pivot block (~s in
// the list) is scaled column by column.  The CTAs never wait on one another.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_front_panel(DevSym d, const int32_t* __restrict__ items, int nitems,
                                                          int nb, C* __restrict__ L, double* __restrict__ D,
                                                          C* __restrict__ DS, const double* __restrict__ adiag,
                                                          DevStatus* status, Strides bs) {
    __shared__ FrontPanelSmem<C> sm;
    const int64_t total = (int64_t)nitems * nb;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int band = (int)(t % nb);
        const int code = items[t / nb];
        C* Lb = L + band * bs.L;
        double* Db = D + band * bs.n;
        C* DSb = DS + band * bs.n;
        const double* ab = adiag + band * bs.n;
        const int base = (int)(band * bs.n);
        __syncthreads();  // the previous front's last phase is done with the shared memory
        if (code < 0) diag_front_body(d, ~code, Lb, Db, DSb, ab, status, base);
        else front_panel_body<C, false>(d, code, Lb, Db, DSb, ab, status, base, sm);
    }
}

// Row tile rt below the diagonal tile of block column b (already updated by
// the block columns before it): L21 = X L11^-T D^-1.  Four lanes per row (warp
// w holds rows 8 w .. 8 w + 7, lane q = lane % 4 of a row's group the columns
// q, q + 4, ...): column c is final at its owner when the columns before it
// have been applied; a shuffle hands it to the row's other lanes, which apply
// it to their later columns.  All four warps work (a narrow FP64 pipe gives
// one warp a quarter of the SM's rate), and the dependency chain per column is
// one shuffle and one multiply-add.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_panel_trsm(DevSym d, const int32_t* __restrict__ items, int b,
                                                         C* __restrict__ L, const double* __restrict__ D,
                                                         Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    __shared__ C Bd[kT][kT + 1];
    __shared__ C dv[kT];
    const int tid = threadIdx.x, lane = tid & 31, q = lane & 3;
    const int s = items[2 * blockIdx.x], rt = items[2 * blockIdx.x + 1];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    C* P = L + d.lptr[s];
    const int c0 = b * kT, w = min(kT, k - c0);
    const int64_t r0 = c0 + w + (int64_t)rt * kT;
    const int nr = (int)(m - r0 < kT ? m - r0 : kT);
    const int r = 8 * (tid >> 5) + (lane >> 2);
    const bool on = r < nr;
    for (int e = tid; e < kT * kT; e += kThreads) {
        const int i = e % kT, j = e / kT;
        Bd[i][j] = (i < w && j < i) ? P[(c0 + i) + (int64_t)(c0 + j) * m] : C(0);
    }
    if (tid < kT) dv[tid] = (tid < w) ? (C)recip_fp64(D[f + c0 + tid]) : C(0);
    C y[kT / 4];  // y[t]: column 4 t + q of row r
#pragma unroll
    for (int t = 0; t < kT / 4; ++t) {
        const int c = 4 * t + q;
        y[t] = (on && c < w) ? P[(r0 + r) + (int64_t)(c0 + c) * m] : C(0);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kT; ++c) {
        if (c >= w) break;
        const C xc = __shfl_sync(0xffffffffu, y[c >> 2], (lane & ~3) | (c & 3));
#pragma unroll
        for (int t = 0; t < kT / 4; ++t) {
            const int cc = 4 * t + q;
            if (4 * t + 3 > c && cc > c && cc < w) y[t] -= xc * Bd[cc][c];
        }
    }
#pragma unroll
    for (int t = 0; t < kT / 4; ++t) {
        const int c = 4 * t + q;
        if (on && c < w) P[(r0 + r) + (int64_t)(c0 + c) * m] = y[t] * dv[c];
    }
}

// Trailing panel update after block column b: for panel columns j in
// [c0+w, k) and rows i >= j, P[i][j] -= sum_{c in block b} L[i][c] d_c L[j][c].
template <typename C>
__global__ void __launch_bounds__(kThreads) k_panel_update(DevSym d, const int32_t* __restrict__ items, int b,
                                                           C* __restrict__ L, double* __restrict__ D,
                                                           C* __restrict__ DS, const double* __restrict__ adiag,
                                                           DevStatus* status, Strides bs) {
    L += blockIdx.y * bs.L;
    D += blockIdx.y * bs.n;
    DS += blockIdx.y * bs.n;
    adiag += blockIdx.y * bs.n;
    __shared__ C Li[kT][kT + 1];
    __shared__ C Lj[kT][kT + 1];
    const int tid = threadIdx.x;
    const int s = items[3 * blockIdx.x], ti = items[3 * blockIdx.x + 1], tj = items[3 * blockIdx.x + 2];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    C* P = L + d.lptr[s];
    const int c0 = b * kT, w = min(kT, k - c0);
    const int cj = c0 + w + tj * kT;
    const int64_t ri = cj + (int64_t)ti * kT;
    const int nj = min(kT, k - cj);
    const int ni = (int)(m - ri < kT ? m - ri : kT);
    for (int e = tid; e < kT * kT; e += kThreads) {
        int i = e % kT, c = e / kT;
        Li[i][c] = (i < ni && c < w) ? P[(ri + i) + (int64_t)(c0 + c) * m] : C(0);
        Lj[i][c] = (i < nj && c < w) ? P[(cj + i) + (int64_t)(c0 + c) * m] * DS[f + c0 + c] : C(0);
    }
    __syncthreads();
    // thread owns row ii and columns j0 + 4 q: a warp's lanes run down one
    // column, so its read-modify-writes of the panel are coalesced
    const int ii = tid % kT, j0 = tid / kT;
    if (ii < ni) {
        C acc[kT / 4];
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) acc[q] = C(0);
#pragma unroll 4
        for (int c = 0; c < w; ++c) {  // the block column's w pivots (FP64 is a narrow pipe: no padding)
            const C ai = Li[ii][c];
#pragma unroll
            for (int q = 0; q < kT / 4; ++q) acc[q] += ai * Lj[j0 + 4 * q][c];
        }
        C old[kT / 4];  // loads first, then the stores (no load waits behind a store)
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) {
            const int jj = j0 + 4 * q;
            old[q] = (jj < nj && ri + ii >= cj + jj) ? P[(ri + ii) + (int64_t)(cj + jj) * m] : C(0);
        }
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) {
            const int jj = j0 + 4 * q;
            if (jj < nj && ri + ii >= cj + jj) P[(ri + ii) + (int64_t)(cj + jj) * m] = old[q] - acc[q];
        }
    }
    if (ti == 0 && tj == 0) {
        // this CTA wrote the last update of the next block column's pivot tile: factor it now
        __shared__ double A[kT][kT + 1];
        __shared__ double dv[kT];
        __syncthreads();
        factor_pivot_tile(A, dv, P, m, cj, nj, f, D, DS, adiag, status, (int)(blockIdx.y * bs.n));
    }
}

// Schur complement tile (ti, tj) of the trailing (m-k)^2 part, added into the parent's front.
template <typename C>
__global__ void __launch_bounds__(kThreads) k_schur_scatter(DevSym d, const int32_t* __restrict__ items,
                                                            C* __restrict__ L, C* __restrict__ F22,
                                                            const C* __restrict__ DS, Strides bs) {
    L += blockIdx.y * bs.L;
    F22 += blockIdx.y * bs.F22;
    DS += blockIdx.y * bs.n;
    __shared__ C Li[kT][kT + 1];
    __shared__ C Lj[kT][kT + 1];
    const int tid = threadIdx.x;
    const int s = items[3 * blockIdx.x], ti = items[3 * blockIdx.x + 1], tj = items[3 * blockIdx.x + 2];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const int64_t mb = m - k;
    const C* P = L + d.lptr[s];
    const int64_t ib = k + (int64_t)ti * kT, jb = k + (int64_t)tj * kT;
    const int ni = (int)(m - ib < kT ? m - ib : kT), nj = (int)(m - jb < kT ? m - jb : kT);
    // thread owns row ii and columns j0 + 4 q: a warp's lanes run down one
    // column, so its atomics into the parent hit consecutive rows
    const int ii = tid % kT, j0 = tid / kT;
    C acc[kT / 4];
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) acc[q] = C(0);
    for (int cb = 0; cb < k; cb += kT) {
        const int cw = min(kT, k - cb);
        __syncthreads();
        for (int e = tid; e < kT * kT; e += kThreads) {
            int i = e % kT, c = e / kT;
            Li[i][c] = (i < ni && c < cw) ? P[(ib + i) + (int64_t)(cb + c) * m] : C(0);
            Lj[i][c] = (i < nj && c < cw) ? P[(jb + i) + (int64_t)(cb + c) * m] * DS[f + cb + c] : C(0);
        }
        __syncthreads();
        if (ii < ni) {
#pragma unroll 4
            for (int c = 0; c < cw; ++c) {  // only the chunk's cw pivots (grouped leaves: often < 32)
                const C ai = Li[ii][c];
#pragma unroll
                for (int q = 0; q < kT / 4; ++q) acc[q] -= ai * Lj[j0 + 4 * q][c];
            }
        }
    }
    const int64_t fo = d.f22ptr[s];
    const int p = d.sparent[s];
    const int kp = d.sfirst[p + 1] - d.sfirst[p];
    const int64_t mp = d.srowptr[p + 1] - d.srowptr[p];
    C* Pp = L + d.lptr[p];
    C* Fp = F22 + (d.f22ptr[p] < 0 ? 0 : d.f22ptr[p]);
    const int32_t* rel = d.relmap + d.srowptr[s];
    if (ii >= ni) return;
    const int64_t il = ib + ii;
    const int qi = rel[il];
    C f22v[kT / 4];  // the update area's entries and the column maps first, then the atomics
    int qjv[kT / 4];
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
        const int64_t jl = jb + j0 + 4 * q;
        const bool on = j0 + 4 * q < nj && il >= jl;
        f22v[q] = (fo >= 0 && on) ? F22[fo + (il - k) + (jl - k) * mb] : C(0);
        qjv[q] = on ? rel[jl] : 0;
    }
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
        const int jj = j0 + 4 * q;
        const int64_t jl = jb + jj;
        if (jj >= nj || il < jl) continue;
        const C v = acc[q] + f22v[q];
        const int qj = qjv[q];
        if (qj < kp) atomicAdd(Pp + qi + (int64_t)qj * mp, v);
        else atomicAdd(Fp + (qi - kp) + (int64_t)(qj - kp) * (mp - kp), v);
    }
}

// ---------------------------------------------------------------------------
// Mixed-precision Schur update on the 5th-generation tensor cores.
//
// C = F22 - L21 D1 L21^T for a 128 x 128 output tile (rows ti, columns tj of
// the trailing (m-k) x (m-k) part) in split precision: every FP32 operand is
// a = a_hi + a_mid + a_lo with three TF32 pieces (33 significant bits), and
// a b = a_hi b_hi + a_hi b_mid + a_mid b_hi + a_hi b_lo + a_lo b_hi
// + a_mid b_mid, the dropped cross terms being below FP32 rounding, so the
// tile is as accurate as an FP32 product.  K (the supernode's pivots) streams
// through shared memory in chunks of 32, two stages: thread t holds row t of
// both operands; it loads the next chunk's FP64 values into registers while
// the tensor cores work on the current one, then writes them to the free
// stage as three TF32 pieces (16-byte stores into the K-major core-matrix
// layout of 8 rows x 16 bytes); one thread issues 4 k-steps x 6
// tcgen05.mma kind::tf32 (M = 128, N = 128, K = 8) accumulating in tensor
// memory, and tcgen05.commit
// signals the stage's mbarrier when those MMAs have read it.  The epilogue
// reads the accumulator with tcgen05.ld (warp w owns lanes 32w..32w+31 =
// tile rows) and adds C into the parent front with FP64 atomics, as the SIMT
// kernel does.  Every mbarrier wait is bounded; on timeout the kernel raises
// FLAG_TIMEOUT, waits (bounded) for its last commit, frees its tensor memory
// and leaves the tile unfinished.
constexpr int kTcStageFloats = 3 * kTcM * kTcK + 3 * kTcN * kTcK;  // A hi/mid/lo, B hi/mid/lo
constexpr size_t kTcSmem = 2 * kTcStageFloats * sizeof(float) + 64;
// polls of one dependency wait of the dependency-driven kernel (about 100 ns
// apart: some seconds, far beyond any task's legitimate wait)
constexpr uint32_t kDagWaitLimit = 1u << 25;

//
// kMode 1 is the same product as the rank-kOuter trailing update of a wide
// front: K = the kOuter columns [c1 - kOuter, c1) that end at block step
// `step` (c1 = (step + 1) * 32), output rows [c1, m) x panel columns [c1, k),
// subtracted in place from the panel (one CTA owns each tile: no atomics).
template <int kMode>
__global__ void __launch_bounds__(128) k_schur_tc(DevSym d, const int32_t* __restrict__ items, int step,
                                                  float* __restrict__ L, float* __restrict__ F22,
                                                  const float* __restrict__ DS, DevStatus* status, Strides bs,
                                                  uint32_t stage_wait_limit) {
    L += blockIdx.y * bs.L;
    F22 += blockIdx.y * bs.F22;
    DS += blockIdx.y * bs.n;
    extern __shared__ __align__(1024) float tcs[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(tcs + 2 * kTcStageFloats);  // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int s = items[3 * blockIdx.x], ti = items[3 * blockIdx.x + 1], tj = items[3 * blockIdx.x + 2];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    float* P = L + d.lptr[s];
    // K range [kb0, kb1); output rows from ib, columns from jb below jlim
    const int c1 = (step + 1) * kT;
    const int kb0 = kMode == 0 ? 0 : c1 - kOuter, kb1 = kMode == 0 ? k : c1;
    const int64_t ib = (kMode == 0 ? k : c1) + (int64_t)ti * kTcM, jb = (kMode == 0 ? k : c1) + (int64_t)tj * kTcN;
    const int64_t jlim = kMode == 0 ? m : k;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(tc_smem_u32(tmem_slot)),
                     "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc_smem_u32(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tc_smem_u32(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    const int nk = (kb1 - kb0 + kTcK - 1) / kTcK;
    // row tid of A (rows from ib) and of B (rows from jb, scaled by D) for one K chunk
    float ra[kTcK], rb[kTcK];
    auto fetch = [&](int kc) {
        const int cb = kb0 + kc * kTcK, cw = min(kTcK, kb1 - cb);
        const bool rowa = ib + tid < m, rowb = jb + tid < jlim;
        const float* pa = P + (ib + tid) + (int64_t)cb * m;
        const float* pb = P + (jb + tid) + (int64_t)cb * m;
#pragma unroll
        for (int c = 0; c < kTcK; ++c) {
            ra[c] = (c < cw && rowa) ? pa[(int64_t)c * m] : 0.f;
            rb[c] = (c < cw && rowb) ? pb[(int64_t)c * m] * DS[f + cb + c] : 0.f;
        }
    };
    if (nk > 0) fetch(0);
    bool ok = true;
    int last = -1;     // last chunk whose MMAs were committed
    int a_start = 0;   // first chunk accumulated into A since S last took it
    int nflush = 0;    // times A was added into S
    for (int kc = 0; kc < nk && ok; ++kc) {
        const int st = kc & 1;
        if (kc >= 2) ok = tc_wait(mbar + st, (uint32_t)((kc - 2) >> 1) & 1u, stage_wait_limit);
        if (__syncthreads_or(!ok)) { ok = false; break; }
        float* Ah = tcs + st * kTcStageFloats;
        float* Am = Ah + kTcM * kTcK;
        float* Al = Am + kTcM * kTcK;
        float* Bh = Al + kTcM * kTcK;
        float* Bm = Bh + kTcN * kTcK;
        float* Bl = Bm + kTcN * kTcK;
#pragma unroll
        for (int c4 = 0; c4 < kTcK / 4; ++c4) {
            const int o = tc_kmajor_off(tid, 4 * c4) >> 2;
            float4 h, mi, lo;
            tc_split3(ra[4 * c4 + 0], h.x, mi.x, lo.x);
            tc_split3(ra[4 * c4 + 1], h.y, mi.y, lo.y);
            tc_split3(ra[4 * c4 + 2], h.z, mi.z, lo.z);
            tc_split3(ra[4 * c4 + 3], h.w, mi.w, lo.w);
            *reinterpret_cast<float4*>(Ah + o) = h;
            *reinterpret_cast<float4*>(Am + o) = mi;
            *reinterpret_cast<float4*>(Al + o) = lo;
            tc_split3(rb[4 * c4 + 0], h.x, mi.x, lo.x);
            tc_split3(rb[4 * c4 + 1], h.y, mi.y, lo.y);
            tc_split3(rb[4 * c4 + 2], h.z, mi.z, lo.z);
            tc_split3(rb[4 * c4 + 3], h.w, mi.w, lo.w);
            *reinterpret_cast<float4*>(Bh + o) = h;
            *reinterpret_cast<float4*>(Bm + o) = mi;
            *reinterpret_cast<float4*>(Bl + o) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int kk = 0; kk < kTcK / 8; ++kk) {
                const uint32_t ko = kk * 256;
                const uint64_t ah = tc_desc(tc_smem_u32(Ah) + ko), am = tc_desc(tc_smem_u32(Am) + ko),
                               al = tc_desc(tc_smem_u32(Al) + ko);
                const uint64_t bh = tc_desc(tc_smem_u32(Bh) + ko), bm = tc_desc(tc_smem_u32(Bm) + ko),
                               bl = tc_desc(tc_smem_u32(Bl) + ko);
                // the five small cross products into B, hi*hi into A
                tc_mma(tmem + kAccB, am, bm, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                tc_mma(tmem + kAccB, al, bh, idesc, 1u);
                tc_mma(tmem + kAccB, ah, bl, idesc, 1u);
                tc_mma(tmem + kAccB, am, bh, idesc, 1u);
                tc_mma(tmem + kAccB, ah, bm, idesc, 1u);
                tc_mma(tmem, ah, bh, idesc, (kc > a_start || kk > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(tc_smem_u32(mbar + st)));
        }
        last = kc;
        if ((kc + 1 - a_start) % kTcFlush == 0 && kc + 1 < nk) {
            // S += A once this chunk's MMAs are done, then A restarts with the next chunk
            ok = tc_wait(mbar + st, (uint32_t)(kc >> 1) & 1u, stage_wait_limit);
            if (__syncthreads_or(!ok)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t row = (uint32_t)(warp * 32) << 16;
            for (int q = 0; q < kTcN / 32; ++q) {
                uint32_t a[32], sv[32];
                tc_ld32(tmem + row + q * 32, a);
                if (nflush > 0) tc_ld32(tmem + row + kAccS + q * 32, sv);
                else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) sv[j] = 0u;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) sv[j] = __float_as_uint(__uint_as_float(sv[j]) + __uint_as_float(a[j]));
                tc_st32(tmem + row + kAccS + q * 32, sv);
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            a_start = kc + 1;
            ++nflush;
        }
        if (kc + 1 < nk) fetch(kc + 1);  // in flight while the MMAs above run
    }
    // the last commit covers every MMA issued before it
    bool fin = last >= 0 ? tc_wait(mbar + (last & 1), (uint32_t)(last >> 1) & 1u, stage_wait_limit) : true;
    fin = !__syncthreads_or(!fin) && ok;
    if (!fin && last >= 0) tc_wait(mbar + (last & 1), (uint32_t)(last >> 1) & 1u);  // drain before release
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!fin) {
        if (tid == 0) atomicOr(&status->flags, FLAG_TIMEOUT);
    } else if (kMode == 1) {
        const int64_t il = ib + warp * 32 + lane;
        for (int q = 0; q < kTcN / 32; ++q) {
            uint32_t r[32];
            tc_acc32(tmem + ((uint32_t)(warp * 32) << 16) + q * 32, nflush > 0, r);
            if (il < m) {
                // all 32 loads first: a load after a store to the same array would wait for it
                float old[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t jl = jb + q * 32 + j;
                    old[j] = (jl < k && jl <= il) ? P[il + jl * m] : 0.f;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t jl = jb + q * 32 + j;
                    if (jl < k && jl <= il) P[il + jl * m] = old[j] - __uint_as_float(r[j]);
                }
            }
        }
    } else {
        const int64_t fo = d.f22ptr[s];
        const int64_t mb = m - k;
        const int p = d.sparent[s];
        const int kp = d.sfirst[p + 1] - d.sfirst[p];
        const int64_t mp = d.srowptr[p + 1] - d.srowptr[p];
        float* Pp = L + d.lptr[p];
        float* Fp = F22 + (d.f22ptr[p] < 0 ? 0 : d.f22ptr[p]);
        const int32_t* rel = d.relmap + d.srowptr[s];
        const int64_t il = ib + warp * 32 + lane;
        const int qi = il < m ? rel[il] : 0;
        for (int q = 0; q < kTcN / 32; ++q) {
            uint32_t r[32];
            tc_acc32(tmem + ((uint32_t)(warp * 32) << 16) + q * 32, nflush > 0, r);
            if (il < m) {
                float f22v[32];  // the update area's entries and the column maps first, then the atomics
                int qjv[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t jl = jb + q * 32 + j;
                    const bool on = jl < m && jl <= il;
                    f22v[j] = (fo >= 0 && on) ? F22[fo + (il - k) + (jl - k) * mb] : 0.f;
                    qjv[j] = on ? rel[jl] : 0;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t jl = jb + q * 32 + j;
                    if (jl >= m || jl > il) continue;
                    const float v = f22v[j] - __uint_as_float(r[j]);
                    const int qj = qjv[j];
                    if (qj < kp) atomicAdd(Pp + qi + (int64_t)qj * mp, v);
                    else atomicAdd(Fp + (qi - kp) + (int64_t)(qj - kp) * (mp - kp), v);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcCols));
}

// ---------------------------------------------------------------------------
// Dependency-driven persistent factorization (launch kind 13).
//
// One launch runs every task of a prefix of the tree's levels: diagonal-pivot
// fronts, whole small fronts (front_panel_body), pivot tiles, 128-row chunks
// of the panel solve, 32 x 32 tiles of the trailing panel update (the first of
// which factors the next pivot tile) and 32 x 32 Schur tiles added into the
// parent.  The host lists the tasks in a topological order -- by level, then
// by phase within each front, a front's Schur tiles right after its last
// phase -- and the CTAs take them in that order from a global counter.  A task
// waits until one counter reaches its value: the tasks of its front's earlier
// phases, or the Schur tiles its front's children add in; it then runs and
// counts itself done.  A task only waits for tasks earlier in the order, which
// CTAs that are running already hold, so every wait ends; each wait is still
// bounded, and when one gives up it raises FLAG_TIMEOUT and every CTA skips
// its remaining tasks.  Data another CTA wrote during the launch is read
// through L2 (ld.global.cg).  This replaces the chain of per-step launches,
// whose gaps and partly idle waves bound the factorization of the wide fronts
// near the root.
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool dag_aborted(const DevStatus* status) {
    return (*reinterpret_cast<const volatile int*>(&status->flags) & FLAG_TIMEOUT) != 0;
}

// Thread 0: wait until *c >= need; false if the wait gave up (limit) or the
// launch was abandoned.
__device__ bool dag_wait(const int* c, int need, const DevStatus* status, uint32_t limit) {
    if (limit == 0) return false;  // spi_options.wait_limit < 0: every wait gives up at once
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire_gpu(c) >= need) return true;
        if (it >= limit) return false;
        if ((it & 31) == 31 && dag_aborted(status)) return false;
        __nanosleep(100);
    }
}

// 128 rows of the panel solve below pivot tile b: L21 = X L11^-T D^-1.
template <typename C>
__device__ void dag_trsm(const DevSym& d, int s, int b, int chunk, C* Lb, const double* Db, FrontPanelSmem<C>& sm) {
    const int tid = threadIdx.x;
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    C* P = Lb + d.lptr[s];
    const int c0 = b * kT, w = min(kT, k - c0);
    for (int e = tid; e < kT * kT; e += kThreads) {
        const int i = e % kT, j = e / kT;
        sm.trsm.Bd[i][j] = (i < w && j < i) ? __ldcg(P + (c0 + i) + (int64_t)(c0 + j) * m) : C(0);
    }
    if (tid < kT) sm.trsm.rd[tid] = tid < w ? (C)(1.0 / __ldcg(Db + f + c0 + tid)) : C(0);
    __syncthreads();
    const int64_t r = c0 + w + (int64_t)chunk * kThreads + tid;
    if (r < m) {
        C* xr = sm.trsm.X[tid];
        for (int c = 0; c < w; ++c) xr[c] = __ldcg(P + r + (int64_t)(c0 + c) * m);
        for (int c = 1; c < w; ++c) {
            C y = xr[c];
            for (int cp = 0; cp < c; ++cp) y -= xr[cp] * sm.trsm.Bd[c][cp];
            xr[c] = y;
        }
        for (int c = 0; c < w; ++c) P[r + (int64_t)(c0 + c) * m] = xr[c] * sm.trsm.rd[c];
    }
}

// Trailing-update tile (ti, tj) after block column b (as k_panel_update); the
// tile (0, 0) then factors the next pivot tile.
template <typename C>
__device__ void dag_update(const DevSym& d, int s, int b, int ti, int tj, C* Lb, double* Db, C* DSb,
                           const double* ab, DevStatus* status, int base, FrontPanelSmem<C>& sm) {
    const int tid = threadIdx.x;
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    C* P = Lb + d.lptr[s];
    const int c0 = b * kT, w = min(kT, k - c0);
    const int cj = c0 + w + tj * kT;
    const int64_t ri = cj + (int64_t)ti * kT;
    const int nj = min(kT, k - cj);
    const int ni = (int)(m - ri < kT ? m - ri : kT);
    for (int e = tid; e < kT * kT; e += kThreads) {
        const int i = e % kT, c = e / kT;
        sm.upd.Li[i][c] = (i < ni && c < w) ? __ldcg(P + (ri + i) + (int64_t)(c0 + c) * m) : C(0);
        sm.upd.Lj[i][c] =
            (i < nj && c < w) ? __ldcg(P + (cj + i) + (int64_t)(c0 + c) * m) * __ldcg(DSb + f + c0 + c) : C(0);
    }
    __syncthreads();
    const int ii = tid % kT, j0 = tid / kT;
    if (ii < ni) {
        C acc[kT / 4];
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) acc[q] = C(0);
#pragma unroll 4
        for (int c = 0; c < w; ++c) {
            const C ai = sm.upd.Li[ii][c];
#pragma unroll
            for (int q = 0; q < kT / 4; ++q) acc[q] += ai * sm.upd.Lj[j0 + 4 * q][c];
        }
        C old[kT / 4];
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) {
            const int jj = j0 + 4 * q;
            old[q] = (jj < nj && ri + ii >= cj + jj) ? __ldcg(P + (ri + ii) + (int64_t)(cj + jj) * m) : C(0);
        }
#pragma unroll
        for (int q = 0; q < kT / 4; ++q) {
            const int jj = j0 + 4 * q;
            if (jj < nj && ri + ii >= cj + jj) P[(ri + ii) + (int64_t)(cj + jj) * m] = old[q] - acc[q];
        }
    }
    if (ti == 0 && tj == 0) {
        __syncthreads();  // the pivot tile's shared memory overlaps the update tiles
        factor_pivot_tile<C, true>(sm.piv.A, sm.piv.dv, P, m, cj, nj, f, Db, DSb, ab, status, base);
    }
}

// Schur tile (ti, tj) of the trailing block, added into the parent front (as k_schur_scatter).
template <typename C>
__device__ void dag_schur(const DevSym& d, int s, int ti, int tj, C* Lb, C* Fb, const C* DSb, FrontPanelSmem<C>& sm) {
    const int tid = threadIdx.x;
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
    const int64_t mb = m - k;
    const C* P = Lb + d.lptr[s];
    const int64_t ib = k + (int64_t)ti * kT, jb = k + (int64_t)tj * kT;
    const int ni = (int)(m - ib < kT ? m - ib : kT), nj = (int)(m - jb < kT ? m - jb : kT);
    const int ii = tid % kT, j0 = tid / kT;
    C acc[kT / 4];
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) acc[q] = C(0);
    for (int cb = 0; cb < k; cb += kT) {
        const int cw = min(kT, k - cb);
        __syncthreads();
        for (int e = tid; e < kT * kT; e += kThreads) {
            const int i = e % kT, c = e / kT;
            sm.upd.Li[i][c] = (i < ni && c < cw) ? __ldcg(P + (ib + i) + (int64_t)(cb + c) * m) : C(0);
            sm.upd.Lj[i][c] =
                (i < nj && c < cw) ? __ldcg(P + (jb + i) + (int64_t)(cb + c) * m) * __ldcg(DSb + f + cb + c) : C(0);
        }
        __syncthreads();
        if (ii < ni) {
#pragma unroll 4
            for (int c = 0; c < cw; ++c) {
                const C ai = sm.upd.Li[ii][c];
#pragma unroll
                for (int q = 0; q < kT / 4; ++q) acc[q] -= ai * sm.upd.Lj[j0 + 4 * q][c];
            }
        }
    }
    const int64_t fo = d.f22ptr[s];
    const int p = d.sparent[s];
    const int kp = d.sfirst[p + 1] - d.sfirst[p];
    const int64_t mp = d.srowptr[p + 1] - d.srowptr[p];
    C* Pp = Lb + d.lptr[p];
    C* Fp = Fb + (d.f22ptr[p] < 0 ? 0 : d.f22ptr[p]);
    const int32_t* rel = d.relmap + d.srowptr[s];
    if (ii >= ni) return;
    const int64_t il = ib + ii;
    const int qi = rel[il];
#pragma unroll
    for (int q = 0; q < kT / 4; ++q) {
        const int jj = j0 + 4 * q;
        const int64_t jl = jb + jj;
        if (jj >= nj || il < jl) continue;
        const C v = acc[q] + (fo >= 0 ? __ldcg(Fb + fo + (il - k) + (jl - k) * mb) : C(0));
        const int qj = rel[jl];
        if (qj < kp) atomicAdd(Pp + qi + (int64_t)qj * mp, v);
        else atomicAdd(Fp + (qi - kp) + (int64_t)(qj - kp) * (mp - kp), v);
    }
}

template <typename C>
__global__ void __launch_bounds__(kThreads) k_factor_dag(DevSym d, const DagTask* __restrict__ tasks, int ntasks,
                                                         int nb, int* cnt, int cstride, C* L, C* F22, double* D,
                                                         C* DS, const double* __restrict__ adiag, DevStatus* status,
                                                         Strides bs, uint32_t wait_limit) {
    __shared__ FrontPanelSmem<C> sm;
    __shared__ int64_t s_t;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    int* next = cnt + (int64_t)nb * cstride;
    const int64_t total = (int64_t)ntasks * nb;
    for (;;) {
        __syncthreads();  // the previous task is finished with s_t, s_ok and the shared memory
        if (tid == 0) {
            const int64_t t = (int64_t)(unsigned)atomicAdd(next, 1);
            int ok = 0;
            if (t < total) {
                const DagTask tk = tasks[t / nb];
                ok = !dag_aborted(status);
                if (ok && tk.wait_val > 0) {
                    ok = dag_wait(cnt + (t % nb) * cstride + tk.wait_idx, tk.wait_val, status, wait_limit);
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
        C* Lb = L + band * bs.L;
        C* Fb = F22 + band * bs.F22;
        double* Db = D + band * bs.n;
        C* DSb = DS + band * bs.n;
        const double* ab = adiag + band * bs.n;
        const int base = (int)(band * bs.n);
        switch (tk.type) {
            case kDagDiagFront: diag_front_body<C, true>(d, tk.s, Lb, Db, DSb, ab, status, base); break;
            case kDagFused: front_panel_body<C, true>(d, tk.s, Lb, Db, DSb, ab, status, base, sm); break;
            case kDagPivot: {
                const int f = d.sfirst[tk.s], k = d.sfirst[tk.s + 1] - f;
                const int64_t m = d.srowptr[tk.s + 1] - d.srowptr[tk.s];
                factor_pivot_tile<C, true>(sm.piv.A, sm.piv.dv, Lb + d.lptr[tk.s], m, 0, min(kT, k), f, Db, DSb, ab,
                                           status, base);
                break;
            }
            case kDagTrsm: dag_trsm(d, tk.s, tk.a, tk.b, Lb, Db, sm); break;
            case kDagUpdate: dag_update(d, tk.s, tk.a, tk.b >> 16, tk.b & 0xFFFF, Lb, Db, DSb, ab, status, base, sm); break;
            default: dag_schur(d, tk.s, tk.a, tk.b, Lb, Fb, DSb, sm); break;
        }
        __threadfence();  // every thread's stores of the task are visible device-wide ...
        __syncthreads();
        if (tid == 0) atomicAdd(cnt + band * cstride + tk.done_idx, 1);  // ... before it counts as done
    }
}

// ---------------------------------------------------------------------------
// Symmetric indefinite fronts (spi_options.pivoting; paper Sec. 5: the SPI
// matrices are symmetric indefinite and need two-by-two pivots).  One CTA per
// front, FP64, all of a level's fronts in one launch.  The k fully-summed
// columns are factored unblocked and right-looking with restricted
// Bunch-Kaufman pivoting (alpha = (1 + sqrt 17) / 8): for column c, lam is
// its largest off-diagonal magnitude over all rows of the front, and only a
// fully-summed row r (c < r < k) may become a pivot:
//   |a_cc| >= alpha lam                          -> 1x1 pivot c;
//   else, with r the largest fully-summed entry of column c (lam_fs) and sig
//   the largest off-diagonal magnitude of column r:
//   |a_cc| sig >= alpha lam^2                    -> 1x1 pivot c;
//   |a_rr| >= alpha sig                          -> swap c, r; 1x1 pivot;
//   lam_fs >= alpha lam (r nearly carries lam)   -> swap c + 1, r; 2x2 pivot;
//   otherwise (or no fully-summed candidate)     -> the front's pivots are
//   delayed: it is recorded and left unfinished, and the host merges it into
//   its parent's front (where its columns are fully summed) and refactors.
// Swaps are symmetric and stay inside the fully-summed block, so the front's
// rows below and its place in the parent do not change; lperm records them.
// Then the Schur complement F22 - L21 D L21^T (D block diagonal) is added
// into the parent front as in the SPD form.
constexpr double kBkAlpha = 0.64038820320220756872;  // (1 + sqrt(17)) / 8
constexpr int kBkThreads = 256;

// Largest |v| over the CTA, with the smallest index attaining it (idx < 0: none).
__device__ void bk_block_max(double v, int idx, double* sv, int* si, double* out_v, int* out_i) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        if (v2 > v || (v2 == v && i2 >= 0 && (idx < 0 || i2 < idx))) { v = v2; idx = i2; }
    }
    if (lane == 0) { sv[warp] = v; si[warp] = idx; }
    __syncthreads();
    if (tid == 0) {
        double bv = -1.0;
        int bi = -1;
        for (int w = 0; w < kBkThreads / 32; ++w)
            if (sv[w] > bv || (sv[w] == bv && si[w] >= 0 && (bi < 0 || si[w] < bi))) { bv = sv[w]; bi = si[w]; }
        *out_v = bv;
        *out_i = bi;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBkThreads) k_front_bk(DevSym d, const int32_t* __restrict__ items, double* L,
                                                         double* F22, BkArgs a, DevStatus* status) {
    __shared__ double sv[kBkThreads / 32];
    __shared__ int si[kBkThreads / 32];
    __shared__ double s_lam, s_lamfs, s_sig;
    __shared__ int s_r, s_dummy, s_size, s_swap_a, s_swap_b;
    const int tid = threadIdx.x;
    const int s = items[blockIdx.x];
    const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
    const int m = (int)(d.srowptr[s + 1] - d.srowptr[s]);
    double* P = L + d.lptr[s];
    auto at = [&](int i, int j) -> double& { return P[(int64_t)i + (int64_t)j * m]; };  // i >= j
    for (int i = tid; i < k; i += kBkThreads) a.lperm[f + i] = i;
    __syncthreads();
    for (int c = 0; c < k;) {
        // lam over every row below c; lam_fs and r over the fully-summed rows
        double v = 0.0, vf = 0.0;
        int iv = -1, ivf = -1;
        for (int i = c + 1 + tid; i < m; i += kBkThreads) {
            const double x = fabs(at(i, c));
            if (x > v) { v = x; iv = i; }
            if (i < k && x > vf) { vf = x; ivf = i; }
        }
        bk_block_max(v, iv, sv, si, &s_lam, &s_dummy);
        bk_block_max(vf, ivf, sv, si, &s_lamfs, &s_r);
        const double lam = s_lam, lamfs = s_lamfs, acc_ = fabs(at(c, c));
        const int r = s_r;
        // sig: the largest off-diagonal entry of column r, when it is needed
        const bool need_sig = !(acc_ >= kBkAlpha * lam) && lamfs > 0.0 && r > c;
        if (need_sig) {
            double w = 0.0;
            for (int i = c + tid; i < m; i += kBkThreads) {
                if (i == r) continue;
                const double x = fabs(i < r ? at(r, i) : at(i, r));
                if (x > w) w = x;
            }
            bk_block_max(w, 0, sv, si, &s_sig, &s_dummy);
        }
        if (tid == 0) {
            int size = 1, sa = -1, sb = -1;
            if (lam == 0.0) {
                if (acc_ == 0.0) size = 0;  // a zero column in the front: delay
            } else if (acc_ >= kBkAlpha * lam) {
            } else if (!need_sig) {
                size = 0;  // no fully-summed candidate
            } else {
                const double sig = s_sig;
                if (acc_ * sig >= kBkAlpha * lam * lam) {
                } else if (fabs(at(r, r)) >= kBkAlpha * sig) {
                    sa = c; sb = r;
                } else if (lamfs >= kBkAlpha * lam && c + 1 < k) {
                    size = 2;
                    if (r != c + 1) { sa = c + 1; sb = r; }
                } else {
                    size = 0;
                }
            }
            s_size = size; s_swap_a = sa; s_swap_b = sb;
        }
        __syncthreads();
        const int size = s_size;
        if (size == 0) {
            if (tid == 0) {
                const int q = atomicAdd(a.delay, 1);
                if (q < a.max_delay) a.delay[1 + q] = s;
                atomicOr(&status->flags, FLAG_DELAY);
            }
            return;  // left unfinished: the host merges this front into its parent and refactors
        }
        const int sa = s_swap_a, sb = s_swap_b;
        if (sa >= 0) {  // symmetric swap of the fully-summed indices sa < sb (lower storage)
            for (int j = tid; j < sa; j += kBkThreads) { const double t = at(sa, j); at(sa, j) = at(sb, j); at(sb, j) = t; }
            for (int j = sa + 1 + tid; j < sb; j += kBkThreads) { const double t = at(j, sa); at(j, sa) = at(sb, j); at(sb, j) = t; }
            for (int i = sb + 1 + tid; i < m; i += kBkThreads) { const double t = at(i, sa); at(i, sa) = at(i, sb); at(i, sb) = t; }
            if (tid == 0) {
                const double t = at(sa, sa); at(sa, sa) = at(sb, sb); at(sb, sb) = t;
                const int32_t q = a.lperm[f + sa]; a.lperm[f + sa] = a.lperm[f + sb]; a.lperm[f + sb] = q;
            }
            __syncthreads();
        }
        const int c2 = c + size;
        if (size == 1) {
            const double dc = at(c, c);
            // rank-1 update of the remaining fully-summed columns, all rows below them
            for (int j = c + 1; j < k; ++j) {
                const double g = at(j, c) / dc;
                for (int i = j + tid; i < m; i += kBkThreads) at(i, j) -= at(i, c) * g;
            }
            __syncthreads();
            for (int i = c + 1 + tid; i < m; i += kBkThreads) at(i, c) /= dc;
            if (tid == 0) { a.Dd[f + c] = dc; a.Doff[f + c] = 0.0; a.pair[f + c] = -1; }
        } else {
            const double p11 = at(c, c), p21 = at(c + 1, c), p22 = at(c + 1, c + 1);
            const double det = p11 * p22 - p21 * p21;
            for (int j = c2; j < k; ++j) {
                const double uj = at(j, c), vj = at(j, c + 1);
                const double g0 = (p22 * uj - p21 * vj) / det, g1 = (p11 * vj - p21 * uj) / det;  // E^-1 [uj vj]
                for (int i = j + tid; i < m; i += kBkThreads) at(i, j) -= at(i, c) * g0 + at(i, c + 1) * g1;
            }
            __syncthreads();
            for (int i = c2 + tid; i < m; i += kBkThreads) {
                const double u = at(i, c), w = at(i, c + 1);
                at(i, c) = (p22 * u - p21 * w) / det;
                at(i, c + 1) = (p11 * w - p21 * u) / det;
            }
            if (tid == 0) {
                at(c + 1, c) = 0.0;  // L is unit lower: the block's coupling lives in D
                a.Dd[f + c] = p11; a.Dd[f + c + 1] = p22;
                a.Doff[f + c] = p21; a.Doff[f + c + 1] = 0.0;
                a.pair[f + c] = f + c + 1; a.pair[f + c + 1] = f + c;
                atomicAdd(a.count2x2, 1);
            }
        }
        __syncthreads();
        c = c2;
    }
    // Schur complement of the rows below, C = F22 - L21 D L21^T, added into the parent front
    const int p = d.sparent[s];
    if (p < 0 || m <= k) return;
    const int kp = d.sfirst[p + 1] - d.sfirst[p];
    const int64_t mp = d.srowptr[p + 1] - d.srowptr[p];
    double* Pp = L + d.lptr[p];
    double* Fp = F22 + (d.f22ptr[p] < 0 ? 0 : d.f22ptr[p]);
    const int64_t fo = d.f22ptr[s];
    const int32_t* rel = d.relmap + d.srowptr[s];
    const int mb = m - k;
    const double* Dd = a.Dd + f;
    const double* Doff = a.Doff + f;
    const int64_t npair = (int64_t)mb * (mb + 1) / 2;
    for (int64_t e = tid; e < npair; e += kBkThreads) {
        // e -> (i, j), i >= j, in the lower triangle of the (m - k)^2 block
        int j = (int)((2.0 * mb + 1.0 - sqrt((2.0 * mb + 1.0) * (2.0 * mb + 1.0) - 8.0 * (double)e)) / 2.0);
        while (j > 0 && (int64_t)j * (2 * mb - j + 1) / 2 > e) --j;
        while ((int64_t)(j + 1) * (2 * mb - j) / 2 <= e) ++j;
        const int i = j + (int)(e - (int64_t)j * (2 * mb - j + 1) / 2);
        const int il = k + i, jl = k + j;
        double acc = fo >= 0 ? F22[fo + i + (int64_t)j * mb] : 0.0;
        for (int cc = 0; cc < k; ++cc) {
            // (L D)[jl][cc] with D block diagonal
            double w = at(jl, cc) * Dd[cc];
            if (a.pair[f + cc] == f + cc + 1) w += at(jl, cc + 1) * Doff[cc];
            else if (cc > 0 && a.pair[f + cc] == f + cc - 1) w += at(jl, cc - 1) * Doff[cc - 1];
            acc -= at(il, cc) * w;
        }
        const int qi = rel[il], qj = rel[jl];
        if (qj < kp) atomicAdd(Pp + qi + (int64_t)qj * mp, acc);
        else atomicAdd(Fp + (qi - kp) + (int64_t)(qj - kp) * (mp - kp), acc);
    }
}

__global__ void k_to_f64(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

}  // namespace

// CTAs of the persistent per-level panel kernel: every SM slot it fits in
int g_panel_grid[2] = {0, 0};  // [0] FP64, [1] mixed
int g_dag_grid[2] = {0, 0};    // the dependency-driven kernel, likewise

cudaError_t factor_kernel_setup() {
    cudaError_t e = cudaFuncSetAttribute(k_schur_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_schur_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, b64 = 0, b32 = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_front_panel<double>, kThreads, 0)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_front_panel<float>, kThreads, 0)) != cudaSuccess)
        return e;
    g_panel_grid[0] = std::max(1, sms * b64);
    g_panel_grid[1] = std::max(1, sms * b32);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_factor_dag<double>, kThreads, 0)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_factor_dag<float>, kThreads, 0)) != cudaSuccess)
        return e;
    g_dag_grid[0] = std::max(1, sms * b64);
    g_dag_grid[1] = std::max(1, sms * b32);
    return cudaSuccess;
}

void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t st) {
    if (n == 0) return;
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_to_f64<<<grid, 256, 0, st>>>(a, b, n);
}

void launch_assemble(const DevSym& d, const int64_t* amap, const double* vals, int64_t nnz, void* L, bool mixed,
                     const int32_t* diag_src, double* adiag, int nb, const Strides& bs, cudaStream_t st) {
    int64_t work = std::max<int64_t>(nnz, d.n);
    if (work == 0 || nb == 0) return;
    int grid = (int)std::min<int64_t>((work + 255) / 256, std::max(1, 152 * 16 / nb));
    if (mixed)
        k_assemble<float><<<dim3(grid, nb), 256, 0, st>>>(amap, vals, nnz, (float*)L, diag_src, d.n, adiag, bs);
    else
        k_assemble<double><<<dim3(grid, nb), 256, 0, st>>>(amap, vals, nnz, (double*)L, diag_src, d.n, adiag, bs);
}

// C is both the arithmetic and the storage type of the panels and update
// areas: double in the FP64 form, float in the mixed form (whose pivot tiles
// are still factored in FP64 and whose pivots D stay FP64; DS is D in C).
template <typename C>
void launch_step_t(const DevSym& d, const Launch& l, const int32_t* items, C* L, C* F22, double* D, C* DS,
                   const double* adiag, DevStatus* status, int nb, const Strides& bs, int wait_limit,
                   cudaStream_t st) {
    const dim3 g(l.count, nb);
    switch (l.kind) {
        case 0: k_diag_tile<C><<<g, kThreads, 0, st>>>(d, items + l.off, l.step, L, D, DS, adiag, status, bs); break;
        case 1: k_panel_trsm<C><<<g, kThreads, 0, st>>>(d, items + 2 * l.off, l.step, L, D, bs); break;
        case 3:
            k_panel_update<C><<<g, kThreads, 0, st>>>(d, items + 3 * l.off, l.step, L, D, DS, adiag, status, bs);
            break;
        case 7:
        case 9:
            if constexpr (std::is_same<C, float>::value) {  // tensor-core items exist only in the mixed form
                const uint32_t lim = wait_limit > 0 ? (uint32_t)wait_limit : wait_limit < 0 ? 0u : kTcWaitLimit;
                if (l.kind == 7)
                    k_schur_tc<0><<<g, 128, kTcSmem, st>>>(d, items + 3 * l.off, 0, L, F22, DS, status, bs, lim);
                else
                    k_schur_tc<1><<<g, 128, kTcSmem, st>>>(d, items + 3 * l.off, l.step, L, F22, DS, status, bs, lim);
            }
            break;
        case 8: k_diag_front<C><<<g, kThreads, 0, st>>>(d, items + l.off, L, D, DS, adiag, status, bs); break;
        case 12: {
            const int64_t total = (int64_t)l.count * nb;
            const int grid = (int)std::min<int64_t>(total, g_panel_grid[std::is_same<C, float>::value ? 1 : 0]);
            k_front_panel<C><<<grid, kThreads, 0, st>>>(d, items + l.off, l.count, nb, L, D, DS, adiag, status, bs);
            break;
        }
        default: k_schur_scatter<C><<<g, kThreads, 0, st>>>(d, items + 3 * l.off, L, F22, DS, bs); break;
    }
}

void launch_front_bk(const DevSym& d, const int32_t* items, int count, double* L, double* F22, const BkArgs& a,
                     DevStatus* status, cudaStream_t st) {
    if (count == 0) return;
    k_front_bk<<<count, kBkThreads, 0, st>>>(d, items, L, F22, a, status);
}

void launch_factor_dag(const DevSym& d, const DagTask* tasks, int ntasks, int* counters, int cstride, void* L,
                       void* F22, double* D, void* DS, const double* adiag, DevStatus* status, bool mixed, int nb,
                       const Strides& bs, int wait_limit, cudaStream_t st) {
    if (ntasks == 0 || nb == 0) return;
    const uint32_t lim = wait_limit > 0 ? (uint32_t)wait_limit : wait_limit < 0 ? 0u : kDagWaitLimit;
    const int64_t total = (int64_t)ntasks * nb;
    if (mixed) {
        const int grid = (int)std::min<int64_t>(total, g_dag_grid[1]);
        k_factor_dag<float><<<grid, kThreads, 0, st>>>(d, tasks, ntasks, nb, counters, cstride, (float*)L, (float*)F22,
                                                       D, (float*)DS, adiag, status, bs, lim);
    } else {
        const int grid = (int)std::min<int64_t>(total, g_dag_grid[0]);
        k_factor_dag<double><<<grid, kThreads, 0, st>>>(d, tasks, ntasks, nb, counters, cstride, (double*)L,
                                                        (double*)F22, D, (double*)DS, adiag, status, bs, lim);
    }
}

void launch_factor_step(const DevSym& d, const Launch& l, const int32_t* items, void* L, void* F22, double* D,
                        void* DS, const double* adiag, DevStatus* status, bool mixed, int nb, const Strides& bs,
                        int wait_limit, cudaStream_t st) {
    if (l.kind < 0 || l.count == 0 || nb == 0) return;
    if (mixed)
        launch_step_t<float>(d, l, items, (float*)L, (float*)F22, D, (float*)DS, adiag, status, nb, bs, wait_limit,
                             st);
    else
        launch_step_t<double>(d, l, items, (double*)L, (double*)F22, D, (double*)DS, adiag, status, nb, bs,
                              wait_limit, st);
}

}  // namespace spi
