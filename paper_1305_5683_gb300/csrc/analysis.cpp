// analysis.cpp -- host-side analysis phase (paper Sec. 3.2.1).
//
// Ordering: nested dissection (Sec. 3.2.1 reorders with nested dissection to
// reduce fill).  Vertices that are a local minimum of the degree and form an
// independent set are eliminated first (for SPI matrices these are the
// per-pointing background columns: their neighbourhoods are almost cliques,
// so eliminating them first creates almost no fill); the rest is bisected
// recursively with breadth-first level structures of the graph those
// eliminations leave behind, traversed as a quotient graph so that the
// eliminated vertices' cliques are never formed.  Separators are numbered
// last; leaves keep the caller's relative order.
//
// Symbolic factorization: elimination tree (Liu's algorithm with path
// compression), postorder (Sec. 3.2.2: subtrees numbered consecutively),
// exact column counts from row subtrees, fundamental supernodes, relaxed
// amalgamation, front row lists, parent-relative index maps (the extend-add
// maps of the multifrontal method), levels of the supernodal tree.
#include "analysis.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

namespace spi {

namespace {
constexpr int kErrArg = 1, kErrPattern = 2, kErrOom = 4;

void build_graph(int32_t n, const int64_t* cp, const int32_t* ri, std::vector<int64_t>& xadj,
                 std::vector<int32_t>& adj) {
    xadj.assign((size_t)n + 1, 0);
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
            int32_t i = ri[p];
            if (i != j) { xadj[i + 1]++; xadj[j + 1]++; }
        }
    for (int32_t v = 0; v < n; ++v) xadj[v + 1] += xadj[v];
    adj.resize((size_t)xadj[n]);
    std::vector<int64_t> fill(xadj.begin(), xadj.end() - 1);
    for (int32_t j = 0; j < n; ++j)
        for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
            int32_t i = ri[p];
            if (i != j) { adj[fill[i]++] = j; adj[fill[j]++] = i; }
        }
}

// ---------------------------------------------------------------- nested dissection
struct ND {
    int32_t n;
    const std::vector<int64_t>& xadj;
    const std::vector<int32_t>& adj;
    int leaf;
    std::vector<char> is_elem;
    // interval of each non-element vertex: smallest and largest rank (position
    // in index order) of the elements adjacent to it; INT32_MAX / -1 if none
    std::vector<int32_t> elo, ehi;
    std::vector<int32_t> stamp, visit, estamp, lev, done;
    int32_t cur_set = 0, cur_bfs = 0, cur_done = 0;
    std::vector<int32_t> out;

    ND(int32_t n_, const std::vector<int64_t>& x, const std::vector<int32_t>& a, int leaf_)
        : n(n_), xadj(x), adj(a), leaf(leaf_), is_elem(n_, 0), elo(n_, INT32_MAX), ehi(n_, -1), stamp(n_, 0),
          visit(n_, 0), estamp(n_, 0), lev(n_, -1), done(n_, 0) {}

    int64_t deg(int32_t v) const { return xadj[v + 1] - xadj[v]; }

    // Breadth-first search in the quotient graph restricted to set `sid`.
    // q receives the vertices in visiting order, ls the level starts.
    template <class F>
    void for_each_nbr(int32_t v, int32_t sid, F&& f) {
        for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p) {
            int32_t w = adj[p];
            if (is_elem[w]) {
                if (estamp[w] == cur_bfs) continue;
                estamp[w] = cur_bfs;
                for (int64_t r = xadj[w]; r < xadj[w + 1]; ++r) {
                    int32_t u = adj[r];
                    if (stamp[u] == sid && !is_elem[u]) f(u);
                }
            } else if (stamp[w] == sid) {
                f(w);
            }
        }
    }

    void bfs(int32_t root, int32_t sid, std::vector<int32_t>& q, std::vector<int32_t>& ls) {
        ++cur_bfs;
        q.clear(); ls.clear();
        q.push_back(root); visit[root] = cur_bfs; lev[root] = 0;
        ls.push_back(0);
        size_t head = 0;
        int32_t L = 0;
        while (head < q.size()) {
            size_t end = q.size();
            for (; head < end; ++head) {
                int32_t v = q[head];
                for_each_nbr(v, sid, [&](int32_t u) {
                    if (visit[u] != cur_bfs) { visit[u] = cur_bfs; lev[u] = L + 1; q.push_back(u); }
                });
            }
            if (q.size() > end) { ls.push_back((int32_t)end); ++L; }
        }
        ls.push_back((int32_t)q.size());
    }

    void emit_sorted(std::vector<int32_t>& S) {
        std::sort(S.begin(), S.end());
        out.insert(out.end(), S.begin(), S.end());
    }

    // Interval cut: when the set's vertices are intervals over the element
    // ranks, a rank t splits them into those ending at or before t (A), those
    // starting after t (B) and those containing the gap (the separator): an
    // element joins only vertices whose intervals contain its rank, so no
    // element connects A with B; a direct edge between A and B (not made by an
    // element) moves its A end into the separator.  Among the cuts leaving at
    // least an eighth of the set on each side, the one minimising
    // |separator| / sqrt(smaller side) is taken (a small separator, traded
    // against balance).  Returns false when no such cut exists.
    bool interval_cut(const std::vector<int32_t>& S, int32_t sid, std::vector<int32_t>& A, std::vector<int32_t>& B,
                      std::vector<int32_t>& sep) {
        int32_t t0 = INT32_MAX, t1 = -1;
        for (int32_t v : S) {
            if (ehi[v] < 0) return false;
            t0 = std::min(t0, elo[v]);
            t1 = std::max(t1, ehi[v]);
        }
        const int32_t span = t1 - t0 + 1;
        if (span < 2) return false;
        std::vector<int32_t> dS((size_t)span + 1, 0), ends((size_t)span, 0);
        for (int32_t v : S) {
            dS[elo[v] - t0]++;
            dS[ehi[v] - t0]--;
            ends[ehi[v] - t0]++;
        }
        const int64_t minside = (int64_t)S.size() / 8;
        int64_t sc = 0, lc = 0;
        double best_s = 1e300;
        int32_t best_t = -1;
        for (int32_t t = 0; t + 1 < span; ++t) {
            sc += dS[t];     // vertices with lo <= t < hi
            lc += ends[t];   // vertices with hi <= t
            const int64_t rc = (int64_t)S.size() - sc - lc;
            if (lc < minside || rc < minside) continue;
            const double cost = (double)sc / std::sqrt((double)std::min(lc, rc));
            if (cost < best_s) { best_s = cost; best_t = t; }
        }
        if (best_t < 0) return false;
        const int32_t t = t0 + best_t;
        A.clear(); B.clear(); sep.clear();
        for (int32_t v : S) {
            if (ehi[v] <= t) {
                bool cross = false;
                for (int64_t p = xadj[v]; p < xadj[v + 1] && !cross; ++p) {
                    const int32_t u = adj[p];
                    cross = !is_elem[u] && stamp[u] == sid && elo[u] > t;
                }
                (cross ? sep : A).push_back(v);
            } else if (elo[v] > t) {
                B.push_back(v);
            } else {
                sep.push_back(v);
            }
        }
        return true;
    }

    void dissect(std::vector<int32_t> S) {
        if ((int64_t)S.size() <= leaf) { emit_sorted(S); return; }
        int32_t sid = ++cur_set;
        for (int32_t v : S) stamp[v] = sid;
        std::vector<int32_t> q, ls;
        // connected components
        bfs(S[0], sid, q, ls);
        if (q.size() < S.size()) {
            int32_t dm = ++cur_done;
            std::vector<std::vector<int32_t>> comps;
            for (int32_t v : S) {
                if (done[v] == dm) continue;
                bfs(v, sid, q, ls);
                for (int32_t u : q) done[u] = dm;
                comps.push_back(q);
            }
            for (auto& c : comps) dissect(std::move(c));
            return;
        }
        // an interval cut when the elements give one, else a level-structure separator
        {
            std::vector<int32_t> Ai, Bi, sepi;
            if (interval_cut(S, sid, Ai, Bi, sepi)) {
                dissect(std::move(Ai));
                dissect(std::move(Bi));
                emit_sorted(sepi);
                return;
            }
        }
        // pseudo-peripheral root: restart from a minimum-degree vertex of the last level
        int32_t root = S[0];
        for (int32_t v : S) if (deg(v) < deg(root)) root = v;
        bfs(root, sid, q, ls);
        int32_t nlev = (int32_t)ls.size() - 1;
        for (int it = 0; it < 4; ++it) {
            int32_t cand = q[ls[nlev - 1]];
            for (int32_t t = ls[nlev - 1]; t < ls[nlev]; ++t)
                if (deg(q[t]) < deg(cand)) cand = q[t];
            std::vector<int32_t> q2, ls2;
            bfs(cand, sid, q2, ls2);
            int32_t nl2 = (int32_t)ls2.size() - 1;
            if (nl2 > nlev) { root = cand; q.swap(q2); ls.swap(ls2); nlev = nl2; }
            else { bfs(root, sid, q, ls); break; }
        }
        if (nlev < 3) { emit_sorted(S); return; }
        // separator: the smallest level near the median vertex
        int64_t half = (int64_t)S.size() / 2, cum = 0;
        int32_t mid = 1;
        for (int32_t l = 0; l < nlev; ++l) {
            cum += ls[l + 1] - ls[l];
            if (cum >= half) { mid = l; break; }
        }
        mid = std::min(std::max(mid, 1), nlev - 2);
        int32_t w = std::max(1, nlev / 10), best = mid;
        for (int32_t l = std::max(1, mid - w); l <= std::min(nlev - 2, mid + w); ++l)
            if (ls[l + 1] - ls[l] < ls[best + 1] - ls[best]) best = l;
        std::vector<int32_t> A(q.begin(), q.begin() + ls[best]);
        std::vector<int32_t> B(q.begin() + ls[best + 1], q.end());
        std::vector<int32_t> sep;
        // thin the separator: a level vertex with no neighbour in the next level joins A
        ++cur_bfs;  // fresh element stamps for the neighbour scans
        int32_t bfs_id = cur_bfs - 1;
        for (int32_t t = ls[best]; t < ls[best + 1]; ++t) {
            int32_t v = q[t];
            bool nb = false;
            // element stamps must not suppress repeated scans for different v
            for (int64_t p = xadj[v]; p < xadj[v + 1] && !nb; ++p) {
                int32_t u = adj[p];
                if (is_elem[u]) {
                    for (int64_t r = xadj[u]; r < xadj[u + 1]; ++r) {
                        int32_t x = adj[r];
                        if (stamp[x] == sid && !is_elem[x] && visit[x] == bfs_id && lev[x] == best + 1) { nb = true; break; }
                    }
                } else if (stamp[u] == sid && visit[u] == bfs_id && lev[u] == best + 1) {
                    nb = true;
                }
            }
            (nb ? sep : A).push_back(v);
        }
        dissect(std::move(A));
        dissect(std::move(B));
        emit_sorted(sep);
    }
};
}  // namespace

std::vector<int32_t> order_nested_dissection(int32_t n, const std::vector<int64_t>& xadj,
                                             const std::vector<int32_t>& adj, int leaf) {
    ND nd(n, xadj, adj, leaf);
    // 1. independent set of local degree minima, eliminated first
    std::vector<int32_t> byd(n);
    std::iota(byd.begin(), byd.end(), 0);
    std::stable_sort(byd.begin(), byd.end(), [&](int32_t a, int32_t b) { return nd.deg(a) < nd.deg(b); });
    std::vector<char> blocked(n, 0);
    std::vector<int32_t> first;
    for (int32_t v : byd) {
        if (blocked[v]) continue;
        bool localmin = true;
        for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p)
            if (nd.deg(adj[p]) < nd.deg(v)) { localmin = false; break; }
        if (!localmin || nd.deg(v) == 0) continue;
        nd.is_elem[v] = 1;
        first.push_back(v);
        blocked[v] = 1;
        for (int64_t p = xadj[v]; p < xadj[v + 1]; ++p) blocked[adj[p]] = 1;
    }
    // an all-elements graph (e.g. diagonal) needs no dissection
    std::vector<int32_t> rest;
    for (int32_t v = 0; v < n; ++v) if (!nd.is_elem[v]) rest.push_back(v);
    std::sort(first.begin(), first.end());
    for (int32_t r = 0; r < (int32_t)first.size(); ++r)
        for (int64_t p = xadj[first[r]]; p < xadj[first[r] + 1]; ++p) {
            const int32_t v = adj[p];
            nd.elo[v] = std::min(nd.elo[v], r);
            nd.ehi[v] = std::max(nd.ehi[v], r);
        }
    nd.out = first;
    if (!rest.empty()) nd.dissect(std::move(rest));
    return nd.out;
}

int analyse(int64_t n64, const int64_t* cp, const int32_t* ri, const AnalyseParams& prm,
            Symbolic& S, std::string& err) {
    if (n64 < 0 || n64 > INT32_MAX - 1) { err = "n out of range"; return kErrArg; }
    const int32_t n = (int32_t)n64;
    if (n > 0 && (!cp || !ri)) { err = "NULL pattern"; return kErrArg; }
    if (n > 0 && cp[0] != 0) { err = "colptr[0] != 0"; return kErrPattern; }
    for (int32_t j = 0; j < n; ++j) {
        if (cp[j + 1] <= cp[j]) { err = "empty column " + std::to_string(j) + " (diagonal missing)"; return kErrPattern; }
        if (ri[cp[j]] != j) { err = "column " + std::to_string(j) + " does not start with its diagonal"; return kErrPattern; }
        for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) {
            if (ri[p] <= ri[p - 1]) { err = "column " + std::to_string(j) + " rows not strictly increasing"; return kErrPattern; }
            if (ri[p] >= n) { err = "row index out of range in column " + std::to_string(j); return kErrPattern; }
        }
    }
    try {
        S = Symbolic();
        S.n = n;
        S.nnz_a = n > 0 ? cp[n] : 0;
        // ---- ordering
        std::vector<int32_t> perm0(n);
        if (prm.ordering == 1 || n == 0) {
            std::iota(perm0.begin(), perm0.end(), 0);
        } else if (prm.ordering == 0) {
            std::vector<int64_t> xadj;
            std::vector<int32_t> adj;
            build_graph(n, cp, ri, xadj, adj);
            perm0 = order_nested_dissection(n, xadj, adj, prm.nd_leaf > 0 ? prm.nd_leaf : 64);
        } else {
            err = "unknown ordering"; return kErrArg;
        }
        std::vector<int32_t> ip0(n);
        for (int32_t k = 0; k < n; ++k) ip0[perm0[k]] = k;
        // ---- lower pattern by rows in the ordered numbering (cols k < i of row i)
        auto rows_of = [&](const std::vector<int32_t>& ip, std::vector<int64_t>& rp, std::vector<int32_t>& rc) {
            rp.assign((size_t)n + 1, 0);
            for (int32_t j = 0; j < n; ++j)
                for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) {
                    int32_t a = ip[ri[p]], b = ip[j];
                    rp[std::max(a, b) + 1]++;
                }
            for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
            rc.resize((size_t)rp[n]);
            std::vector<int64_t> f(rp.begin(), rp.end() - 1);
            for (int32_t j = 0; j < n; ++j)
                for (int64_t p = cp[j] + 1; p < cp[j + 1]; ++p) {
                    int32_t a = ip[ri[p]], b = ip[j];
                    rc[f[std::max(a, b)]++] = std::min(a, b);
                }
        };
        std::vector<int64_t> rp;
        std::vector<int32_t> rc;
        rows_of(ip0, rp, rc);
        // ---- elimination tree (Liu, path compression)
        std::vector<int32_t> par(n, -1), anc(n, -1);
        for (int32_t i = 0; i < n; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int32_t r = rc[p];
                while (r != -1 && r < i) {
                    int32_t nx = anc[r];
                    anc[r] = i;
                    if (nx == -1) { par[r] = i; break; }
                    r = nx;
                }
            }
        // ---- postorder: childless children first, then the others, each in increasing
        //      order, so that a node's leaf children are numbered consecutively
        std::vector<int32_t> head(n, -1), nxt(n, -1), post, nkids(n, 0);
        post.reserve(n);
        for (int32_t v = 0; v < n; ++v) if (par[v] != -1) nkids[par[v]]++;
        // a column whose supernode must merge into its parent's is visited last among its
        // parent's children, so that it is numbered just before its parent (contiguous)
        const bool forcing = !prm.force_merge.empty();
        auto forced0 = [&](int32_t v) { return forcing && prm.force_merge[(size_t)perm0[v]] != 0; };
        for (int32_t v = n - 1; v >= 0; --v)
            if (par[v] != -1 && forced0(v)) { nxt[v] = head[par[v]]; head[par[v]] = v; }
        for (int pass = 0; pass < 2; ++pass)
            for (int32_t v = n - 1; v >= 0; --v)
                if (par[v] != -1 && !forced0(v) && (nkids[v] == 0) == (pass == 1)) {
                    nxt[v] = head[par[v]];
                    head[par[v]] = v;
                }
        if (!forcing) {
            std::vector<int32_t> stk;
            for (int32_t r = 0; r < n; ++r) {
                if (par[r] != -1) continue;
                stk.push_back(r);
                while (!stk.empty()) {
                    int32_t v = stk.back();
                    if (head[v] != -1) { int32_t c = head[v]; head[v] = nxt[c]; stk.push_back(c); }
                    else { stk.pop_back(); post.push_back(v); }
                }
            }
        } else {
            // Forced columns are numbered late: a forced column is held back (with the
            // forced columns below it that were held back) until its parent's subtree is
            // otherwise complete, then all are numbered just before the parent.  The
            // order stays topological (every column after its descendants), so the
            // elimination tree and the fill are unchanged; subtrees of forced columns are
            // no longer contiguous, which only widens the variance plan's active ranges.
            struct Frame { int32_t v; bool held; size_t dstart; };
            std::vector<Frame> st;
            std::vector<int32_t> held;
            for (int32_t r = 0; r < n; ++r) {
                if (par[r] != -1) continue;
                st.push_back(Frame{r, false, held.size()});
                while (!st.empty()) {
                    Frame& F = st.back();
                    if (head[F.v] != -1) {
                        const int32_t c = head[F.v];
                        head[F.v] = nxt[c];
                        st.push_back(Frame{c, forced0(c), held.size()});
                        continue;
                    }
                    const Frame done = F;
                    st.pop_back();
                    if (done.held) {
                        held.push_back(done.v);  // the held region moves up with it
                    } else {
                        for (size_t q = done.dstart; q < held.size(); ++q) post.push_back(held[q]);
                        held.resize(done.dstart);
                        post.push_back(done.v);
                    }
                }
            }
        }
        std::vector<int32_t> newpos(n);
        for (int32_t k = 0; k < n; ++k) newpos[post[k]] = k;
        S.perm.resize(n); S.iperm.resize(n); S.parent.assign(n, -1);
        for (int32_t k = 0; k < n; ++k) {
            S.perm[k] = perm0[post[k]];
            S.iperm[S.perm[k]] = k;
            int32_t pv = par[post[k]];
            S.parent[k] = pv == -1 ? -1 : newpos[pv];
        }
        rows_of(S.iperm, rp, rc);
        // ---- column counts from row subtrees
        std::vector<int32_t> cnt(n, 0), mark(n, -1);
        for (int32_t i = 0; i < n; ++i) {
            mark[i] = i;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                for (int32_t j = rc[p]; mark[j] != i; j = S.parent[j]) { cnt[j]++; mark[j] = i; }
        }
        S.colcount.resize(n);
        S.nnz_l = 0; S.factor_flops = 0;
        for (int32_t j = 0; j < n; ++j) {
            S.colcount[j] = cnt[j] + 1;
            S.nnz_l += cnt[j];
            S.factor_flops += (double)S.colcount[j] * S.colcount[j] - 1.0;
        }
        {
            std::vector<double> ps(n, 0.0);
            S.diag_flops_all = 0;
            for (int32_t j = n - 1; j >= 0; --j) {
                ps[j] = 2.0 * S.colcount[j] + (S.parent[j] == -1 ? 0.0 : ps[S.parent[j]]);
                S.diag_flops_all += ps[j];
            }
        }
        S.fdesc.resize(n);
        std::iota(S.fdesc.begin(), S.fdesc.end(), 0);
        std::vector<int32_t> ncc(n, 0);
        for (int32_t j = 0; j < n; ++j)
            if (S.parent[j] != -1) {
                S.fdesc[S.parent[j]] = std::min(S.fdesc[S.parent[j]], S.fdesc[j]);
                ncc[S.parent[j]]++;
            }
        // input column access in pivot numbering: lower entries (r >= c) grouped by column c
        std::vector<int64_t> ccp((size_t)n + 1, 0);
        std::vector<int32_t> crow;
        {
            for (int32_t i = 0; i < n; ++i)
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) ccp[rc[p] + 1]++;
            for (int32_t j = 0; j < n; ++j) ccp[j + 1] += ccp[j];
            crow.resize((size_t)ccp[n]);
            std::vector<int64_t> f(ccp.begin(), ccp.end() - 1);
            for (int32_t i = 0; i < n; ++i)
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) crow[f[rc[p]]++] = i;
        }
        // ---- fundamental supernodes
        std::vector<int32_t> sf;
        for (int32_t j = 0; j < n; ++j) {
            bool cont = j > 0 && S.parent[j - 1] == j && S.colcount[j - 1] == S.colcount[j] + 1 && ncc[j] == 1;
            if (!cont) sf.push_back(j);
        }
        sf.push_back(n);
        int32_t nf = (int32_t)sf.size() - 1;
        // supernode parent (via the last column) for the fundamental partition
        std::vector<int32_t> fsn(n);
        for (int32_t s = 0; s < nf; ++s)
            for (int32_t j = sf[s]; j < sf[s + 1]; ++j) fsn[j] = s;
        // ---- relaxed amalgamation: merge a supernode into its parent when it is the
        //      parent's last child (columns contiguous) and the explicit zeros stay small
        std::vector<int32_t> grp(nf);          // representative (the surviving parent) of each
        std::vector<int64_t> gm(nf), gk(nf), gz(nf), gf(nf);
        for (int32_t s = 0; s < nf; ++s) {
            grp[s] = s; gk[s] = sf[s + 1] - sf[s]; gm[s] = S.colcount[sf[s]]; gz[s] = 0; gf[s] = sf[s];
        }
        std::vector<char> merged(nf, 0);
        if (prm.relax > 0) {
            for (int32_t s = 0; s < nf; ++s) {
                int32_t lc = sf[s + 1] - 1;
                int32_t pc = S.parent[lc];
                if (pc == -1) continue;
                int32_t p = fsn[pc];
                if (sf[p] != lc + 1) continue;  // not contiguous (not the last child)
                // s (with whatever merged into it) is the group of s; p is a fundamental supernode
                int64_t ks = gk[s], ms = gm[s], kp = gk[p], mp = gm[p];
                int64_t mnew = ks + mp, knew = ks + kp;
                int64_t znew = gz[s] + gz[p] + ks * (mnew - ms);
                int64_t stored = knew * mnew - knew * (knew + 1) / 2;
                bool ok = (double)znew <= prm.relax / 100.0 * (double)stored ||
                          (knew <= 16 && 2 * znew <= stored);
                if (!ok) continue;
                gk[p] = knew; gm[p] = mnew; gz[p] = znew; gf[p] = gf[s];
                merged[s] = 1;
            }
        }
        std::vector<int32_t> part;
        for (int32_t s = 0; s < nf; ++s)
            if (!merged[s]) part.push_back((int32_t)gf[s]);
        part.push_back(n);
        // forced merges: from the last group back, a group whose last column is forced
        // joins the group right after it when that group holds its parent (the forced
        // columns were numbered just before their parents, above)
        if (forcing && part.size() > 2) {
            const int32_t ng = (int32_t)part.size() - 1;
            std::vector<char> start((size_t)ng, 1);
            int32_t end_next = part[ng];  // end of the (merged) group that starts at part[g + 1]
            for (int32_t g = ng - 2; g >= 0; --g) {
                const int32_t b = part[g + 1] - 1, pb = S.parent[b];
                const bool fb = prm.force_merge[(size_t)S.perm[b]] != 0;
                if (fb && pb >= part[g + 1] && pb < end_next) {
                    start[(size_t)g + 1] = 0;  // merged: the group now starts at part[g]
                } else {
                    end_next = part[g + 1];
                }
            }
            std::vector<int32_t> p2;
            for (int32_t g = 0; g < ng; ++g)
                if (start[(size_t)g]) p2.push_back(part[g]);
            p2.push_back(n);
            part.swap(p2);
        }
        // ---- sibling grouping: consecutive childless supernodes with the same parent are
        //      merged into one front (their columns are independent: a diagonal pivot block)
        //      while the merged rank-k update costs at most 2.5x the separate updates
        if (prm.relax > 0 && prm.group_max > 1) {
            const int32_t np_ = (int32_t)part.size() - 1;
            std::vector<int32_t> pn(n), ppar(np_, -1);
            std::vector<char> haskid(np_, 0);
            for (int32_t s = 0; s < np_; ++s)
                for (int32_t j = part[s]; j < part[s + 1]; ++j) pn[j] = s;
            for (int32_t s = 0; s < np_; ++s) {
                int32_t pc = S.parent[part[s + 1] - 1];
                if (pc != -1) { ppar[s] = pn[pc]; haskid[pn[pc]] = 1; }
            }
            std::vector<int32_t> stamp(n, -1), grouped;
            int32_t s = 0;
            while (s < np_) {
                grouped.push_back(part[s]);
                if (haskid[s] || ppar[s] == -1) { ++s; continue; }
                // start a group at s
                auto add_rows = [&](int32_t t, int32_t g, int64_t& cnt) {
                    for (int32_t j = part[t]; j < part[t + 1]; ++j)
                        for (int64_t p = ccp[j]; p < ccp[j + 1]; ++p) {
                            int32_t r = crow[p];
                            if (r >= part[t + 1] && stamp[r] != g) { stamp[r] = g; ++cnt; }
                        }
                };
                auto below = [&](int32_t t) {  // |rows below| of a childless supernode
                    return (int64_t)S.colcount[part[t]] - (part[t + 1] - part[t]);
                };
                int64_t ucnt = 0, kg = part[s + 1] - part[s];
                double exact = (double)below(s) * below(s) * kg;
                add_rows(s, s, ucnt);
                int32_t t = s + 1;
                while (t < np_ && !haskid[t] && ppar[t] == ppar[s]) {
                    int64_t kt = part[t + 1] - part[t];
                    if (kg + kt > prm.group_max) break;
                    int64_t trial = ucnt;
                    // count without committing: stamp with a temporary id then roll back if rejected
                    std::vector<int32_t> added;
                    for (int32_t j = part[t]; j < part[t + 1]; ++j)
                        for (int64_t p = ccp[j]; p < ccp[j + 1]; ++p) {
                            int32_t r = crow[p];
                            if (r >= part[t + 1] && stamp[r] != s) { stamp[r] = s; ++trial; added.push_back(r); }
                        }
                    double ex2 = exact + (double)below(t) * below(t) * kt;
                    double merged_cost = (double)trial * trial * (kg + kt);
                    if (merged_cost > prm.group_cost * ex2) {
                        for (int32_t r : added) stamp[r] = -1;
                        break;
                    }
                    ucnt = trial; kg += kt; exact = ex2;
                    ++t;
                }
                s = t;
            }
            grouped.push_back(n);
            part.swap(grouped);
        }
        S.sfirst = part;
        // a front whose columns are all childless and have no entry between them has a
        // diagonal pivot block (grouped sibling leaves)
        {
            const int32_t np2 = (int32_t)S.sfirst.size() - 1;
            S.sdiag.assign(np2, 0);
            for (int32_t s2 = 0; s2 < np2; ++s2) {
                const int32_t f = S.sfirst[s2], l = S.sfirst[s2 + 1] - 1;
                if (l == f) continue;
                bool diag = true;
                for (int32_t j = f; j <= l && diag; ++j) {
                    if (ncc[j] != 0) diag = false;
                    for (int64_t p = ccp[j]; p < ccp[j + 1] && diag; ++p)
                        if (crow[p] > j && crow[p] <= l) diag = false;
                }
                S.sdiag[s2] = diag ? 1 : 0;
            }
        }
        S.ns = (int32_t)S.sfirst.size() - 1;
        const int32_t ns = S.ns;
        S.snode_of.resize(n);
        for (int32_t s = 0; s < ns; ++s)
            for (int32_t j = S.sfirst[s]; j < S.sfirst[s + 1]; ++j) S.snode_of[j] = s;
        S.sparent.assign(ns, -1);
        S.nchild.assign(ns, 0);
        for (int32_t s = 0; s < ns; ++s) {
            int32_t pc = S.parent[S.sfirst[s + 1] - 1];
            if (pc != -1) { S.sparent[s] = S.snode_of[pc]; S.nchild[S.sparent[s]]++; }
        }
        // ---- front row lists: own columns, input rows below, children's rows below
        std::vector<int32_t> cfirst(ns + 1, 0), clist(ns);
        for (int32_t s = 0; s < ns; ++s) if (S.sparent[s] != -1) cfirst[S.sparent[s] + 1]++;
        for (int32_t s = 0; s < ns; ++s) cfirst[s + 1] += cfirst[s];
        {
            std::vector<int32_t> f(cfirst.begin(), cfirst.end() - 1);
            for (int32_t s = 0; s < ns; ++s) if (S.sparent[s] != -1) clist[f[S.sparent[s]]++] = s;
        }
        S.srowptr.assign((size_t)ns + 1, 0);
        S.srows.clear();
        std::fill(mark.begin(), mark.end(), -1);
        std::vector<int32_t> tmp;
        for (int32_t s = 0; s < ns; ++s) {
            int32_t f = S.sfirst[s], l = S.sfirst[s + 1] - 1;
            tmp.clear();
            for (int32_t j = f; j <= l; ++j) { tmp.push_back(j); mark[j] = s; }
            for (int32_t j = f; j <= l; ++j)
                for (int64_t p = ccp[j]; p < ccp[j + 1]; ++p) {
                    int32_t r = crow[p];
                    if (r > l && mark[r] != s) { mark[r] = s; tmp.push_back(r); }
                }
            for (int32_t t = cfirst[s]; t < cfirst[s + 1]; ++t) {
                int32_t c = clist[t];
                for (int64_t p = S.srowptr[c]; p < S.srowptr[c + 1]; ++p) {
                    int32_t r = S.srows[p];
                    if (r > l && mark[r] != s) { mark[r] = s; tmp.push_back(r); }
                }
            }
            std::sort(tmp.begin() + (l - f + 1), tmp.end());
            S.srows.insert(S.srows.end(), tmp.begin(), tmp.end());
            S.srowptr[s + 1] = (int64_t)S.srows.size();
        }
        // ---- relative maps, storage offsets, levels
        S.relmap.assign(S.srows.size(), -1);
        S.lptr.assign((size_t)ns + 1, 0);
        S.f22ptr.assign(ns, -1);
        S.f22_total = 0;
        S.max_front = 0;
        S.nnz_l_stored = 0;
        for (int32_t s = 0; s < ns; ++s) {
            int64_t m = S.m_of(s), k = S.k_of(s);
            S.lptr[s + 1] = S.lptr[s] + m * k;
            S.nnz_l_stored += m * k - k * (k + 1) / 2;
            S.max_front = std::max(S.max_front, m);
            if (S.nchild[s] > 0 && m > k) { S.f22ptr[s] = S.f22_total; S.f22_total += (m - k) * (m - k); }
            int32_t p = S.sparent[s];
            if (p == -1) {
                if (m != k) { err = "internal: root front with rows below"; return kErrPattern; }
                continue;
            }
            const int32_t* pr = &S.srows[S.srowptr[p]];
            int64_t mp = S.m_of(p), q = 0;
            for (int64_t t = k; t < m; ++t) {
                int32_t r = S.srows[S.srowptr[s] + t];
                while (q < mp && pr[q] < r) ++q;
                if (q == mp || pr[q] != r) { err = "internal: child row missing in parent front"; return kErrPattern; }
                S.relmap[S.srowptr[s] + t] = (int32_t)q;
            }
        }
        S.level.assign(ns, 0);
        int32_t maxl = 0;
        for (int32_t s = 0; s < ns; ++s) {
            int32_t p = S.sparent[s];
            if (p != -1) S.level[p] = std::max(S.level[p], S.level[s] + 1);
            maxl = std::max(maxl, S.level[s]);
        }
        S.nlevels = ns > 0 ? maxl + 1 : 0;
        S.level_ptr.assign((size_t)S.nlevels + 1, 0);
        for (int32_t s = 0; s < ns; ++s) S.level_ptr[S.level[s] + 1]++;
        for (int32_t l = 0; l < S.nlevels; ++l) S.level_ptr[l + 1] += S.level_ptr[l];
        S.level_list.resize(ns);
        {
            std::vector<int32_t> f(S.level_ptr.begin(), S.level_ptr.end() - 1);
            for (int32_t s = 0; s < ns; ++s) S.level_list[f[S.level[s]]++] = s;
        }
        // ---- input entry -> panel offset
        S.amap.resize((size_t)S.nnz_a);
        S.diag_src.resize(n);
        for (int32_t j = 0; j < n; ++j) {
            S.diag_src[S.iperm[j]] = (int32_t)cp[j];
            for (int64_t p = cp[j]; p < cp[j + 1]; ++p) {
                int32_t a = S.iperm[ri[p]], b = S.iperm[j];
                int32_t r = std::max(a, b), c = std::min(a, b);
                int32_t s = S.snode_of[c];
                const int32_t* rows = &S.srows[S.srowptr[s]];
                int64_t m = S.m_of(s);
                int64_t t = std::lower_bound(rows, rows + m, r) - rows;
                if (t == m || rows[t] != r) { err = "internal: input entry outside its front"; return kErrPattern; }
                S.amap[p] = S.lptr[s] + t + (int64_t)(c - S.sfirst[s]) * m;
            }
        }
    } catch (const std::bad_alloc&) {
        err = "host allocation failed";
        return kErrOom;
    }
    return 0;
}

void build_diag_plan(const Symbolic& S, const std::vector<int32_t>& pivots,
                     const std::vector<int32_t>& out_pos, int B, DiagPlan& P) {
    P = DiagPlan();
    P.B = B;
    const int64_t nr = (int64_t)pivots.size();
    P.nrhs = nr;
    std::vector<int64_t> ord(nr);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return pivots[a] < pivots[b]; });
    P.rhs_col.resize(nr); P.rhs_out.resize(nr);
    for (int64_t t = 0; t < nr; ++t) { P.rhs_col[t] = pivots[ord[t]]; P.rhs_out[t] = out_pos[ord[t]]; }
    P.nblocks = (int32_t)((nr + B - 1) / B);
    P.blk_ptr.resize((size_t)P.nblocks + 1);
    for (int32_t b = 0; b <= P.nblocks; ++b) P.blk_ptr[b] = (int32_t)std::min<int64_t>(nr, (int64_t)b * B);
    // algorithmic flops: sum over requested i of sum over j on path(i) of 2 c_j
    std::vector<double> pathsum(S.n, 0.0);
    for (int32_t j = S.n - 1; j >= 0; --j)
        pathsum[j] = 2.0 * S.colcount[j] + (S.parent[j] == -1 ? 0.0 : pathsum[S.parent[j]]);
    for (int64_t t = 0; t < nr; ++t) P.flops += pathsum[P.rhs_col[t]];
    std::vector<int32_t> mark(S.ns, -1), zloc(S.ns, 0);
    std::vector<int32_t> U;
    std::vector<double> bwork(P.nblocks, 0.0);
    P.uptr.assign(1, 0);
    P.zbase.assign(1, 0);
    for (int32_t b = 0; b < P.nblocks; ++b) {
        U.clear();
        int32_t r0 = P.blk_ptr[b], r1 = P.blk_ptr[b + 1];
        for (int32_t t = r0; t < r1; ++t)
            for (int32_t s = S.snode_of[P.rhs_col[t]]; s != -1 && mark[s] != b; s = S.sparent[s]) {
                mark[s] = b;
                U.push_back(s);
            }
        std::sort(U.begin(), U.end());
        int32_t z = 0;
        for (int32_t s : U) { zloc[s] = z; z += S.k_of(s); }
        for (int32_t t = r0; t < r1; ++t) {
            int32_t col = P.rhs_col[t], sn = S.snode_of[col];
            P.rhs_zrow.push_back(zloc[sn] + (col - S.sfirst[sn]));
        }
        for (int32_t s : U) {
            // subtree of the supernode: [fdesc(last column), last column], or its own columns
            // for a group of sibling leaves
            int32_t lcol = S.sfirst[s + 1] - 1, lo_col = std::min(S.fdesc[lcol], S.sfirst[s]);
            auto beg = P.rhs_col.begin() + r0, end = P.rhs_col.begin() + r1;
            int32_t lo = (int32_t)(std::lower_bound(beg, end, lo_col) - beg);
            int32_t hi = (int32_t)(std::upper_bound(beg, end, lcol) - beg);
            P.us.push_back(s); P.ulo.push_back(lo); P.uhi.push_back(hi); P.uzoff.push_back(zloc[s]);
            P.urel.push_back((int64_t)P.rel.size());
            int64_t m = S.m_of(s), k = S.k_of(s);
            for (int64_t t = k; t < m; ++t) {
                int32_t col = S.srows[S.srowptr[s] + t];
                int32_t sn = S.snode_of[col];
                P.rel.push_back(zloc[sn] + (col - S.sfirst[sn]));
            }
            // executed flops: per 32-column block, the triangle, the padded update of the
            // rows below and the variance terms, for each active right-hand side
            // (per block column only the right-hand sides in the union of its columns' subtrees)
            double w = 0.0;
            for (int64_t cb = 0; cb < k; cb += 32) {
                const double wc = (double)std::min<int64_t>(32, k - cb), w4 = wc;
                const int32_t j0 = S.sfirst[s] + (int32_t)cb, j1 = j0 + (int32_t)wc - 1;
                int32_t first = j0;
                for (int32_t j = j0; j <= j1; ++j) first = std::min(first, S.fdesc[j]);
                const double nbe = (double)(std::lower_bound(beg + lo, beg + hi, j1 + 1) -
                                            std::lower_bound(beg + lo, beg + hi, first));
                w += nbe * (wc * (wc - 1.0) + 2.0 * (double)(m - cb - (int64_t)wc) * w4 + 3.0 * wc);
            }
            P.work_flops += w;
            bwork[b] += w;
        }
        P.uptr.push_back((int32_t)P.us.size());
        P.zbase.push_back(P.zbase.back() + (int64_t)z * B);
    }
    P.order.resize(P.nblocks);
    std::iota(P.order.begin(), P.order.end(), 0);
    std::stable_sort(P.order.begin(), P.order.end(), [&](int32_t a, int32_t b) { return bwork[a] > bwork[b]; });
}

}  // namespace spi
