// analysis.h -- host-side analysis phase (paper Sec. 3.2.1): ordering,
// elimination tree, postorder, column counts, supernodes, multifrontal
// assembly maps, level schedule, and the right-hand-side block plans of the
// pruned variance solves (Sec. 3.3.1).  Pure C++; no CUDA.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace spi {

struct AnalyseParams {
    int ordering = 0;  // 0 nested dissection, 1 natural
    int relax = 10;    // amalgamation: allowed explicit zeros, percent of the merged panel
    int nd_leaf = 0;   // nested-dissection leaf size, 0 = default
    int group_max = 32;  // most columns in one front of grouped sibling leaves
    double group_cost = 2.5;  // grouped leaves' update may cost this many times their separate updates
    // by caller column: 1 = the supernode holding this column is merged into its parent's
    // (the delayed pivots of a symmetric indefinite factorization); empty = none
    std::vector<uint8_t> force_merge;
};

struct Symbolic {
    int32_t n = 0;
    int64_t nnz_a = 0;
    std::vector<int32_t> perm;      // perm[k] = caller index of pivot k
    std::vector<int32_t> iperm;     // iperm[i] = pivot of caller index i
    std::vector<int32_t> parent;    // column elimination tree (pivot numbering), -1 = root
    std::vector<int32_t> colcount;  // |L(:,j)| + 1 (exact, before amalgamation)
    std::vector<int32_t> fdesc;     // first (smallest) pivot of the subtree of j
    // supernodes (postorder, contiguous pivot ranges)
    int32_t ns = 0;
    std::vector<int32_t> sfirst;    // [ns+1]
    std::vector<int32_t> sparent;   // [ns], -1 = root
    std::vector<int32_t> snode_of;  // [n]
    std::vector<int64_t> srowptr;   // [ns+1]
    std::vector<int32_t> srows;     // pivot rows of each front; the first k are its own columns
    std::vector<int32_t> relmap;    // aligned with srows: for t >= k, position in the parent's rows
    std::vector<int64_t> lptr;      // [ns+1] offsets of the m x k column-major panels
    std::vector<int64_t> f22ptr;    // [ns] offset of the (m-k)^2 update area, -1 if no child
    int64_t f22_total = 0;
    std::vector<int32_t> nchild;    // children per supernode
    std::vector<uint8_t> sdiag;     // 1: the pivot block is diagonal (a group of independent leaf columns)
    std::vector<int32_t> level;     // height of each supernode (leaves 0)
    std::vector<int32_t> level_ptr; // [nlevels+1]
    std::vector<int32_t> level_list;// supernodes by level
    std::vector<int64_t> amap;      // [nnz_a] offset in the panels of each input entry
    std::vector<int32_t> diag_src;  // [n] input position of the diagonal of pivot k
    double factor_flops = 0;        // sum_j (c_j^2 - 1)
    double diag_flops_all = 0;      // sum_i sum_{j in path(i)} 2 c_j over all pivots i
    int64_t nnz_l = 0;              // sum_j (c_j - 1)
    int64_t nnz_l_stored = 0;       // sum_s m_s k_s
    int64_t max_front = 0;
    int32_t nlevels = 0;

    int32_t k_of(int32_t s) const { return sfirst[s + 1] - sfirst[s]; }
    int32_t m_of(int32_t s) const { return (int32_t)(srowptr[s + 1] - srowptr[s]); }
};

// Block plan of the pruned forward solves for a set of right-hand sides e_i.
struct DiagPlan {
    int32_t B = 128;
    int32_t nblocks = 0;
    int64_t nrhs = 0;
    std::vector<int32_t> rhs_col;   // pivot of each RHS slot, ascending
    std::vector<int32_t> rhs_out;   // output position of each RHS slot
    std::vector<int32_t> rhs_zrow;  // local Z row of each RHS slot's own pivot
    std::vector<int32_t> blk_ptr;   // [nblocks+1] into rhs slots
    std::vector<int32_t> uptr;      // [nblocks+1] into the per-block supernode list
    std::vector<int32_t> us;        // supernode (ascending within a block)
    std::vector<int32_t> ulo, uhi;  // active RHS range [lo, hi) of the block at that supernode
    std::vector<int32_t> uzoff;     // local Z row of the supernode's first column
    std::vector<int64_t> urel;      // offset into rel of the supernode's below-row map
    std::vector<int32_t> rel;       // local Z rows of the below rows
    std::vector<int64_t> zbase;     // [nblocks+1] Z offsets (rows * B doubles)
    std::vector<int32_t> order;     // blocks by decreasing estimated work
    double flops = 0;               // algorithmic: sum_i sum_{j in path(i)} 2 c_j
    double work_flops = 0;          // what the blocked kernel executes
};

// Returns 0 on success, or an spi_status code with a message in err.
int analyse(int64_t n, const int64_t* colptr, const int32_t* rowind, const AnalyseParams& prm,
            Symbolic& S, std::string& err);

// pivots: requested pivots (any order, no duplicates checked by caller);
// out_pos[t] is where RHS t writes its result.
void build_diag_plan(const Symbolic& S, const std::vector<int32_t>& pivots,
                     const std::vector<int32_t>& out_pos, int B, DiagPlan& P);

// Orderings (exposed for tests through the C ABI's perm export).
std::vector<int32_t> order_nested_dissection(int32_t n, const std::vector<int64_t>& xadj,
                                             const std::vector<int32_t>& adj, int leaf);

}  // namespace spi
