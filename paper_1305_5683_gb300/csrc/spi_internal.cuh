// spi_internal.cuh -- device-side data of a context and the kernel entry
// points shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "analysis.h"
#include "diag_tc_plan.h"
#include "spi.h"

namespace spi {

constexpr int kT = 32;  // tile edge of the front kernels

enum DevFlags : int { FLAG_NOT_SPD = 1, FLAG_TIMEOUT = 2, FLAG_BAD_INDEX = 4, FLAG_DELAY = 8 };

struct DevStatus {
    int flags;
    int bad_pivot;  // smallest failing pivot (atomicMin), INT32_MAX if none
};

// Pointers to the symbolic structure on the device.
struct DevSym {
    int32_t n = 0, ns = 0;
    const int32_t* sfirst = nullptr;
    const int64_t* srowptr = nullptr;
    const int32_t* srows = nullptr;
    const int32_t* relmap = nullptr;
    const int32_t* sparent = nullptr;
    const int64_t* lptr = nullptr;
    const int64_t* f22ptr = nullptr;
    const int32_t* perm = nullptr;
    const int32_t* snode_of = nullptr;
    const int32_t* fdesc = nullptr;   // first pivot of the subtree of each pivot
    // symmetric indefinite factorizations (spi_options.pivoting): D^-1 block by block;
    // null in the SPD form, where D is diagonal
    const double* dinv_a = nullptr;   // diagonal of D^-1 at each pivot
    const double* dinv_b = nullptr;   // D^-1 between a pivot and its 2x2 partner
    const int32_t* pair = nullptr;    // the partner pivot of a 2x2 block, -1 for a 1x1 pivot
};

// Outputs of the pivoting factorization (k_front_bk).
struct BkArgs {
    double* Dd;      // [n] diagonal of D
    double* Doff;    // [n] D[p + 1][p] at the first pivot p of a 2x2 block, else 0
    int32_t* pair;   // [n] partner of each pivot in a 2x2 block, -1 for a 1x1 pivot
    int32_t* lperm;  // [n] for pivot f + i of a supernode: the local index (before the
                     //     symmetric swaps) of the column eliminated there
    int* delay;      // [0] number of fronts that could not pivot, [1 ..] those supernodes
    int max_delay;
    int* count2x2;   // number of 2x2 pivots taken
};
void launch_front_bk(const DevSym& d, const int32_t* items, int count, double* L, double* F22, const BkArgs& a,
                     DevStatus* status, cudaStream_t st);

// Per-band strides of the batched (same-pattern) buffers; blockIdx.y selects
// the band.  All zero-stride fields are unused for a single problem.
struct Strides {
    int64_t L = 0;    // panel doubles per band (also FP32 panel floats per band)
    int64_t F22 = 0;  // update-area doubles per band
    int64_t n = 0;    // vector length per band
    int64_t nnz = 0;  // input values per band
    int64_t Z = 0;    // variance workspace elements per band
    int64_t out = 0;  // variance outputs per band
    int64_t Dn = 0;   // pivots of D per band in the solves (n; 0 when the right-hand sides
                      // of one factor take the band index, with L = 0 as well)
};

// A flattened work list of one kernel launch.
struct Launch {
    int kind;        // 0 pivot tile, 1 panel TRSM, 2 Schur+scatter, 3 trailing panel update,
                     // 7 tensor-core Schur+scatter (mixed precision), 8 diagonal-pivot front,
                     // 9 tensor-core trailing panel update of a wide front (mixed precision),
                     // 14 symmetric indefinite fronts with 2x2 pivots (one CTA each);
                     // 12 persistent per-level kernel: whole panels of small fronts, one CTA
                     // per front at a time; solves: 4 forward step, 5 backward first launch of
                     // a level, 6 backward step, 10 / 11 forward / backward sweep of a whole
                     // level, 15 / 16 forward / backward step of 128 columns (mixed form,
                     // inverted diagonal tiles); -1 a timing marker of the autotuner (no
                     // launch; `step` = group)
    int step;        // block column b for kinds 0/1
    int64_t off;     // offset into the item array of the kind
    int32_t count;   // CTAs (kind 12: fronts)
};

// One task of the dependency-driven factorization kernel (launch kind 13).
enum DagType : int32_t {
    kDagDiagFront = 0, kDagFused = 1, kDagPivot = 2, kDagTrsm = 3, kDagUpdate = 4, kDagSchur = 5,  // factorization
    kSolveFwd = 6, kSolveBwdInit = 7, kSolveBwdStep = 8                                            // solve
};
struct DagTask {
    int32_t type;      // DagType
    int32_t s;         // supernode
    int32_t a, b;      // kDagTrsm: block step, 128-row chunk; kDagUpdate: block step, ti << 16 | tj;
                       // kDagSchur: ti, tj
    int32_t wait_idx;  // the task waits until counter[wait_idx] >= wait_val (0: no wait); counters
    int32_t wait_val;  //   [0, ns): tasks done of each front, [ns, 2 ns): children's Schur tiles added
    int32_t done_idx;  // counter incremented when the task is done
    int32_t pad;       // solve tasks: a second counter incremented when done (-1: none)
};

struct FactorPlan {
    std::vector<int32_t> diag_items;  // supernode
    std::vector<int32_t> trsm_items;  // pairs (supernode, row tile)
    std::vector<int32_t> schur_items; // triples (supernode, ti, tj)
    std::vector<int32_t> update_items;// triples (supernode, ti, tj) of the trailing panel
    std::vector<int32_t> schur_tc_items; // triples (supernode, 128-row tile, 64-column tile)
    std::vector<int32_t> dfront_items;   // supernodes with a diagonal pivot block
    std::vector<int32_t> panel_tc_items; // triples (supernode, 128-row tile, 64-column tile)
    std::vector<int32_t> fused_items;    // kind 12: supernode, or ~supernode for a diagonal pivot block
    std::vector<int32_t> bk_items;       // kind 14: supernodes of the pivoting (indefinite) form
    std::vector<DagTask> dag;            // kind 13: the tasks of the dependency-driven kernel, in order
    int32_t dag_levels = 0;              // levels [0, dag_levels) run in it
    std::vector<Launch> launches;
    std::vector<int32_t> level_launch_ptr;  // launches of level l: [ptr[l], ptr[l+1])
    // timing groups of an autotuner plan (markers): what the launches up to the
    // next marker do, for one front-size bucket of one level
    enum GroupKind { kPanel = 0, kSchur = 1, kDiagFronts = 2, kEnd = 3 };
    struct Group {
        int kind;
        int32_t bucket;
    };
    std::vector<Group> groups;
    int64_t n_kernel_launches = 0, n_fused_launches = 0, n_tc_launches = 0, n_tc_tiles = 0;
    double tc_flops = 0;    // TF32 flops the tensor cores execute (every MMA of every tile)
    double work_flops = 0;  // flops the SIMT kernels execute (full tiles, explicit zeros)
};

// Per front-size bucket choices of the factorization: the autotuner's table.
// A panel bucket is (floor(log2 m), floor(log2 k)) of a front (m rows, k
// pivots), a Schur bucket (floor(log2 (m - k)), floor(log2 k)), each packed
// as 32 * first + second.  A bucket missing from the table takes the built-in rule.
struct FactorChoice {
    std::map<int32_t, uint8_t> panel;  // 1: whole panel in one CTA of the per-level kernel; 0: block-step chain
    std::map<int32_t, uint8_t> schur;  // 1: tensor-core Schur complement (mixed precision); 0: SIMT
    int dag = 0;                       // 1: levels below the first tensor-core level in one dependency-driven launch
    int force_panel = 0;               // 1 every front tiled, 2 every front fused (tests, tuning)
    int force_schur = 0;               // 1 SIMT everywhere, 2 tensor cores wherever legal
    bool fused(int64_t m, int64_t k) const;
    bool schur_tc(int64_t m, int64_t k) const;
};
int32_t panel_bucket(int64_t m, int64_t k);
int32_t schur_bucket(int64_t m, int64_t k);
bool rule_fused(int64_t m, int64_t k);
bool rule_schur_tc(int64_t m, int64_t k);
bool wide_front(bool tensor_cores, int64_t m, int64_t k);
bool schur_tc_legal(bool tensor_cores, int64_t m, int64_t k);
bool fused_legal(int64_t m, int64_t k);

// markers: insert a timing marker before every (bucket, level) group, each
// group launched on its own (the autotuner's plans)
void build_factor_plan(const Symbolic& S, FactorPlan& F, bool tensor_cores, const FactorChoice& ch, bool markers);
cudaError_t factor_kernel_setup();
cudaError_t solve_kernel_setup();

struct SolvePlan {
    std::vector<int32_t> fwd_items;  // pairs (supernode, row chunk)
    std::vector<int32_t> bwd_items;  // pairs (supernode, column chunk)
    std::vector<Launch> fwd_launches; // kind 4, bottom-up
    std::vector<Launch> bwd_launches; // kinds 5 (level init) and 6 (block steps), top-down
    std::vector<std::vector<Launch>> bwd_level_launches;
    std::vector<DagTask> dag;  // both sweeps as tasks of one dependency-driven launch; counters:
                               // [0, ns) forward tasks done, [ns, 2 ns) children's forward tasks
                               // done, [2 ns, 3 ns) backward tasks done
};

// batch: bands per launch (the fused per-level sweeps are used for batches only);
// wide: per supernode, 1 = steps of 128 columns with the inverted diagonal tiles of
// the mixed form (launch kinds 15 and 16; such a plan is run with FP32 panels)
void build_solve_plan(const Symbolic& S, SolvePlan& P, int batch, const uint8_t* wide = nullptr);
void build_solve_dag(const Symbolic& S, SolvePlan& P);
// both sweeps in one dependency-driven launch; counters: nb * cstride + 1 ints, zeroed before
void launch_solve_dag(const DevSym& d, const DagTask* tasks, int ntasks, int* counters, int cstride, const double* L,
                      const double* D, double* w, double* z, double* x, DevStatus* status, int nb, const Strides& bs,
                      int wait_limit, int grid, cudaStream_t st, const float* L32 = nullptr);
cudaError_t solve_dag_grid(int* grid);
// variances from unpruned forward solves (the pruning ablation of spi_diag_inverse)
void launch_zsq_var(int32_t n, const double* z, const double* dinv, int R, double* out, cudaStream_t st);
void launch_reciprocal(int32_t n, const double* D, double* dinv, cudaStream_t st);
// variances with the factor's first-order error removed (spi_diag_inverse_refined)
void launch_set_units(int32_t n, const int32_t* pos, int R, double* w, cudaStream_t st);
void launch_refined_var(int32_t n, const double* v, const double* r, const int32_t* idx, int R, double* out,
                        cudaStream_t st);

struct DevDiagPlan {
    int32_t B = 0, nblocks = 0;
    int64_t nrhs = 0;
    int32_t *order = nullptr, *blk_ptr = nullptr, *uptr = nullptr, *us = nullptr, *ulo = nullptr,
            *uhi = nullptr, *uzoff = nullptr, *rel = nullptr, *rhs_out = nullptr, *rhs_zrow = nullptr,
            *rhs_col = nullptr;
    int64_t *urel = nullptr, *zbase = nullptr;
    double* Z = nullptr;
    int64_t zsize = 0;
    // spi_inverse_block plans: pivot of each row of the gathered matrix, and
    // the gathered row of each block-local Z row (concatenated by block)
    int32_t* zpiv = nullptr;
    int32_t* rowmap = nullptr;
    double flops = 0, work_flops = 0;
    double tc_flops = 0;  // TF32 MMA flops of the tensor-core variance kernel on this plan
    std::vector<void*> allocs;
};

// ---- kernel launchers (factor.cu)
// The factorization's panels L and update areas F22 hold double in the FP64
// form and float in the mixed form (void* below); D is always FP64, DS is D
// in the panels' type (the same array as D in the FP64 form).
void launch_assemble(const DevSym& d, const int64_t* amap, const double* vals, int64_t nnz, void* L, bool mixed,
                     const int32_t* diag_src, double* adiag, int nb, const Strides& bs, cudaStream_t st);
void launch_factor_step(const DevSym& d, const Launch& l, const int32_t* items, void* L, void* F22, double* D,
                        void* DS, const double* adiag, DevStatus* status, bool mixed, int nb, const Strides& bs,
                        int wait_limit, cudaStream_t st);
void launch_to_f64(const float* a, double* b, int64_t n, cudaStream_t st);
// the dependency-driven kernel over `tasks`; counters: nb * cstride + 1 ints, zeroed before
void launch_factor_dag(const DevSym& d, const DagTask* tasks, int ntasks, int* counters, int cstride, void* L,
                       void* F22, double* D, void* DS, const double* adiag, DevStatus* status, bool mixed, int nb,
                       const Strides& bs, int wait_limit, cudaStream_t st);
// ---- solve.cu
void launch_permute_in(int32_t n, const int32_t* perm, const double* b, double* w, int nb, cudaStream_t st);
void launch_permute_out(int32_t n, const int32_t* perm, const double* w, double* x, int nb, cudaStream_t st);
// L32: the mixed form's FP32 panels (read instead of L, the same values), or null
// The inverted 128 x 128 diagonal tiles of the mixed form's tensor-core supernodes, for the
// solve's wide steps (launch kinds 15 and 16).
struct WideArgs {
    const float* xinv = nullptr;   // [bands][tiles][128 x 128], row-major
    const int32_t* xptr = nullptr; // [ns] first tile of each supernode
    int64_t xband = 0;             // floats per band
};
void launch_solve_step(const DevSym& d, const Launch& l, const int32_t* fwd_items, const int32_t* bwd_items,
                       const double* L, const double* D, double* w, double* z, double* x, int nb,
                       const Strides& bs, cudaStream_t st, const float* L32 = nullptr,
                       const WideArgs* wa = nullptr);
void launch_sym_residual(int32_t n, const int64_t* cp, const int32_t* ri, const double* va, const double* x,
                         double* r, int nb, int64_t nnz, cudaStream_t st);
void launch_norms2(int32_t n, const double* a, const double* b, double* out, int nb, cudaStream_t st);
void launch_axpy(int32_t n, const double* dx, double* x, int nb, cudaStream_t st);
// ---- diag.cu
void launch_diag_inverse(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D, double* out,
                         int nb, const Strides& bs, size_t smem_min, cudaStream_t st);
// skip: supernodes left to the tensor-core kernel (null: none)
void launch_diag_inverse_f32(const DevSym& d, const DevDiagPlan& p, const float* L, const double* D, double* out,
                             int nb, const Strides& bs, size_t smem_min, const uint8_t* skip, cudaStream_t st);
// out[dst[e]] = G[src[e]] for e < cnt (entries picked from a block of the inverse)
void launch_pick_entries(const double* G, const int64_t* src, const int64_t* dst, int64_t cnt, double* out,
                         cudaStream_t st);
// smem_min: the launches' dynamic shared memory is at least this (0: what they need)
cudaError_t diag_kernel_setup(int B, size_t smem_min);
// (N^-1)(I, I) for the pivots of a plan with zpiv/rowmap: the blocks' forward
// solves (variances to var_scratch), their vectors gathered into Zg (R rows x
// nrhs), then the Gram product into out (ldo = leading dimension, positions
// from the plan's rhs_out).
void launch_inverse_block(const DevSym& d, const DevDiagPlan& p, const double* L, const double* D,
                          double* var_scratch, double* Zg, int64_t R, double* out, int64_t ldo, cudaStream_t st);

// ---- diag_tc.cu: the mixed form's variances on the tensor cores for the
// supernodes with at least min_k pivots and their ancestors
struct DevDiagTc {
    int32_t ntc = 0;
    int64_t npt = 0, ndt = 0;
    int bands = 0;                // bands the buffers hold
    uint8_t* tc = nullptr;
    int64_t* tptr = nullptr;
    int32_t *xptr = nullptr, *ptiles = nullptr, *dtiles = nullptr;
    float* xinv = nullptr;        // [bands][ndt][128 x 128] inverses of the diagonal tiles
    float* pack = nullptr;        // [bands][npt][hi, lo][128 x 32] packed left operands
    alignas(64) unsigned char tmap[128];  // CUtensorMap over pack
    std::vector<void*> allocs;
};
cudaError_t diag_tc_setup();
size_t diag_tc_pack_floats(int64_t npt);
size_t diag_tc_xinv_floats(int64_t ndt);
cudaError_t diag_tc_tensor_map(float* pack, int64_t npt, int bands, void* map_out);
// the left operands from the FP32 panels of nb bands (once per factorization)
void launch_diag_tc_pack(const DevSym& d, const DevDiagTc& p, const float* L32, int nb, const Strides& bs,
                         cudaStream_t st);
// after launch_diag_inverse_f32 with skip = p.tc on the same plan and outputs
void launch_diag_inv_tc(const DevSym& d, const DevDiagPlan& dp, const DevDiagTc& p, const double* D, double* out,
                        int nb, const Strides& bs, DevStatus* status, int wait_limit, cudaStream_t st);

// ---- normal.cu: N = H^T W H and b = H^T W y on the device
struct NormalArgs {
    const int64_t* rowptr;      // H's CSR row pointers [nrows + 1]
    const int32_t* colind;      // H's column indices (caller numbering)
    const int32_t* ent_pos;     // per entry of H: its column's index in its group's union
    const int64_t* grp_row;     // [ngroups + 1] row ranges
    const int64_t* grp_colptr;  // [ngroups + 1] into grp_cols
    const int32_t* grp_cols;    // each group's column union, ascending
    const int64_t* cp;          // N's pattern (caller numbering, lower CSC)
    const int32_t* ri;
    const int64_t* pairptr;     // [ngroups]: start of each group's pair table, or null
    const int32_t* pairpos;     // position in N of pair (a, b), b-major, -1 if absent; or null
};
size_t normal_smem_bytes(int32_t max_dense_entries, int32_t max_rows, int32_t max_cols);
cudaError_t normal_kernel_setup(size_t smem);
// bw: per-row coefficients of b = H^T bw (null: w * y)
void launch_normal(const NormalArgs& a, const int32_t* groups, int32_t ngroups, const double* hv, const double* w,
                   const double* y, const double* bw, const uint8_t* mark, bool zero_pass, double* nv, double* bv,
                   int* flag, size_t smem, cudaStream_t st);
void launch_spmv_rows(int64_t nrows, const int64_t* rowptr, const int32_t* colind, const double* hv, const double* x,
                      double* e, cudaStream_t st);
void launch_mle_rows(int64_t nrows, const double* e, const double* y, double* w, double* v, double* acc,
                     cudaStream_t st);
void launch_step(int32_t n, const double* x, const double* dx, double t, double* xt, cudaStream_t st);
// Algorithm 1 (the empty-field pattern): background entries, the pattern's sums
// and statistic, the pattern update
void launch_bg_locate(int64_t nrows, const int64_t* rowptr, const int32_t* colind, int32_t k0, const int32_t* upat,
                      int32_t npat, int64_t* bgpos, int* flag, cudaStream_t st);
void launch_bg_write(int64_t nrows, const int64_t* bgpos, const int32_t* upat, const double* t, const double* U,
                     double* hv, cudaStream_t st);
void launch_bg_sums(bool mle, int64_t nrows, const int64_t* rowptr, const int32_t* colind, const double* hv,
                    const double* x, int32_t k0, const int64_t* bgpos, const int32_t* upat, const double* t,
                    const double* y, const double* w, int32_t npat, double* sums, double* acc, cudaStream_t st);
void launch_bg_pattern(int32_t npat, const double* sums, double* U, cudaStream_t st);

// Sums over the 32 lanes of a warp of each of v[0..31]: lane j returns the sum of v[j].
// Recursive halving: at distance h every lane keeps the half of its values whose index
// has bit h equal to its own, adds its partner's copy of that half and sends the other
// half (31 shuffles for the 32 sums).  v is overwritten.
template <typename T>
__device__ __forceinline__ T lane_sums(T (&v)[32], int lane) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const T send = up ? v[i] : v[i + h];
            const T keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

}  // namespace spi
