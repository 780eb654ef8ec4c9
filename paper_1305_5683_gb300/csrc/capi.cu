// capi.cu -- the extern "C" entry points declared in include/spi.h.
//
// A context owns the host symbolic analysis of one pattern and every device
// buffer.  Device memory is laid out once, at the first factorization, for
// `opt.batch` same-pattern bands (band b of every per-band buffer starts at
// b * stride):
//   panels L (sum_s m_s k_s doubles, column-major per supernode), D (n),
//   F22 update areas (sum over supernodes with children of (m-k)^2), the
//   input values, the solve vectors, the symbolic arrays and launch item
//   lists (shared by all bands), and per-plan Z workspaces of the variance
//   solves (rows of the union of a block's paths x B, per band).
// Single-problem calls are the batch-1 case of the batched calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "spi_internal.cuh"

using namespace spi;

struct spi_ctx {
    Symbolic S;
    spi_options opt{};
    FactorPlan FP;
    SolvePlan SP;
    int device = -1;
    bool dev_ready = false, factored = false;
    int factored_nb = 0;
    std::vector<void*> allocs;
    int64_t device_bytes = 0;
    DevSym dsym;
    Strides bs;
    int64_t* d_amap = nullptr;
    int32_t *d_diag_src = nullptr, *d_fwd_items = nullptr, *d_bwd_items = nullptr;
    // the factorization's launch items on the device (per plan: the autotuner's plans have their own)
    struct DevFactorPlan {
        int32_t* items[15] = {};  // by launch kind
        DagTask* dag = nullptr;   // the dependency-driven kernel's tasks
        int* counters = nullptr;  // its counters: opt.batch x 2 ns, then the work counter
        std::vector<void*> allocs;
    } dfp;
    bool factor_plan_ready = false;  // c->FP is final (tuned or by rule) and uploaded
    FactorChoice choice;             // the bucket table behind c->FP
    int tune_source = 0;             // 0 built-in rules, 1 timed here, 2 read from the tune cache
    double tune_seconds = 0;
    int64_t tune_panel_buckets = 0, tune_panel_fused = 0, tune_schur_buckets = 0, tune_schur_tc = 0;
    double tune_dag_ms[2] = {-1.0, -1.0};  // timed factorization: launches per level / dependency-driven
    // the solve's dependency-driven form: tasks, counters, grid; whether it is in use
    // (-1: not decided yet), and its timing against the per-level launches
    DagTask* d_solve_dag = nullptr;
    int* d_solve_cnt = nullptr;
    int solve_dag_grid_size = 1;
    int solve_dag = -1;
    double tune_solve_ms[2] = {-1.0, -1.0};
    std::map<int, cudaGraphExec_t> g_solve_dag;
    // symmetric indefinite factorizations (spi_options.pivoting): the analysis parameters
    // (re-analysed with forced merges when a front's pivots are delayed), the pivoting
    // outputs, and the solve structure in the pivots' final order
    AnalyseParams prm;
    bool piv_ready = false;
    Symbolic S_sol;
    DevSym dsym_sol;
    double *d_Dd = nullptr, *d_Doff = nullptr, *d_dinv_a = nullptr, *d_dinv_b = nullptr;
    int32_t *d_pair = nullptr, *d_lperm = nullptr, *d_pair_sol = nullptr, *d_srows_sol = nullptr,
            *d_perm_sol = nullptr, *d_fdesc_sol = nullptr;
    int* d_delay = nullptr;
    int64_t piv_2x2 = 0, piv_delays = 0, piv_restarts = 0;
    double *d_L = nullptr, *d_F22 = nullptr, *d_D = nullptr, *d_adiag = nullptr, *d_vals = nullptr,
           *d_w = nullptr, *d_z = nullptr, *d_xp = nullptr, *d_vec = nullptr, *d_out = nullptr;
    DevStatus* d_status = nullptr;
    DevStatus* h_status = nullptr;
    // mixed precision: FP32 copy of the panels, the input pattern for the FP64 residual
    float* d_L32 = nullptr;   // also the working panels of the mixed factorization
    float* d_F22f = nullptr;  // mixed form: FP32 update areas
    float* d_Df = nullptr;    // mixed form: D in FP32 (scaling in the update kernels)
    int64_t* d_cp = nullptr;
    int32_t* d_ri = nullptr;
    double *d_b2 = nullptr, *d_x = nullptr, *d_r = nullptr, *d_dx = nullptr, *d_norm = nullptr, *h_norm = nullptr;
    int64_t refine_steps = 0;
    int64_t refine_planned = -1;  // correction steps the last converged solve took (-1: none yet)
    double solve_relres = 0;
    // CUDA graphs of the launch sequences that touch only context buffers, per band count
    cudaStream_t cap = nullptr;
    std::map<int, cudaGraphExec_t> g_factor, g_solve;
    // variance plans: all indices, and the last index subset
    DevDiagPlan plan_all;
    bool plan_all_ready = false;
    DevDiagPlan plan_sub;
    std::vector<int32_t> plan_sub_key;
    bool plan_sub_ready = false;
    // spi_inverse_block: its single-block plan (cached per index set) and output scratch
    DevDiagPlan plan_blk;
    std::vector<int32_t> plan_blk_key;
    bool plan_blk_ready = false;
    double* d_blk = nullptr;
    double* d_zg = nullptr;      // gathered vectors (rows of the paths' union x indices)
    double* d_mle = nullptr;     // spi_mle_newton: x, trial x, step, rhs, e, w, v, sums
    int64_t mle_steps = 0;       // spi_mle_newton: steps and final Cash statistic
    double mle_cash = 0.0;
    struct Background {          // spi_background_fit: each row's background entry, copies of
        int64_t* pos = nullptr;  // the pattern indices and t, the patterns, sums and previous x
        int32_t* pat = nullptr;
        double* vec = nullptr;
    } bg;
    int64_t bg_iters = 0;        // spi_background_fit: solves and the returned statistic
    double bg_stat = 0.0;
    // spi_normal_*: the design matrix's row groups (host and device) and scratch
    struct Normal {
        bool ready = false;
        int64_t nrows = 0, nnzh = 0;
        int32_t ngroups = 0;
        size_t smem = 0;
        std::vector<int64_t> grp_row;
        std::vector<int32_t> row_grp;
        std::vector<int64_t> hcp;  // H's pattern by columns: rows of each column
        std::vector<int32_t> hri;
        NormalArgs args{};
        int32_t *d_groups = nullptr, *d_sel = nullptr, *d_flag = nullptr;
        uint8_t* d_mark = nullptr;
        double *d_hv = nullptr, *d_w = nullptr, *d_y = nullptr, *d_nv = nullptr, *d_b = nullptr;
    } nrm;
    int64_t zg_cap = 0, blk_rows = 0;
    size_t diag_smem_pad = 0;  // dynamic shared memory of a variance CTA at least this (diag_ctas_per_sm)
    int rhs_block_used = 0;
    double last_diag_flops = 0, last_diag_work = 0;
    // variances of the mixed form on the tensor cores (the supernodes with at least
    // diag_tc_min_pivots pivots and their ancestors)
    DiagTcHost dtc_h;
    DevDiagTc dtc;
    double last_diag_tc_flops = 0;
    // the mixed solve's plan with 128-column steps for those supernodes (their inverted
    // diagonal tiles); the FP64-panel paths keep SP
    SolvePlan SPw;
    int32_t *d_fwd_items_w = nullptr, *d_bwd_items_w = nullptr;
    WideArgs wa;
    bool wide_ready = false;
    int64_t bad_pivot = -1, bad_band = -1;
    std::vector<int64_t> in_colptr;  // kept until the device copy exists (mixed precision)
    std::vector<int32_t> in_rowind;
    double analyse_seconds = 0;
    std::string tune_cache_path;  // the caller's spi_options.tune_cache, copied
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SPI_ERR_OOM : SPI_ERR_CUDA; }

// symmetric indefinite form: fronts recorded per factorization as unable to pivot,
// and factorizations retried after merging them into their parents
constexpr int kMaxDelay = 4096;
constexpr int kMaxRestarts = 256;

// The structure the solves and variances use: in the pivots' final order after a
// symmetric indefinite factorization, else the analysis itself.
const Symbolic& sym_sol(const spi_ctx* c) { return c->piv_ready ? c->S_sol : c->S; }
const DevSym& dev_sol(const spi_ctx* c) { return c->piv_ready ? c->dsym_sol : c->dsym; }

template <class T>
cudaError_t dev_alloc(spi_ctx* c, T** p, size_t count, std::vector<void*>* track = nullptr) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e == cudaSuccess) {
        (track ? *track : c->allocs).push_back(*p);
        c->device_bytes += (int64_t)(count * sizeof(T));
    }
    return e;
}

template <class T>
cudaError_t dev_upload(spi_ctx* c, T** p, const std::vector<T>& v, std::vector<void*>* track = nullptr) {
    cudaError_t e = dev_alloc(c, p, v.size(), track);
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

#define CK(x)                                            \
    do {                                                 \
        cudaError_t e__ = (x);                           \
        if (e__ != cudaSuccess) return cuda_fail(e__);   \
    } while (0)

bool mixed_of(const spi_ctx* c) { return c->opt.precision == SPI_PREC_MIXED_FP32; }

int ensure_device(spi_ctx* c) {
    if (c->dev_ready) return SPI_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return SPI_ERR_CUDA;
    CK(cudaGetDevice(&c->device));
    const Symbolic& S = c->S;
    const size_t nb = (size_t)c->opt.batch;
    int32_t *sfirst, *srows, *relmap, *sparent, *perm, *snode_of, *fdesc;
    int64_t *srowptr, *lptr, *f22ptr;
    CK(dev_upload(c, &sfirst, S.sfirst));
    CK(dev_upload(c, &srowptr, S.srowptr));
    CK(dev_upload(c, &srows, S.srows));
    CK(dev_upload(c, &relmap, S.relmap));
    CK(dev_upload(c, &sparent, S.sparent));
    CK(dev_upload(c, &lptr, S.lptr));
    CK(dev_upload(c, &f22ptr, S.f22ptr));
    CK(dev_upload(c, &perm, S.perm));
    CK(dev_upload(c, &snode_of, S.snode_of));
    CK(dev_upload(c, &fdesc, S.fdesc));
    c->dsym = DevSym{S.n, S.ns, sfirst, srowptr, srows, relmap, sparent, lptr, f22ptr, perm, snode_of, fdesc};
    c->bs.L = S.lptr[S.ns];
    c->bs.F22 = S.f22_total;
    c->bs.n = S.n;
    c->bs.Dn = S.n;
    c->bs.nnz = S.nnz_a;
    CK(dev_upload(c, &c->d_amap, S.amap));
    CK(dev_upload(c, &c->d_diag_src, S.diag_src));
    CK(dev_upload(c, &c->d_fwd_items, c->SP.fwd_items));
    CK(dev_upload(c, &c->d_bwd_items, c->SP.bwd_items));
    CK(dev_upload(c, &c->d_solve_dag, c->SP.dag));
    CK(dev_alloc(c, &c->d_solve_cnt, nb * 3 * (size_t)S.ns + 1));
    CK(solve_dag_grid(&c->solve_dag_grid_size));
    if (c->opt.dag == 1) c->solve_dag = 0;
    if (c->opt.dag == 2) c->solve_dag = 1;
    CK(dev_alloc(c, &c->d_L, (size_t)S.lptr[S.ns] * nb));
    if (!mixed_of(c)) CK(dev_alloc(c, &c->d_F22, (size_t)S.f22_total * nb));
    CK(dev_alloc(c, &c->d_D, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_adiag, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_vals, (size_t)S.nnz_a * nb));
    CK(dev_alloc(c, &c->d_w, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_z, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_xp, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_vec, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_out, (size_t)S.n * nb));
    CK(dev_alloc(c, &c->d_status, 1));
    CK(cudaMallocHost((void**)&c->h_status, sizeof(DevStatus)));
    CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    if (mixed_of(c)) {
        CK(dev_alloc(c, &c->d_L32, (size_t)S.lptr[S.ns] * nb));
        CK(dev_alloc(c, &c->d_F22f, (size_t)S.f22_total * nb));
        CK(dev_alloc(c, &c->d_Df, (size_t)S.n * nb));
        if (!c->d_cp) CK(dev_upload(c, &c->d_cp, c->in_colptr));
        if (!c->d_ri) CK(dev_upload(c, &c->d_ri, c->in_rowind));
        CK(dev_alloc(c, &c->d_b2, (size_t)S.n * nb));
        CK(dev_alloc(c, &c->d_x, (size_t)S.n * nb));
        CK(dev_alloc(c, &c->d_r, (size_t)S.n * nb));
        CK(dev_alloc(c, &c->d_dx, (size_t)S.n * nb));
        CK(dev_alloc(c, &c->d_norm, 2 * nb));
        CK(cudaMallocHost((void**)&c->h_norm, 2 * nb * sizeof(double)));
    }
    if (c->opt.pivoting) {
        CK(dev_alloc(c, &c->d_Dd, (size_t)S.n));
        CK(dev_alloc(c, &c->d_Doff, (size_t)S.n));
        CK(dev_alloc(c, &c->d_pair, (size_t)S.n));
        CK(dev_alloc(c, &c->d_lperm, (size_t)S.n));
        CK(dev_alloc(c, &c->d_delay, (size_t)kMaxDelay + 2));
        CK(dev_alloc(c, &c->d_dinv_a, (size_t)S.n));
        CK(dev_alloc(c, &c->d_dinv_b, (size_t)S.n));
        CK(dev_alloc(c, &c->d_pair_sol, (size_t)S.n));
        CK(dev_alloc(c, &c->d_perm_sol, (size_t)S.n));
        CK(dev_alloc(c, &c->d_srows_sol, S.srows.size()));
        CK(dev_alloc(c, &c->d_fdesc_sol, (size_t)S.n));
    }
    if (c->opt.diag_ctas_per_sm > 0) {  // pad the variance kernels' shared memory: at most k per SM
        int dev = 0, per_sm = 0, reserved = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        CK(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int k = c->opt.diag_ctas_per_sm;
        size_t pad = (size_t)(per_sm / (k + 1) - reserved + 128);
        pad = (pad + 127) & ~(size_t)127;
        // k + 1 CTAs of pad + reserved bytes exceed the SM; k still fit
        if ((int64_t)k * (int64_t)(pad + reserved) <= per_sm) c->diag_smem_pad = pad;
    }
    CK(diag_kernel_setup(512, c->diag_smem_pad));
    CK(factor_kernel_setup());
    CK(solve_kernel_setup());
    if (mixed_of(c) && !c->opt.pivoting && c->opt.diag_tc_min_pivots >= 0) {
        build_diag_tc(S, c->opt.diag_tc_min_pivots > 0 ? c->opt.diag_tc_min_pivots : kDiagTcMinPivots, c->dtc_h);
        DevDiagTc& t = c->dtc;
        t = DevDiagTc();
        if (c->dtc_h.ntc > 0) {
            const DiagTcHost& h = c->dtc_h;
            CK(dev_upload(c, &t.tc, h.tc));
            CK(dev_upload(c, &t.tptr, h.tptr));
            CK(dev_upload(c, &t.xptr, h.xptr));
            CK(dev_upload(c, &t.ptiles, h.ptiles));
            CK(dev_upload(c, &t.dtiles, h.dtiles));
            CK(dev_alloc(c, &t.xinv, diag_tc_xinv_floats(h.ndt) * nb));
            CK(dev_alloc(c, &t.pack, diag_tc_pack_floats(h.npt) * nb));
            CK(diag_tc_tensor_map(t.pack, h.npt, (int)nb, t.tmap));
            CK(diag_tc_setup());
            t.ntc = h.ntc;
            t.npt = h.npt;
            t.ndt = h.ndt;
            t.bands = (int)nb;
            build_solve_plan(S, c->SPw, c->opt.batch, h.tc.data());
            CK(dev_upload(c, &c->d_fwd_items_w, c->SPw.fwd_items));
            CK(dev_upload(c, &c->d_bwd_items_w, c->SPw.bwd_items));
            c->wa = WideArgs{t.xinv, t.xptr, (int64_t)diag_tc_xinv_floats(h.ndt)};
            c->wide_ready = true;
        }
    }
    c->dev_ready = true;
    return SPI_OK;
}

void free_plan(DevDiagPlan& p) {
    for (void* a : p.allocs) cudaFree(a);
    p = DevDiagPlan();
}

int upload_plan(spi_ctx* c, const DiagPlan& h, DevDiagPlan& d) {
    free_plan(d);
    d.B = h.B; d.nblocks = h.nblocks; d.nrhs = h.nrhs; d.flops = h.flops; d.work_flops = h.work_flops;
    d.tc_flops = c->dtc.ntc > 0 && h.B <= kDiagTcMaxBlock ? diag_tc_mma_flops(sym_sol(c), c->dtc_h, h) : 0.0;
    std::vector<void*>* tr = &d.allocs;
    CK(dev_upload(c, &d.order, h.order, tr));
    CK(dev_upload(c, &d.blk_ptr, h.blk_ptr, tr));
    CK(dev_upload(c, &d.uptr, h.uptr, tr));
    CK(dev_upload(c, &d.us, h.us, tr));
    CK(dev_upload(c, &d.ulo, h.ulo, tr));
    CK(dev_upload(c, &d.uhi, h.uhi, tr));
    CK(dev_upload(c, &d.uzoff, h.uzoff, tr));
    CK(dev_upload(c, &d.rel, h.rel, tr));
    CK(dev_upload(c, &d.rhs_out, h.rhs_out, tr));
    CK(dev_upload(c, &d.rhs_zrow, h.rhs_zrow, tr));
    CK(dev_upload(c, &d.rhs_col, h.rhs_col, tr));
    CK(dev_upload(c, &d.urel, h.urel, tr));
    CK(dev_upload(c, &d.zbase, h.zbase, tr));
    d.zsize = h.zbase.empty() ? 0 : h.zbase.back();
    // FP64 elements per band are enough for both element types
    CK(dev_alloc(c, &d.Z, (size_t)std::max<int64_t>(d.zsize, 1) * (size_t)c->opt.batch, tr));
    return SPI_OK;
}

// Record `body(stream)` once into a CUDA graph and replay it on `st`; if the
// capture fails, run the launches directly on `st`.
template <class F>
cudaError_t run_graph(spi_ctx* c, std::map<int, cudaGraphExec_t>& cache, int key, cudaStream_t st, F&& body) {
    auto it = cache.find(key);
    if (it == cache.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            body(c->cap);
            e = cudaStreamEndCapture(c->cap, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            body(st);
            return cudaGetLastError();
        }
        it = cache.emplace(key, exec).first;
    }
    return cudaGraphLaunch(it->second, st);
}

__global__ void k_reset_status(DevStatus* s) {
    s->flags = 0;
    s->bad_pivot = INT_MAX;
}

int finish(spi_ctx* c, cudaStream_t st) {
    CK(cudaGetLastError());
    if (c->opt.async) return SPI_OK;
    CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (c->h_status->flags & FLAG_NOT_SPD) {
        const int64_t bp = c->h_status->bad_pivot, n = c->S.n;
        if (bp >= 0 && n > 0 && bp < n * c->opt.batch) {
            c->bad_band = bp / n;
            c->bad_pivot = c->S.perm[bp % n];
        }
        c->factored = false;
        return SPI_ERR_NOT_SPD;
    }
    if (c->h_status->flags & FLAG_TIMEOUT) {
        c->factored = false;
        return SPI_ERR_TIMEOUT;
    }
    return SPI_OK;
}

void free_factor_plan(spi_ctx::DevFactorPlan& d) {
    for (void* a : d.allocs) cudaFree(a);
    d = spi_ctx::DevFactorPlan();
}

int upload_factor_plan(spi_ctx* c, const FactorPlan& F, spi_ctx::DevFactorPlan& d) {
    free_factor_plan(d);
    std::vector<void*>* tr = &d.allocs;
    CK(dev_upload(c, &d.items[0], F.diag_items, tr));
    CK(dev_upload(c, &d.items[1], F.trsm_items, tr));
    CK(dev_upload(c, &d.items[2], F.schur_items, tr));
    CK(dev_upload(c, &d.items[3], F.update_items, tr));
    CK(dev_upload(c, &d.items[7], F.schur_tc_items, tr));
    CK(dev_upload(c, &d.items[8], F.dfront_items, tr));
    CK(dev_upload(c, &d.items[9], F.panel_tc_items, tr));
    CK(dev_upload(c, &d.items[12], F.fused_items, tr));
    CK(dev_upload(c, &d.items[14], F.bk_items, tr));
    if (!F.dag.empty()) {
        CK(dev_upload(c, &d.dag, F.dag, tr));
        CK(dev_alloc(c, &d.counters, (size_t)c->opt.batch * 2 * (size_t)c->S.ns + 1, tr));
    }
    return SPI_OK;
}

// Zeroed panels and update areas, then the input values scattered into the
// fronts, on s2 (launched on every call: the values' address changes).
cudaError_t factor_assemble(spi_ctx* c, int nb, const double* vals, cudaStream_t s2) {
    const Symbolic& S = c->S;
    const bool mixed = mixed_of(c);
    void* Lw = mixed ? (void*)c->d_L32 : (void*)c->d_L;
    void* Fw = mixed ? (void*)c->d_F22f : (void*)c->d_F22;
    const size_t esz = mixed ? sizeof(float) : sizeof(double);
    cudaError_t e = cudaMemsetAsync(Lw, 0, (size_t)S.lptr[S.ns] * nb * esz, s2);
    if (e == cudaSuccess && S.f22_total) e = cudaMemsetAsync(Fw, 0, (size_t)S.f22_total * nb * esz, s2);
    if (e != cudaSuccess) return e;
    launch_assemble(c->dsym, c->d_amap, vals, S.nnz_a, Lw, mixed, c->d_diag_src, c->d_adiag, nb, c->bs, s2);
    return cudaGetLastError();
}

// Every launch of plan F on s2 (a timing marker records evs[group]).
void factor_launches(spi_ctx* c, int nb, const FactorPlan& F, const spi_ctx::DevFactorPlan& dp, cudaStream_t s2,
                     const std::vector<cudaEvent_t>* evs) {
    const bool mixed = mixed_of(c);
    void* Lw = mixed ? (void*)c->d_L32 : (void*)c->d_L;
    void* Fw = mixed ? (void*)c->d_F22f : (void*)c->d_F22;
    void* DS = mixed ? (void*)c->d_Df : (void*)c->d_D;
    for (const Launch& l : F.launches) {
        if (l.kind < 0) {
            if (evs) cudaEventRecord((*evs)[(size_t)l.step], s2);
            continue;
        }
        if (l.kind == 14) {
            BkArgs a{c->d_Dd, c->d_Doff, c->d_pair, c->d_lperm, c->d_delay, kMaxDelay,
                     c->d_delay + 1 + kMaxDelay};
            launch_front_bk(c->dsym, dp.items[14] + l.off, l.count, c->d_L, c->d_F22, a, c->d_status, s2);
            continue;
        }
        if (l.kind == 13) {
            const int cstride = 2 * c->S.ns;
            cudaMemsetAsync(dp.counters, 0, ((size_t)nb * cstride + 1) * sizeof(int), s2);
            launch_factor_dag(c->dsym, dp.dag, l.count, dp.counters, cstride, Lw, Fw, c->d_D, DS, c->d_adiag,
                              c->d_status, mixed, nb, c->bs, c->opt.wait_limit, s2);
            continue;
        }
        launch_factor_step(c->dsym, l, dp.items[l.kind], Lw, Fw, c->d_D, DS, c->d_adiag, c->d_status, mixed, nb,
                           c->bs, c->opt.wait_limit, s2);
    }
}

// ---------------------------------------------------------------------------
// Autotuner of the factorization (tile path per front-size bucket).
//
// Two plans are built in which every bucket takes one candidate: all panels
// on the block-step chain with SIMT Schur complements, and all panels in the
// persistent per-level kernel with tensor-core Schur complements wherever
// legal.  In both, each (bucket, level) group is launched on its own between
// timing markers.  Each plan is recorded as a CUDA graph (with its event
// nodes), replayed twice on the caller's values, and the second replay's
// group times are summed per bucket; every bucket keeps its faster candidate.
// The table can be kept in a text file (spi_options.tune_cache), one line
// per bucket: device, precision, batch class, P (panel) or S (Schur), bucket,
// choice, milliseconds of the two candidates.  The same file keeps the other
// timed choices, one line each: D (one dependency-driven factor launch or
// launches level by level), V (the same for the solve) and B (the variance
// right-hand-side block).

std::string tune_key(spi_ctx* c, int nb) {
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) dev = prop.name;
    for (char& ch : dev)
        if (ch == ' ' || ch == '\t') ch = '_';
    return dev + " " + (mixed_of(c) ? "mixed" : "fp64") + " " + (nb > 1 ? "batch" : "single");
}

// The buckets whose choice matters for this tree: panel buckets of fronts that
// may run either way, Schur buckets of fronts that may use the tensor cores.
void tunable_buckets(const spi_ctx* c, std::vector<int32_t>& pb, std::vector<int32_t>& sb) {
    const Symbolic& S = c->S;
    const bool tc = mixed_of(c);
    std::map<int32_t, int> a, b;
    for (int32_t s = 0; s < S.ns; ++s) {
        const int64_t k = S.k_of(s), m = S.m_of(s);
        if (!S.sdiag[s] && !wide_front(tc, m, k) && fused_legal(m, k)) a[panel_bucket(m, k)] = 1;
        if (S.sparent[s] != -1 && m > k && schur_tc_legal(tc, m, k)) b[schur_bucket(m, k)] = 1;
    }
    pb.clear();
    sb.clear();
    for (auto& kv : a) pb.push_back(kv.first);
    for (auto& kv : b) sb.push_back(kv.first);
}

struct TuneLine {
    char kind;
    int32_t bucket;
    int choice;
    double ms0, ms1;
};

void read_tune_cache(const char* path, const std::string& key, std::vector<TuneLine>& out,
                     std::vector<std::string>* other) {
    FILE* fp = path ? std::fopen(path, "r") : nullptr;
    if (!fp) return;
    char buf[512];
    while (std::fgets(buf, sizeof buf, fp)) {
        char dev[256], prec[32], cls[32], kind[8];
        int bucket = 0, choice = 0;
        double a = 0, b = 0;
        if (buf[0] == '#' ||
            std::sscanf(buf, "%255s %31s %31s %7s %d %d %lf %lf", dev, prec, cls, kind, &bucket, &choice, &a, &b) != 8) {
            continue;
        }
        const std::string k = std::string(dev) + " " + prec + " " + cls;
        if (k == key && std::strchr("PSDVB", kind[0]))
            out.push_back(TuneLine{kind[0], bucket, choice, a, b});
        else if (other) other->push_back(buf);
    }
    std::fclose(fp);
}

void write_tune_cache(const char* path, const std::string& key, const std::vector<TuneLine>& lines) {
    if (!path) return;
    std::vector<TuneLine> mine;
    std::vector<std::string> other;
    read_tune_cache(path, key, mine, &other);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* fp = std::fopen(tmp.c_str(), "w");
    if (!fp) return;
    std::fprintf(fp, "# spi autotuner: device precision batch kind bucket choice ms_candidate0 ms_candidate1"
                     " (P panel, S Schur, D dependency-driven factor, V dependency-driven solve, B variance"
                     " right-hand-side block)\n");
    for (const std::string& l : other) std::fputs(l.c_str(), fp);
    for (const TuneLine& t : lines)
        std::fprintf(fp, "%s %c %d %d %.6f %.6f\n", key.c_str(), t.kind, t.bucket, t.choice, t.ms0, t.ms1);
    std::fclose(fp);
    std::rename(tmp.c_str(), path);
}

// Replace this key's lines of the given kinds by `fresh`, keeping every other line.
void tune_cache_update(const char* path, const std::string& key, const char* kinds,
                       const std::vector<TuneLine>& fresh) {
    if (!path) return;
    std::vector<TuneLine> cached, keep;
    read_tune_cache(path, key, cached, nullptr);
    for (const TuneLine& t : cached)
        if (!std::strchr(kinds, t.kind)) keep.push_back(t);
    keep.insert(keep.end(), fresh.begin(), fresh.end());
    write_tune_cache(path, key, keep);
}

// Time one candidate plan: per (kind, bucket), the summed milliseconds.  The
// plan is replayed from a CUDA graph (as the factorization runs); if its
// event nodes cannot be timed, the launches are issued directly instead.
int time_plan(spi_ctx* c, int nb, const double* vals, const FactorChoice& ch, cudaStream_t st,
              std::map<std::pair<int, int32_t>, double>& ms) {
    FactorPlan F;
    build_factor_plan(c->S, F, mixed_of(c), ch, true);
    spi_ctx::DevFactorPlan dp;
    int rc = upload_factor_plan(c, F, dp);
    if (rc) { free_factor_plan(dp); return rc; }
    std::vector<cudaEvent_t> ev(F.groups.size(), nullptr);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { rc = SPI_ERR_CUDA; break; }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph = false;
    if (!rc) {
        graph = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (graph) {
            factor_launches(c, nb, F, dp, c->cap, &ev);
            graph = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        }
        if (!graph) cudaGetLastError();
    }
    std::map<std::pair<int, int32_t>, double> got;
    for (int attempt = graph ? 0 : 1; !rc && attempt < 2; ++attempt) {
        const bool use_graph = attempt == 0;
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            k_reset_status<<<1, 1, 0, st>>>(c->d_status);
            if (factor_assemble(c, nb, vals, st) != cudaSuccess) { rc = SPI_ERR_CUDA; break; }
            if (use_graph) {
                if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = SPI_ERR_CUDA;
            } else {
                factor_launches(c, nb, F, dp, st, &ev);
            }
            if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = SPI_ERR_CUDA;
        }
        if (rc) break;
        got.clear();
        bool timed = true;
        for (size_t q = 0; q + 1 < F.groups.size(); ++q) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[q], ev[q + 1]) != cudaSuccess) { timed = false; break; }
            const FactorPlan::Group& gr = F.groups[q];
            if (gr.kind == FactorPlan::kPanel || gr.kind == FactorPlan::kSchur) got[{gr.kind, gr.bucket}] += t;
        }
        if (timed) break;
        cudaGetLastError();
        if (!use_graph) rc = SPI_ERR_CUDA;  // neither form could be timed
    }
    if (!rc) ms = got;
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    free_factor_plan(dp);
    return rc;
}

// Milliseconds of one factorization with plan F (its launches recorded as a CUDA
// graph, the second of two replays), or a negative value if it could not be timed.
double time_whole_plan(spi_ctx* c, int nb, const double* vals, const FactorPlan& F, cudaStream_t st) {
    spi_ctx::DevFactorPlan dp;
    if (upload_factor_plan(c, F, dp)) { free_factor_plan(dp); return -1.0; }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    double ms = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
              cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        factor_launches(c, nb, F, dp, c->cap, nullptr);
        ok = cudaStreamEndCapture(c->cap, &g) == cudaSuccess && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
    }
    for (int rep = 0; ok && rep < 2; ++rep) {
        k_reset_status<<<1, 1, 0, st>>>(c->d_status);
        ok = factor_assemble(c, nb, vals, st) == cudaSuccess && cudaEventRecord(e0, st) == cudaSuccess &&
             cudaGraphLaunch(exec, st) == cudaSuccess && cudaEventRecord(e1, st) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
        float t = 0.f;
        if (ok && rep == 1 && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t;
    }
    if (!ok) cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    free_factor_plan(dp);
    return ms;
}

// Make c->FP final and upload it: from the tune cache, by timing, or by the
// built-in rules (see spi_options.autotune).
int prepare_factor_plan(spi_ctx* c, int nb, const double* vals, cudaStream_t st) {
    const Symbolic& S = c->S;
    FactorChoice ch;
    ch.force_panel = c->opt.force_panel;
    ch.force_schur = c->opt.force_schur;
    std::vector<int32_t> pb, sb;
    tunable_buckets(c, pb, sb);
    if (ch.force_panel) pb.clear();
    if (ch.force_schur) sb.clear();
    c->tune_source = 0;
    c->tune_seconds = 0;
    if (!pb.empty() || !sb.empty()) {
        const std::string key = tune_key(c, nb);
        std::vector<TuneLine> cached;
        read_tune_cache(c->opt.tune_cache, key, cached, nullptr);
        for (const TuneLine& t : cached) (t.kind == 'P' ? ch.panel : ch.schur)[t.bucket] = (uint8_t)(t.choice != 0);
        bool missing = false;
        for (int32_t b : pb) missing |= !ch.panel.count(b);
        for (int32_t b : sb) missing |= !ch.schur.count(b);
        const bool timing = c->opt.autotune > 0 || (c->opt.autotune == 0 && S.factor_flops >= 2e8);
        if (!missing) {
            c->tune_source = 2;
        } else if (timing) {
            auto t0 = std::chrono::steady_clock::now();
            FactorChoice a = ch, b = ch;
            a.panel.clear(); a.schur.clear(); b.panel.clear(); b.schur.clear();
            a.force_panel = ch.force_panel ? ch.force_panel : 1;
            a.force_schur = ch.force_schur ? ch.force_schur : 1;
            b.force_panel = ch.force_panel ? ch.force_panel : 2;
            b.force_schur = ch.force_schur ? ch.force_schur : 2;
            std::map<std::pair<int, int32_t>, double> ma, mb;
            int rc = time_plan(c, nb, vals, a, st, ma);
            if (!rc) rc = time_plan(c, nb, vals, b, st, mb);
            if (rc) return rc;
            std::vector<TuneLine> lines;
            for (int32_t bk : pb) {
                const double t0a = ma[{FactorPlan::kPanel, bk}], t1 = mb[{FactorPlan::kPanel, bk}];
                ch.panel[bk] = (uint8_t)(t1 < t0a);
                lines.push_back(TuneLine{'P', bk, t1 < t0a ? 1 : 0, t0a, t1});
            }
            for (int32_t bk : sb) {
                const double t0a = ma[{FactorPlan::kSchur, bk}], t1 = mb[{FactorPlan::kSchur, bk}];
                ch.schur[bk] = (uint8_t)(t1 < t0a);
                lines.push_back(TuneLine{'S', bk, t1 < t0a ? 1 : 0, t0a, t1});
            }
            tune_cache_update(c->opt.tune_cache, key, "PS", lines);
            c->tune_source = 1;
            c->tune_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
    }
    c->tune_panel_buckets = (int64_t)pb.size();
    c->tune_schur_buckets = (int64_t)sb.size();
    c->tune_panel_fused = c->tune_schur_tc = 0;
    for (int32_t b : pb) {
        auto it = ch.panel.find(b);
        c->tune_panel_fused += it != ch.panel.end() ? it->second : 0;
    }
    for (int32_t b : sb) {
        auto it = ch.schur.find(b);
        c->tune_schur_tc += it != ch.schur.end() ? it->second : 0;
    }
    // one dependency-driven launch for the levels below the first tensor-core level, or
    // launches level by level: as forced, timed with the table above, cached, or on by rule
    c->tune_dag_ms[0] = c->tune_dag_ms[1] = -1.0;
    if (c->opt.dag == 1 || c->opt.dag == 2) {
        ch.dag = c->opt.dag == 2;
    } else {
        const std::string key = tune_key(c, nb);
        std::vector<TuneLine> cached;
        read_tune_cache(c->opt.tune_cache, key, cached, nullptr);
        int found = -1;
        for (const TuneLine& t : cached)
            if (t.kind == 'D') found = t.choice;
        const bool timing = c->opt.autotune > 0 || (c->opt.autotune == 0 && S.factor_flops >= 2e8);
        if (found >= 0) {
            ch.dag = found;
        } else if (timing) {
            auto t0 = std::chrono::steady_clock::now();
            FactorPlan F0, F1;
            FactorChoice c0 = ch, c1 = ch;
            c0.dag = 0;
            c1.dag = 1;
            build_factor_plan(S, F0, mixed_of(c), c0, false);
            build_factor_plan(S, F1, mixed_of(c), c1, false);
            c->tune_dag_ms[0] = time_whole_plan(c, nb, vals, F0, st);
            c->tune_dag_ms[1] = F1.dag.empty() ? -1.0 : time_whole_plan(c, nb, vals, F1, st);
            ch.dag = c->tune_dag_ms[1] >= 0.0 && c->tune_dag_ms[0] >= 0.0 && c->tune_dag_ms[1] < c->tune_dag_ms[0];
            tune_cache_update(c->opt.tune_cache, key, "D",
                              {TuneLine{'D', 0, ch.dag, c->tune_dag_ms[0], c->tune_dag_ms[1]}});
            c->tune_source = 1;
            c->tune_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        } else {
            ch.dag = 1;
        }
    }
    c->choice = ch;
    build_factor_plan(S, c->FP, mixed_of(c), ch, false);
    for (auto& kv : c->g_factor) cudaGraphExecDestroy(kv.second);
    c->g_factor.clear();
    int rc = upload_factor_plan(c, c->FP, c->dfp);
    if (rc) return rc;
    c->factor_plan_ready = true;
    return SPI_OK;
}

// Every device resource of the context released (before re-planning it for a new
// symbolic structure); the next call sets the device up again.
void reset_device(spi_ctx* c) {
    free_plan(c->plan_all);
    free_plan(c->plan_sub);
    free_plan(c->plan_blk);
    free_factor_plan(c->dfp);
    c->plan_all_ready = c->plan_sub_ready = c->plan_blk_ready = false;
    for (auto* g : {&c->g_factor, &c->g_solve, &c->g_solve_dag}) {
        for (auto& kv : *g) cudaGraphExecDestroy(kv.second);
        g->clear();
    }
    if (c->cap) { cudaStreamDestroy(c->cap); c->cap = nullptr; }
    for (void* a : c->allocs) cudaFree(a);
    c->allocs.clear();
    c->device_bytes = 0;
    if (c->h_status) { cudaFreeHost(c->h_status); c->h_status = nullptr; }
    if (c->h_norm) { cudaFreeHost(c->h_norm); c->h_norm = nullptr; }
    c->d_cp = nullptr;
    c->d_ri = nullptr;
    c->d_zg = nullptr;
    c->zg_cap = 0;
    c->d_blk = nullptr;
    c->d_mle = nullptr;
    c->bg = spi_ctx::Background();
    c->nrm = spi_ctx::Normal();
    c->dtc = DevDiagTc();
    c->wide_ready = false;
    c->dev_ready = false;
    c->factor_plan_ready = false;
    c->piv_ready = false;
}

// The pivoting form's plan: one launch per level over all its fronts.
void build_bk_plan(const Symbolic& S, FactorPlan& F) {
    F = FactorPlan();
    F.level_launch_ptr.push_back(0);
    for (int32_t l = 0; l < S.nlevels; ++l) {
        const int32_t cnt = S.level_ptr[l + 1] - S.level_ptr[l];
        F.launches.push_back(Launch{14, 0, (int64_t)F.bk_items.size(), cnt});
        F.bk_items.insert(F.bk_items.end(), S.level_list.begin() + S.level_ptr[l], S.level_list.begin() + S.level_ptr[l + 1]);
        F.level_launch_ptr.push_back((int32_t)F.launches.size());
        F.n_kernel_launches++;
    }
}

// The solve structure after a symmetric indefinite factorization: the pivots'
// final order (perm), the rows below each front relabelled to it, and D^-1 block
// by block, on the host (for the variance plans) and the device.
int build_solve_structure(spi_ctx* c, cudaStream_t st) {
    const Symbolic& S = c->S;
    const int32_t n = S.n;
    std::vector<int32_t> lperm((size_t)n), pair((size_t)n);
    std::vector<double> Dd((size_t)n), Doff((size_t)n);
    CK(cudaMemcpyAsync(lperm.data(), c->d_lperm, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(pair.data(), c->d_pair, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Dd.data(), c->d_Dd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(Doff.data(), c->d_Doff, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st));
    int cnt2 = 0;
    CK(cudaMemcpyAsync(&cnt2, c->d_delay + 1 + kMaxDelay, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    c->piv_2x2 = cnt2;
    Symbolic& T = c->S_sol;
    T = S;
    std::vector<int32_t> newpos((size_t)n);
    for (int32_t sn = 0; sn < S.ns; ++sn)
        for (int32_t j = S.sfirst[sn]; j < S.sfirst[sn + 1]; ++j) {
            const int32_t old = S.sfirst[sn] + lperm[(size_t)j];
            if (old < S.sfirst[sn] || old >= S.sfirst[sn + 1]) return SPI_ERR_CUDA;
            T.perm[(size_t)j] = S.perm[(size_t)old];
            newpos[(size_t)old] = j;
        }
    for (int32_t j = 0; j < n; ++j) T.iperm[(size_t)T.perm[(size_t)j]] = j;
    for (int32_t sn = 0; sn < S.ns; ++sn) {
        const int64_t k = S.k_of(sn);
        for (int64_t e = S.srowptr[sn] + k; e < S.srowptr[sn + 1]; ++e) T.srows[(size_t)e] = newpos[(size_t)S.srows[(size_t)e]];
        // After pivoting the front's diagonal block is dense in the new order (and a merged
        // front's columns need not form a chain), so a right-hand side that reaches the
        // front may have nonzeros in any of its columns: every column takes the front's
        // first descendant, and the variance kernels' per-column ranges span the subtree.
        int32_t fmin = S.sfirst[sn];
        for (int32_t j = S.sfirst[sn]; j < S.sfirst[sn + 1]; ++j) fmin = std::min(fmin, S.fdesc[(size_t)j]);
        for (int32_t j = S.sfirst[sn]; j < S.sfirst[sn + 1]; ++j) T.fdesc[(size_t)j] = fmin;
    }
    std::vector<double> da((size_t)n), db((size_t)n, 0.0);
    for (int32_t j = 0; j < n; ++j) {
        if (pair[(size_t)j] < 0) {
            da[(size_t)j] = 1.0 / Dd[(size_t)j];
        } else if (pair[(size_t)j] == j + 1) {
            const double a = Dd[(size_t)j], b = Doff[(size_t)j], e = Dd[(size_t)j + 1], det = a * e - b * b;
            da[(size_t)j] = e / det;
            da[(size_t)j + 1] = a / det;
            db[(size_t)j] = db[(size_t)j + 1] = -b / det;
        }
    }
    CK(cudaMemcpyAsync(c->d_perm_sol, T.perm.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_srows_sol, T.srows.data(), T.srows.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_pair_sol, pair.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_dinv_a, da.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_dinv_b, db.data(), (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->d_fdesc_sol, T.fdesc.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    c->dsym_sol = c->dsym;
    c->dsym_sol.srows = c->d_srows_sol;
    c->dsym_sol.perm = c->d_perm_sol;
    c->dsym_sol.dinv_a = c->d_dinv_a;
    c->dsym_sol.dinv_b = c->d_dinv_b;
    c->dsym_sol.pair = c->d_pair_sol;
    c->dsym_sol.fdesc = c->d_fdesc_sol;
    c->plan_all_ready = c->plan_sub_ready = c->plan_blk_ready = false;  // the structure they follow changed
    c->piv_ready = true;
    return SPI_OK;
}

// Symmetric indefinite factorization (spi_options.pivoting): every front with
// restricted Bunch-Kaufman pivots (k_front_bk), level by level.  A front that
// cannot find a stable pivot among its fully-summed columns has its pivots
// delayed to its parent: the analysis is redone with that supernode merged
// into its parent's (where its columns are fully summed) and the factorization
// restarts.  A root front that cannot pivot means a singular matrix.
int factor_pivoting(spi_ctx* c, const double* values, int values_on_device, cudaStream_t st) {
    if (!values && c->S.nnz_a > 0) return SPI_ERR_ARG;
    c->factored = false;
    c->bad_pivot = c->bad_band = -1;
    c->piv_restarts = c->piv_delays = 0;
    for (int attempt = 0;; ++attempt) {
        int rc = ensure_device(c);
        if (rc) return rc;
        const Symbolic& S = c->S;
        if (!c->factor_plan_ready) {
            build_bk_plan(S, c->FP);
            rc = upload_factor_plan(c, c->FP, c->dfp);
            if (rc) return rc;
            c->factor_plan_ready = true;
        }
        const double* vals = values;
        if (S.nnz_a > 0 && !values_on_device) {
            CK(cudaMemcpyAsync(c->d_vals, values, (size_t)S.nnz_a * sizeof(double), cudaMemcpyHostToDevice, st));
            vals = c->d_vals;
        }
        k_reset_status<<<1, 1, 0, st>>>(c->d_status);
        CK(cudaMemsetAsync(c->d_delay, 0, (kMaxDelay + 2) * sizeof(int), st));
        CK(factor_assemble(c, 1, vals, st));
        factor_launches(c, 1, c->FP, c->dfp, st, nullptr);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
        int ndelay = 0;
        CK(cudaMemcpyAsync(&ndelay, c->d_delay, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (!(c->h_status->flags & FLAG_DELAY)) break;
        std::vector<int> list((size_t)std::min(ndelay, kMaxDelay));
        if (!list.empty())
            CK(cudaMemcpy(list.data(), c->d_delay + 1, list.size() * sizeof(int), cudaMemcpyDeviceToHost));
        if (c->prm.force_merge.empty()) c->prm.force_merge.assign((size_t)S.n, 0);
        // A front above a delayed one ran on an incomplete front (the delayed front added
        // nothing to it), so only the first failures on each path count: delayed fronts
        // with no delayed descendant.
        std::vector<char> delayed((size_t)S.ns, 0), below((size_t)S.ns, 0);
        for (int sn : list) {
            if (sn < 0 || sn >= S.ns) return SPI_ERR_CUDA;
            delayed[(size_t)sn] = 1;
        }
        for (int sn : list)
            for (int32_t q = S.sparent[sn]; q != -1 && !below[(size_t)q]; q = S.sparent[q]) below[(size_t)q] = 1;
        int merged = 0;
        for (int sn : list) {
            if (below[(size_t)sn]) continue;
            if (S.sparent[sn] == -1) {  // every row of a root front is fully summed: singular
                c->bad_pivot = S.perm[(size_t)S.sfirst[sn]];
                return SPI_ERR_NOT_SPD;
            }
            for (int32_t j = S.sfirst[sn]; j < S.sfirst[sn + 1]; ++j) c->prm.force_merge[(size_t)S.perm[(size_t)j]] = 1;
            ++merged;
        }
        c->piv_delays += merged;
        if (attempt >= kMaxRestarts) return SPI_ERR_NOT_SPD;
        // the delayed fronts merged into their parents: a new structure, a new device setup
        Symbolic S2;
        std::string err;
        const int64_t n = S.n;
        rc = analyse(n, c->in_colptr.data(), c->in_rowind.data(), c->prm, S2, err);
        if (rc) return rc;
        reset_device(c);
        c->S = std::move(S2);
        build_solve_plan(c->S, c->SP, 1);
        build_solve_dag(c->S, c->SP);
        c->piv_restarts++;
    }
    int rc = build_solve_structure(c, st);
    if (rc) return rc;
    rc = finish(c, st);
    if (rc == SPI_OK) {
        c->factored = true;
        c->factored_nb = 1;
    }
    return rc;
}

int factor_impl(spi_ctx* c, int nb, const double* values, int values_on_device, cudaStream_t st) {
    if (!c || nb < 1 || nb > c->opt.batch) return SPI_ERR_ARG;
    if (c->opt.pivoting) return factor_pivoting(c, values, values_on_device, st);
    if (!values && c->S.nnz_a > 0) return SPI_ERR_ARG;
    int rc = ensure_device(c);
    if (rc) return rc;
    const Symbolic& S = c->S;
    const bool mixed = mixed_of(c);
    c->factored = false;
    c->bad_pivot = c->bad_band = -1;
    const double* vals = values;
    if (S.nnz_a > 0 && (!values_on_device || mixed)) {
        CK(cudaMemcpyAsync(c->d_vals, values, (size_t)S.nnz_a * nb * sizeof(double),
                           values_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
        vals = c->d_vals;
    }
    if (!c->factor_plan_ready) {
        rc = prepare_factor_plan(c, nb, vals, st);
        if (rc) return rc;
    }
    k_reset_status<<<1, 1, 0, st>>>(c->d_status);
    // panels and update areas in the factorization's storage type (FP32 in the mixed form)
    CK(factor_assemble(c, nb, vals, st));
    CK(run_graph(c, c->g_factor, nb, st, [&](cudaStream_t s2) {
        factor_launches(c, nb, c->FP, c->dfp, s2, nullptr);
        // the solves, inverse blocks and the allocation-free variances read the FP64 panels
        if (mixed) launch_to_f64(c->d_L32, c->d_L, S.lptr[S.ns] * nb, s2);
        // the variances' tensor-core operands (inverted diagonal tiles, packed TF32 pairs)
        if (mixed) launch_diag_tc_pack(c->dsym, c->dtc, c->d_L32, nb, c->bs, s2);
    }));
    rc = finish(c, st);
    if (rc == SPI_OK) {
        c->factored = true;
        c->factored_nb = nb;
    }
    return rc;
}

// x = P^T L^-T D^-1 L^-1 P b on device buffers of nb bands (b, x distinct from d_w/d_z/d_xp).
cudaError_t solve_core(spi_ctx* c, int nb, const double* b, double* x, cudaStream_t st) {
    const Symbolic& S = c->S;
    const DevSym& ds = dev_sol(c);
    launch_permute_in(S.n, ds.perm, b, c->d_w, nb, st);
    if (c->solve_dag == 1) {
        cudaError_t e = run_graph(c, c->g_solve_dag, nb, st, [&](cudaStream_t s2) {
            const int cstride = 3 * S.ns;
            cudaMemsetAsync(c->d_solve_cnt, 0, ((size_t)nb * cstride + 1) * sizeof(int), s2);
            launch_solve_dag(c->dsym, c->d_solve_dag, (int)c->SP.dag.size(), c->d_solve_cnt, cstride, c->d_L, c->d_D,
                             c->d_w, c->d_z, c->d_xp, c->d_status, nb, c->bs, c->opt.wait_limit,
                             c->solve_dag_grid_size, s2, mixed_of(c) ? c->d_L32 : nullptr);
        });
        launch_permute_out(S.n, c->dsym.perm, c->d_xp, x, nb, st);
        return e;
    }
    cudaError_t e = run_graph(c, c->g_solve, nb, st, [&](cudaStream_t s2) {
        // the mixed form's solves read its FP32 panels (the FP64 copy holds the same values)
        // and take 128-column steps where the factorization left inverted diagonal tiles
        const float* L32 = mixed_of(c) ? c->d_L32 : nullptr;
        const bool wide = L32 && c->wide_ready;
        const SolvePlan& P = wide ? c->SPw : c->SP;
        const int32_t* fi = wide ? c->d_fwd_items_w : c->d_fwd_items;
        const int32_t* bi = wide ? c->d_bwd_items_w : c->d_bwd_items;
        for (const Launch& l : P.fwd_launches)
            launch_solve_step(ds, l, fi, bi, c->d_L, c->d_D, c->d_w, c->d_z, c->d_xp, nb, c->bs, s2, L32,
                              wide ? &c->wa : nullptr);
        for (const Launch& l : P.bwd_launches)
            launch_solve_step(ds, l, fi, bi, c->d_L, c->d_D, c->d_w, c->d_z, c->d_xp, nb, c->bs, s2, L32,
                              wide ? &c->wa : nullptr);
    });
    launch_permute_out(S.n, ds.perm, c->d_xp, x, nb, st);
    return e;
}

// The solve's form (dependency-driven launch or launches level by level), decided
// at the first solve when spi_options.dag = 0: timed on the caller's right-hand
// side when spi_options.autotune allows (the faster of two runs each), else the
// dependency-driven launch.
int choose_solve_form(spi_ctx* c, int nb, const double* bd, cudaStream_t st) {
    if (c->solve_dag >= 0) return SPI_OK;
    const std::string key = tune_key(c, nb);
    {
        std::vector<TuneLine> cached;
        read_tune_cache(c->opt.tune_cache, key, cached, nullptr);
        for (const TuneLine& t : cached)
            if (t.kind == 'V') c->solve_dag = t.choice != 0 && !c->SP.dag.empty();
        if (c->solve_dag >= 0) return SPI_OK;
    }
    const bool timing = c->opt.autotune > 0 || (c->opt.autotune == 0 && c->S.factor_flops >= 2e8);
    if (!timing || c->SP.dag.empty()) {
        c->solve_dag = c->SP.dag.empty() ? 0 : 1;
        return SPI_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = SPI_OK;
    for (int form = 0; form < 2 && rc == SPI_OK; ++form) {
        c->solve_dag = form;
        double best = -1.0;
        for (int rep = 0; rep < 3 && rc == SPI_OK; ++rep) {
            cudaEventRecord(e0, st);
            if (solve_core(c, nb, bd, c->d_x ? c->d_x : c->d_out, st) != cudaSuccess) rc = SPI_ERR_CUDA;
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (rc == SPI_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                rep > 0 && (best < 0 || ms < best))
                best = ms;
        }
        c->tune_solve_ms[form] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->solve_dag = c->tune_solve_ms[1] >= 0 && c->tune_solve_ms[1] < c->tune_solve_ms[0] ? 1 : 0;
    tune_cache_update(c->opt.tune_cache, key, "V",
                      {TuneLine{'V', 0, c->solve_dag, c->tune_solve_ms[0], c->tune_solve_ms[1]}});
    return finish(c, st);
}

int solve_impl(spi_ctx* c, int nb, const double* b, double* x, int on_device, cudaStream_t st) {
    if (!c || nb < 1 || (!b && c->S.n) || (!x && c->S.n)) return SPI_ERR_ARG;
    if (!c->factored) return SPI_ERR_STATE;
    if (nb > c->factored_nb) return SPI_ERR_ARG;
    const int32_t n = c->S.n;
    const size_t bytes = (size_t)n * nb * sizeof(double);
    const double* bd = b;
    if (!on_device && n) {
        CK(cudaMemcpyAsync(c->d_vec, b, bytes, cudaMemcpyHostToDevice, st));
        bd = c->d_vec;
    }
    {
        const int rc = choose_solve_form(c, nb, bd, st);
        if (rc) return rc;
    }
    double* xd = on_device ? x : c->d_vec;
    if (!mixed_of(c)) {
        CK(solve_core(c, nb, bd, xd, st));
    } else if (n) {
        // FP64 iterative refinement against N: x += solve(b - N x), every band until all converge.
        // The correction steps the last converged solve needed run first without a look at
        // the residual (no host round trip between them); then the residual is checked after
        // every step until it is below refine_tol.
        CK(cudaMemcpyAsync(c->d_b2, bd, bytes, cudaMemcpyDeviceToDevice, st));
        CK(solve_core(c, nb, c->d_b2, c->d_x, st));
        std::vector<double> bnorm(nb, -1.0);
        c->refine_steps = 0;
        const int64_t blind = std::min<int64_t>(std::max<int64_t>(c->refine_planned, 0), c->opt.refine_max);
        for (int64_t q = 0; q < blind; ++q) {
            CK(cudaMemcpyAsync(c->d_r, c->d_b2, bytes, cudaMemcpyDeviceToDevice, st));
            launch_sym_residual(n, c->d_cp, c->d_ri, c->d_vals, c->d_x, c->d_r, nb, c->S.nnz_a, st);
            CK(solve_core(c, nb, c->d_r, c->d_dx, st));
            launch_axpy(n, c->d_dx, c->d_x, nb, st);
            c->refine_steps++;
        }
        for (int it = 0;; ++it) {
            CK(cudaMemcpyAsync(c->d_r, c->d_b2, bytes, cudaMemcpyDeviceToDevice, st));
            launch_sym_residual(n, c->d_cp, c->d_ri, c->d_vals, c->d_x, c->d_r, nb, c->S.nnz_a, st);
            CK(cudaMemsetAsync(c->d_norm, 0, 2 * nb * sizeof(double), st));
            launch_norms2(n, c->d_r, it == 0 ? c->d_b2 : nullptr, c->d_norm, nb, st);
            CK(cudaMemcpyAsync(c->h_norm, c->d_norm, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            bool done = true;
            double worst = 0.0;
            for (int k = 0; k < nb; ++k) {
                if (it == 0) bnorm[k] = std::sqrt(c->h_norm[2 * k + 1]);
                const double rn = std::sqrt(c->h_norm[2 * k]);
                worst = std::max(worst, bnorm[k] > 0 ? rn / bnorm[k] : rn);
                if (rn > c->opt.refine_tol * bnorm[k]) done = false;
            }
            c->solve_relres = worst;
            if (done) c->refine_planned = c->refine_steps;
            if (done || c->refine_steps >= c->opt.refine_max) break;
            CK(solve_core(c, nb, c->d_r, c->d_dx, st));
            launch_axpy(n, c->d_dx, c->d_x, nb, st);
            c->refine_steps++;
        }
        CK(cudaMemcpyAsync(xd, c->d_x, bytes, cudaMemcpyDeviceToDevice, st));
    }
    if (!on_device && n) {
        CK(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return finish(c, st);
}

void launch_diag(spi_ctx* c, const DevDiagPlan& p, int nb, int64_t nout, double* out, cudaStream_t st) {
    Strides bs = c->bs;
    bs.Z = p.zsize;
    bs.out = nout;
    if (mixed_of(c)) {
        const bool tc = c->dtc.ntc > 0 && p.B <= kDiagTcMaxBlock;
        launch_diag_inverse_f32(c->dsym, p, c->d_L32, c->d_D, out, nb, bs, c->diag_smem_pad,
                                tc ? c->dtc.tc : nullptr, st);
        if (tc) launch_diag_inv_tc(c->dsym, p, c->dtc, c->d_D, out, nb, bs, c->d_status, c->opt.wait_limit, st);
    } else {
        launch_diag_inverse(dev_sol(c), p, c->d_L, c->d_D, out, nb, bs, c->diag_smem_pad, st);
    }
}

// Build the plan for the pivots `piv`; with an automatic block size (the
// autotuner), time each candidate once on the current factor and keep the
// fastest for every later plan of this context.
int make_plan(spi_ctx* c, const std::vector<int32_t>& piv, const std::vector<int32_t>& pos, DevDiagPlan& dst,
              int nb, int64_t nout, double* out, cudaStream_t st) {
    std::vector<int> cands;
    if (c->opt.rhs_block > 0) cands.push_back(c->opt.rhs_block);
    else if (c->rhs_block_used > 0) cands.push_back(c->rhs_block_used);
    else if (mixed_of(c)) cands = {32, 64, 128};
    else cands = {16, 32, 64};
    if (cands.size() > 1 && piv.size() < 4096) cands = {mixed_of(c) ? 64 : 32};  // too small to time
    const std::string key = tune_key(c, nb);
    if (cands.size() > 1) {
        std::vector<TuneLine> cached;
        read_tune_cache(c->opt.tune_cache, key, cached, nullptr);
        for (const TuneLine& t : cached)
            if (t.kind == 'B' && std::find(cands.begin(), cands.end(), t.choice) != cands.end()) cands = {t.choice};
    }
    if (cands.size() == 1) {
        DiagPlan h;
        build_diag_plan(sym_sol(c), piv, pos, cands[0], h);
        if (c->opt.rhs_block == 0 && c->rhs_block_used == 0 && piv.size() >= 4096) c->rhs_block_used = cands[0];
        return upload_plan(c, h, dst);
    }
    float best = 1e30f;
    int bestB = cands[0];
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = SPI_OK;
    for (int B : cands) {
        DiagPlan h;
        build_diag_plan(sym_sol(c), piv, pos, B, h);
        rc = upload_plan(c, h, dst);
        if (rc) break;
        cudaEventRecord(e0, st);
        launch_diag(c, dst, nb, nout, out, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = SPI_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bestB = B; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->rhs_block_used = bestB;
    tune_cache_update(c->opt.tune_cache, key, "B", {TuneLine{'B', 0, bestB, best, 0.0}});
    DiagPlan h;
    build_diag_plan(sym_sol(c), piv, pos, bestB, h);
    return upload_plan(c, h, dst);
}

// The pruning ablation (spi_options.diag_unpruned): every variance from a full forward
// solve z = L^-1 e_i over all supernodes (32 right-hand sides per pass, FP64 panels),
// var_i = sum_k z_k^2 / d_k.  Band 0 only.
int diag_unpruned_impl(spi_ctx* c, const int32_t* idx, int64_t nidx, double* out, int on_device,
                       cudaStream_t st) {
    const Symbolic& S = c->S;
    const int32_t n = S.n;
    std::vector<int32_t> key;
    if (!idx) {
        key.resize((size_t)n);
        for (int32_t i = 0; i < n; ++i) key[(size_t)i] = i;
        nidx = n;
    } else {
        if (nidx < 0 || nidx > S.n) return SPI_ERR_ARG;
        key.resize((size_t)nidx);
        if (nidx) {
            if (on_device) {
                CK(cudaMemcpyAsync(key.data(), idx, (size_t)nidx * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            } else {
                std::memcpy(key.data(), idx, (size_t)nidx * sizeof(int32_t));
            }
        }
        for (int32_t v : key)
            if (v < 0 || v >= n) return SPI_ERR_ARG;
    }
    if (nidx == 0) return SPI_OK;
    constexpr int kR = 32;
    const size_t vec = (size_t)std::min<int64_t>(kR, nidx) * (size_t)n;
    double* buf = nullptr;
    const size_t bytes = (2 * vec + (size_t)n + (size_t)nidx) * sizeof(double) + (size_t)kR * sizeof(int32_t);
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SPI_ERR_OOM;
    }
    double *w = buf, *z = w + vec, *dinv = z + vec, *dout = dinv + n;
    int32_t* dpos = reinterpret_cast<int32_t*>(dout + nidx);
    Strides bs = c->bs;
    bs.L = 0;  // one factor for every right-hand side
    bs.Dn = 0;
    auto run = [&]() -> cudaError_t {
        launch_reciprocal(n, c->d_D, dinv, st);
        for (int64_t t0 = 0; t0 < nidx; t0 += kR) {
            const int R = (int)std::min<int64_t>(kR, nidx - t0);
            std::vector<int32_t> pos((size_t)R);
            for (int t = 0; t < R; ++t) pos[(size_t)t] = S.iperm[key[(size_t)(t0 + t)]];
            cudaError_t e = cudaMemcpyAsync(dpos, pos.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            e = cudaMemsetAsync(w, 0, (size_t)R * n * sizeof(double), st);
            if (e != cudaSuccess) return e;
            launch_set_units(n, dpos, R, w, st);
            for (const Launch& l : c->SP.fwd_launches)
                launch_solve_step(c->dsym, l, c->d_fwd_items, c->d_bwd_items, c->d_L, c->d_D, w, z, nullptr, R, bs, st);
            launch_zsq_var(n, z, dinv, R, dout + t0, st);
            e = cudaStreamSynchronize(st);  // pos is reused by the next pass
            if (e != cudaSuccess) return e;
        }
        return cudaMemcpyAsync(out, dout, (size_t)nidx * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    };
    cudaError_t ce = run();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (ce != cudaSuccess) return cuda_fail(ce);
    // the ablation's work: every forward solve walks all of L
    c->last_diag_flops = 0;
    c->last_diag_work = 2.0 * (double)S.lptr[S.ns] * (double)nidx;
    return finish(c, st);
}

int diag_impl(spi_ctx* c, int nb, const int32_t* idx, int64_t nidx, double* out, int on_device, cudaStream_t st) {
    if (!c || !out || nb < 1) return SPI_ERR_ARG;
    if (!c->factored) return SPI_ERR_STATE;
    if (nb > c->factored_nb) return SPI_ERR_ARG;
    if (c->opt.diag_unpruned) {
        if (nb != 1) return SPI_ERR_ARG;
        return diag_unpruned_impl(c, idx, nidx, out, on_device, st);
    }
    const Symbolic& S = sym_sol(c);
    DevDiagPlan* plan;
    int64_t nout;
    double* od = on_device ? out : c->d_out;
    if (!idx) {
        nout = S.n;
        if (!c->plan_all_ready) {
            std::vector<int32_t> piv(S.n), pos(S.n);
            for (int32_t k = 0; k < S.n; ++k) { piv[k] = k; pos[k] = S.perm[k]; }
            int rc = make_plan(c, piv, pos, c->plan_all, nb, nout, od, st);
            if (rc) return rc;
            c->plan_all_ready = true;
        }
        plan = &c->plan_all;
    } else {
        if (nidx < 0 || nidx > S.n) return SPI_ERR_ARG;
        nout = nidx;
        std::vector<int32_t> key((size_t)nidx);
        if (nidx) {
            if (on_device) {
                CK(cudaMemcpyAsync(key.data(), idx, (size_t)nidx * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            } else {
                std::memcpy(key.data(), idx, (size_t)nidx * sizeof(int32_t));
            }
        }
        for (int32_t v : key)
            if (v < 0 || v >= S.n) return SPI_ERR_ARG;
        if (!c->plan_sub_ready || key != c->plan_sub_key) {
            std::vector<int32_t> piv((size_t)nidx), pos((size_t)nidx);
            for (int64_t t = 0; t < nidx; ++t) { piv[t] = S.iperm[key[t]]; pos[t] = (int32_t)t; }
            int rc = make_plan(c, piv, pos, c->plan_sub, nb, nout, od, st);
            if (rc) return rc;
            c->plan_sub_key.swap(key);
            c->plan_sub_ready = true;
        }
        plan = &c->plan_sub;
    }
    launch_diag(c, *plan, nb, nout, od, st);
    if (!on_device && nout) {
        CK(cudaMemcpyAsync(out, od, (size_t)nout * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    c->last_diag_flops = plan->flops * nb;
    c->last_diag_work = plan->work_flops * nb;
    c->last_diag_tc_flops = plan->tc_flops * nb;
    return finish(c, st);
}

// ---------------------------------------------------------------------------
// Variances without any device allocation (spi_diag_inverse_noalloc).
//
// Some callers cannot allocate device memory at the moment they need
// variances: a host thread that must not touch the CUDA allocator (a
// real-time acquisition loop, a callback of another runtime), or a process
// whose device memory is entirely handed out by another allocator.  For them
// the variance computation below uses a fixed scratch array that every GPU
// which loads this library holds from module load until the process exits.
// The caller provides the factored context, the index set and the output,
// all already on the device.
//
// Scratch layout (doubles): [0] error flag word, [1 .. 1+ceil(n/2)) the
// inverse permutation as int32, then one length-n work vector per concurrent
// right-hand side.  Each call clears the flag and every work vector before
// use, so the contents left by an earlier call do not matter; two calls that
// overlap on the GPU (different streams, or different contexts) share the
// array and race.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 21;  // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kNoAllocMaxDevices = 64;
// Device address of the array, per device, looked up on the first call on that
// device.  Several host threads may make their first call at the same time:
// the slots are atomics and the lookup itself is serialised by a mutex.
std::atomic<double*> g_noalloc_ptr[kNoAllocMaxDevices];
std::mutex g_noalloc_mutex;

// The array's device address on the current device `dev`, or nullptr if the
// lookup failed.
double* noalloc_scratch(int dev) {
    double* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
    if (p) return p;
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) {
        cudaGetLastError();  // the failed lookup's own error, not one the caller left pending
        return nullptr;
    }
    p = static_cast<double*>(a);
    g_noalloc_ptr[dev].store(p, std::memory_order_release);
    return p;
}

__global__ void k_noalloc_prepare(const int32_t* __restrict__ perm, int32_t n, double* scratch, int64_t zlen) {
    int32_t* iperm = reinterpret_cast<int32_t*>(scratch + 1);
    double* z = scratch + 1 + (n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) scratch[0] = 0.0;
    for (int64_t k = t0; k < n; k += stride) iperm[perm[k]] = (int32_t)k;
    for (int64_t i = t0; i < zlen; i += stride) z[i] = 0.0;
}

// One right-hand side per CTA at a time, walking the elimination-tree path of
// its pivot supernode by supernode; the work vector is restored to zero on
// the way (every entry it touches is a column of a later supernode of the path).
__global__ void __launch_bounds__(256) k_diag_inv_noalloc(DevSym d, const double* __restrict__ L,
                                                          const double* __restrict__ D,
                                                          const int32_t* __restrict__ idx, int64_t nidx,
                                                          double* __restrict__ out, double* scratch) {
    __shared__ double zc_s;
    const int32_t n = d.n;
    const int32_t* iperm = reinterpret_cast<const int32_t*>(scratch + 1);
    double* z = scratch + 1 + (n + 1) / 2 + (int64_t)blockIdx.x * n;
    for (int64_t t = blockIdx.x; t < nidx; t += gridDim.x) {
        const int32_t i = idx[t];
        if (i < 0 || i >= n) {
            if (threadIdx.x == 0) { scratch[0] = 1.0; out[t] = __longlong_as_double(0x7ff8000000000000LL); }
            continue;
        }
        const int32_t piv = iperm[i];
        if (threadIdx.x == 0) z[piv] = 1.0;
        __syncthreads();
        double var = 0.0;
        for (int s = d.snode_of[piv]; s != -1; s = d.sparent[s]) {
            const int f = d.sfirst[s], k = d.sfirst[s + 1] - f;
            const int64_t m = d.srowptr[s + 1] - d.srowptr[s];
            const double* P = L + d.lptr[s];
            const int32_t* rows = d.srows + d.srowptr[s];
            for (int c = (piv > f ? piv - f : 0); c < k; ++c) {
                if (threadIdx.x == 0) {
                    zc_s = z[f + c];
                    z[f + c] = 0.0;
                }
                __syncthreads();
                const double zc = zc_s;
                if (threadIdx.x == 0) var += zc * zc / D[f + c];
                if (zc != 0.0)
                    for (int64_t r = c + 1 + threadIdx.x; r < m; r += blockDim.x)
                        z[r < k ? f + r : rows[r]] -= P[r + (int64_t)c * m] * zc;
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) out[t] = var;
        __syncthreads();
    }
}

}  // namespace

extern "C" {

void spi_default_options(spi_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = SPI_PREC_FP64;
    o->ordering = SPI_ORDER_ND;
    o->rhs_block = 0;
    o->relax = 1;
    o->refine_max = 10;
    o->refine_tol = 1e-13;
    o->async = 0;
    o->nd_leaf = 0;
    o->batch = 1;
}

const char* spi_strerror(int s) {
    switch (s) {
        case SPI_OK: return "ok";
        case SPI_ERR_ARG: return "invalid argument";
        case SPI_ERR_PATTERN: return "invalid sparsity pattern (lower CSC, sorted rows, full diagonal)";
        case SPI_ERR_NOT_SPD: return "matrix not positive definite (non-positive pivot)";
        case SPI_ERR_OOM: return "out of memory";
        case SPI_ERR_CUDA: return "CUDA error or no usable GPU";
        case SPI_ERR_TIMEOUT: return "bounded device wait timed out";
        case SPI_ERR_STATE: return "call out of order";
        case SPI_ERR_SCRATCH:
            return "order n too large for the fixed scratch of spi_diag_inverse_noalloc (n <= 1398100)";
        default: return "unknown status";
    }
}

int spi_analyse(int64_t n, const int64_t* colptr, const int32_t* rowind, const spi_options* opt,
                spi_ctx** out) {
    if (!out) return SPI_ERR_ARG;
    *out = nullptr;
    spi_options o;
    spi_default_options(&o);
    if (opt) o = *opt;
    if (o.batch <= 0) o.batch = 1;
    if (o.rhs_block < 0 || o.rhs_block > 512 || o.precision < 0 || o.precision > 1 || o.ordering < 0 ||
        o.ordering > 1 || o.relax < 0 || o.refine_max < 0 || o.nd_leaf < 0 || o.diag_ctas_per_sm < 0 ||
        o.diag_unpruned < 0 || o.diag_unpruned > 1 || o.autotune < -1 || o.autotune > 1 || o.force_panel < 0 ||
        o.force_panel > 2 || o.force_schur < 0 || o.force_schur > 2 || o.dag < 0 || o.dag > 2 || o.pivoting < 0 ||
        o.pivoting > 1 || (o.pivoting && (o.precision != SPI_PREC_FP64 || o.batch > 1 || o.diag_unpruned)))
        return SPI_ERR_ARG;
    if (o.pivoting) o.dag = 1;  // the pivoting form runs level by level
    if (o.precision == SPI_PREC_MIXED_FP32 && o.rhs_block > 0) o.rhs_block = (o.rhs_block + 7) & ~7;
    spi_ctx* c = new (std::nothrow) spi_ctx();
    if (!c) return SPI_ERR_OOM;
    c->opt = o;
    if (o.tune_cache) {
        c->tune_cache_path = o.tune_cache;
        c->opt.tune_cache = c->tune_cache_path.c_str();
    }
    auto t0 = std::chrono::steady_clock::now();
    AnalyseParams prm;
    prm.ordering = o.ordering;
    prm.relax = o.relax;
    prm.nd_leaf = o.nd_leaf;
    if (o.pivoting) prm.group_max = 1;  // no diagonal-block groups of leaves: every front pivots alike
    std::string err;
    int rc = analyse(n, colptr, rowind, prm, c->S, err);
    c->prm = prm;
    if (rc != 0) { delete c; return rc; }
    try {
        FactorChoice ch;  // the built-in rules until the first factorization makes the plan final
        ch.force_panel = o.force_panel;
        ch.force_schur = o.force_schur;
        ch.dag = o.dag != 1;
        build_factor_plan(c->S, c->FP, o.precision == SPI_PREC_MIXED_FP32, ch, false);
        build_solve_plan(c->S, c->SP, std::max(1, o.batch));
        build_solve_dag(c->S, c->SP);
        if (n > 0) {  // the residual of the mixed form and the normal-equation assembly use it
            c->in_colptr.assign(colptr, colptr + n + 1);
            c->in_rowind.assign(rowind, rowind + colptr[n]);
        }
    } catch (const std::bad_alloc&) {
        delete c;
        return SPI_ERR_OOM;
    }
    c->analyse_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = c;
    return SPI_OK;
}

int spi_analyse_multi(int32_t nprob, const int64_t* n, const int64_t* const* colptr,
                      const int32_t* const* rowind, const spi_options* opt, spi_ctx** out) {
    if (!out || nprob < 0 || (nprob > 0 && (!n || !colptr || !rowind))) return SPI_ERR_ARG;
    *out = nullptr;
    int64_t ntot = 0, nnz = 0;
    for (int32_t p = 0; p < nprob; ++p) {
        if (n[p] < 0 || (n[p] > 0 && (!colptr[p] || !rowind[p]))) return SPI_ERR_ARG;
        ntot += n[p];
        nnz += n[p] > 0 ? colptr[p][n[p]] : 0;
    }
    if (ntot > INT32_MAX - 1) return SPI_ERR_ARG;
    std::vector<int64_t> cp;
    std::vector<int32_t> ri;
    try {
        cp.reserve((size_t)ntot + 1);
        ri.reserve((size_t)nnz);
        cp.push_back(0);
        int64_t base = 0;
        for (int32_t p = 0; p < nprob; ++p) {
            for (int64_t j = 0; j < n[p]; ++j) {
                for (int64_t q = colptr[p][j]; q < colptr[p][j + 1]; ++q) {
                    const int32_t r = rowind[p][q];
                    if (r < 0 || r >= n[p]) return SPI_ERR_PATTERN;
                    ri.push_back((int32_t)(base + r));
                }
                cp.push_back((int64_t)ri.size());
            }
            base += n[p];
        }
    } catch (const std::bad_alloc&) {
        return SPI_ERR_OOM;
    }
    return spi_analyse(ntot, cp.data(), ri.data(), opt, out);
}

int spi_factor(spi_ctx* c, const double* values, int values_on_device, void* stream) {
    return factor_impl(c, 1, values, values_on_device, (cudaStream_t)stream);
}

int spi_factor_batch(spi_ctx* c, int32_t nbatch, const double* values, int values_on_device, void* stream) {
    return factor_impl(c, nbatch, values, values_on_device, (cudaStream_t)stream);
}

int spi_solve(spi_ctx* c, const double* b, double* x, int on_device, void* stream) {
    return solve_impl(c, 1, b, x, on_device, (cudaStream_t)stream);
}

int spi_solve_batch(spi_ctx* c, int32_t nbatch, const double* b, double* x, int on_device, void* stream) {
    return solve_impl(c, nbatch, b, x, on_device, (cudaStream_t)stream);
}

int spi_diag_inverse(spi_ctx* c, const int32_t* idx, int64_t nidx, double* out, int on_device, void* stream) {
    return diag_impl(c, 1, idx, nidx, out, on_device, (cudaStream_t)stream);
}

int spi_diag_inverse_batch(spi_ctx* c, int32_t nbatch, const int32_t* idx, int64_t nidx, double* out,
                           int on_device, void* stream) {
    return diag_impl(c, nbatch, idx, nidx, out, on_device, (cudaStream_t)stream);
}

namespace {
// (N^-1)[key, key] (row-major, |key| x |key|) into the device buffer od; key: distinct caller
// indices, at most SPI_INVERSE_BLOCK_MAX, already checked.  The plan is cached per key.
int inverse_block_impl(spi_ctx* c, std::vector<int32_t>& key, double* od, cudaStream_t st) {
    const Symbolic& S = c->S;
    const int64_t nidx = (int64_t)key.size();
    if (!c->plan_blk_ready || key != c->plan_blk_key) {
        c->plan_blk_ready = false;
        std::vector<int32_t> piv((size_t)nidx), pos((size_t)nidx);
        for (int64_t t = 0; t < nidx; ++t) { piv[t] = S.iperm[key[t]]; pos[t] = (int32_t)t; }
        DiagPlan h;
        build_diag_plan(S, piv, pos, c->rhs_block_used > 0 ? c->rhs_block_used : 32, h);
        int rc = upload_plan(c, h, c->plan_blk);
        if (rc) return rc;
        // rows of the union of all blocks' paths (ascending pivots), and each
        // block-local Z row's position among them; a block's supernodes own
        // consecutive local rows from uzoff
        std::vector<int32_t> gidx((size_t)S.n, -1), zpiv, rowmap((size_t)(h.zbase.back() / h.B), -1);
        for (int bl = 0; bl < h.nblocks; ++bl)
            for (int u = h.uptr[bl]; u < h.uptr[bl + 1]; ++u)
                for (int32_t j = S.sfirst[h.us[u]]; j < S.sfirst[h.us[u] + 1]; ++j) gidx[(size_t)j] = 0;
        for (int32_t j = 0; j < S.n; ++j)
            if (gidx[(size_t)j] == 0) { gidx[(size_t)j] = (int32_t)zpiv.size(); zpiv.push_back(j); }
        for (int bl = 0; bl < h.nblocks; ++bl) {
            const int64_t base = h.zbase[bl] / h.B, rows = (h.zbase[bl + 1] - h.zbase[bl]) / h.B;
            for (int u = h.uptr[bl]; u < h.uptr[bl + 1]; ++u) {
                const int32_t sn = h.us[u], f = S.sfirst[sn], k = S.sfirst[sn + 1] - f;
                for (int32_t j = 0; j < k; ++j) {
                    const int64_t r = (int64_t)h.uzoff[u] + j;
                    if (r < 0 || r >= rows) return SPI_ERR_ARG;
                    rowmap[(size_t)(base + r)] = gidx[(size_t)(f + j)];
                }
            }
        }
        for (int32_t v : rowmap)
            if (v < 0) return SPI_ERR_ARG;
        CK(dev_upload(c, &c->plan_blk.zpiv, zpiv, &c->plan_blk.allocs));
        CK(dev_upload(c, &c->plan_blk.rowmap, rowmap, &c->plan_blk.allocs));
        c->blk_rows = (int64_t)zpiv.size();
        if (c->blk_rows * nidx > c->zg_cap) {
            if (c->d_zg) { cudaFree(c->d_zg); c->d_zg = nullptr; c->zg_cap = 0; }
            if (cudaMalloc(&c->d_zg, (size_t)c->blk_rows * (size_t)nidx * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                c->d_zg = nullptr;
                return SPI_ERR_OOM;
            }
            c->zg_cap = c->blk_rows * nidx;
        }
        c->plan_blk_key.swap(key);
        c->plan_blk_ready = true;
    }
    launch_inverse_block(c->dsym, c->plan_blk, c->d_L, c->d_D, c->d_out, c->d_zg, c->blk_rows, od, nidx, st);
    return SPI_OK;
}
}  // namespace

int spi_inverse_block(spi_ctx* c, const int32_t* idx, int64_t nidx, double* out, int on_device, void* stream) {
    if (!c || c->opt.pivoting) return SPI_ERR_ARG;
    if (!c->factored) return SPI_ERR_STATE;
    if (nidx < 0 || nidx > SPI_INVERSE_BLOCK_MAX || (nidx > 0 && (!idx || !out))) return SPI_ERR_ARG;
    if (nidx == 0) return SPI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const Symbolic& S = c->S;
    std::vector<int32_t> key((size_t)nidx);
    if (on_device) {
        CK(cudaMemcpyAsync(key.data(), idx, (size_t)nidx * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(key.data(), idx, (size_t)nidx * sizeof(int32_t));
    }
    {
        std::vector<int32_t> srt(key);
        std::sort(srt.begin(), srt.end());
        if (srt.front() < 0 || srt.back() >= S.n) return SPI_ERR_ARG;
        if (std::adjacent_find(srt.begin(), srt.end()) != srt.end()) return SPI_ERR_ARG;
    }
    if (!on_device && !c->d_blk)
        CK(dev_alloc(c, &c->d_blk, (size_t)SPI_INVERSE_BLOCK_MAX * SPI_INVERSE_BLOCK_MAX));
    double* od = on_device ? out : c->d_blk;
    int rc = inverse_block_impl(c, key, od, st);
    if (rc) return rc;
    if (!on_device) {
        CK(cudaMemcpyAsync(out, od, (size_t)nidx * nidx * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return finish(c, st);
}

int spi_diag_inverse_refined(spi_ctx* c, const int32_t* idx, int64_t nidx, double* out, int on_device,
                             void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->factored) return SPI_ERR_STATE;
    if (nidx < 0 || (nidx > 0 && (!idx || !out))) return SPI_ERR_ARG;
    if (nidx == 0) return SPI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // an FP64 factor's variances have no first-order error to remove
    if (!mixed_of(c)) return diag_impl(c, 1, idx, nidx, out, on_device, st);
    const Symbolic& S = c->S;
    const int32_t n = S.n;
    std::vector<int32_t> key((size_t)nidx);
    if (on_device) {
        CK(cudaMemcpyAsync(key.data(), idx, (size_t)nidx * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(key.data(), idx, (size_t)nidx * sizeof(int32_t));
    }
    for (int32_t i : key)
        if (i < 0 || i >= n) return SPI_ERR_ARG;
    constexpr int kR = 32;  // right-hand sides per pass
    const int64_t R0 = std::min<int64_t>(kR, nidx);
    const size_t vec = (size_t)R0 * (size_t)n;
    // w, z, xp (pivot order), x (caller order), r; then pivots, indices and outputs of a pass
    double* buf = nullptr;
    const size_t bytes = 5 * vec * sizeof(double) + 2 * (size_t)kR * sizeof(int32_t) + (size_t)nidx * sizeof(double);
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SPI_ERR_OOM;
    }
    double *w = buf, *z = w + vec, *xp = z + vec, *x = xp + vec, *r = x + vec;
    int32_t* dpos = reinterpret_cast<int32_t*>(r + vec);
    int32_t* didx = dpos + kR;
    double* dout = reinterpret_cast<double*>(didx + kR);
    Strides bs = c->bs;
    bs.L = 0;   // one factor for every right-hand side
    bs.Dn = 0;
    int rc = SPI_OK;
    auto run = [&]() -> cudaError_t {
        for (int64_t t0 = 0; t0 < nidx; t0 += kR) {
            const int R = (int)std::min<int64_t>(kR, nidx - t0);
            std::vector<int32_t> pos((size_t)R);
            for (int t = 0; t < R; ++t) pos[(size_t)t] = S.iperm[key[(size_t)(t0 + t)]];
            cudaError_t e = cudaMemcpyAsync(dpos, pos.data(), (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            e = cudaMemcpyAsync(didx, key.data() + t0, (size_t)R * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return e;
            // v = F^-1 e_i: the full forward and backward sweeps with the factor in FP64 arithmetic
            e = cudaMemsetAsync(w, 0, (size_t)R * n * sizeof(double), st);
            if (e != cudaSuccess) return e;
            launch_set_units(n, dpos, R, w, st);
            for (const Launch& l : c->SP.fwd_launches)
                launch_solve_step(c->dsym, l, c->d_fwd_items, c->d_bwd_items, c->d_L, c->d_D, w, z, xp, R, bs, st);
            for (const Launch& l : c->SP.bwd_launches)
                launch_solve_step(c->dsym, l, c->d_fwd_items, c->d_bwd_items, c->d_L, c->d_D, w, z, xp, R, bs, st);
            launch_permute_out(n, c->dsym.perm, xp, x, R, st);
            // r = -N v with the FP64 input matrix, then 2 v_i - v^T N v
            e = cudaMemsetAsync(r, 0, (size_t)R * n * sizeof(double), st);
            if (e != cudaSuccess) return e;
            launch_sym_residual(n, c->d_cp, c->d_ri, c->d_vals, x, r, R, 0, st);
            launch_refined_var(n, x, r, didx, R, dout + t0, st);
            e = cudaStreamSynchronize(st);  // pos and the index slice are reused by the next pass
            if (e != cudaSuccess) return e;
        }
        return cudaMemcpyAsync(out, dout, (size_t)nidx * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    };
    cudaError_t ce = run();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) rc = cuda_fail(ce);
    cudaFree(buf);
    if (rc) return rc;
    return finish(c, st);
}

int spi_inverse_entries(spi_ctx* c, const int32_t* rows, const int32_t* cols, int64_t nent, double* out,
                        int on_device, void* stream) {
    if (!c || c->opt.pivoting) return SPI_ERR_ARG;
    if (!c->factored) return SPI_ERR_STATE;
    if (nent < 0 || (nent > 0 && (!rows || !cols || !out))) return SPI_ERR_ARG;
    if (nent == 0) return SPI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const Symbolic& S = c->S;
    std::vector<int32_t> ri((size_t)nent), ci((size_t)nent);
    if (on_device) {
        CK(cudaMemcpyAsync(ri.data(), rows, (size_t)nent * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ci.data(), cols, (size_t)nent * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    } else {
        std::memcpy(ri.data(), rows, (size_t)nent * sizeof(int32_t));
        std::memcpy(ci.data(), cols, (size_t)nent * sizeof(int32_t));
    }
    // the distinct indices in pivot order, cut into groups of half a block: a pair's
    // entry comes from the block of its two groups (their paths overlap the most
    // when the groups are consecutive in the elimination order)
    std::vector<int32_t> uniq;
    uniq.reserve((size_t)nent * 2);
    for (int64_t t = 0; t < nent; ++t) {
        if (ri[t] < 0 || ri[t] >= S.n || ci[t] < 0 || ci[t] >= S.n) return SPI_ERR_ARG;
        uniq.push_back(ri[t]);
        uniq.push_back(ci[t]);
    }
    std::sort(uniq.begin(), uniq.end(), [&](int32_t a, int32_t b) { return S.iperm[a] < S.iperm[b]; });
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    constexpr int64_t kGroup = SPI_INVERSE_BLOCK_MAX / 2;
    std::vector<int32_t> rank((size_t)S.n, -1);
    for (size_t u = 0; u < uniq.size(); ++u) rank[(size_t)uniq[u]] = (int32_t)u;
    // requested entries by group pair (ga <= gb)
    std::map<std::pair<int64_t, int64_t>, std::vector<int64_t>> buckets;
    for (int64_t t = 0; t < nent; ++t) {
        int64_t ga = rank[(size_t)ri[t]] / kGroup, gb = rank[(size_t)ci[t]] / kGroup;
        if (ga > gb) std::swap(ga, gb);
        buckets[{ga, gb}].push_back(t);
    }
    if (!c->d_blk) CK(dev_alloc(c, &c->d_blk, (size_t)SPI_INVERSE_BLOCK_MAX * SPI_INVERSE_BLOCK_MAX));
    double* od = out;
    double* staged = nullptr;
    if (!on_device) {
        if (cudaMalloc(&staged, (size_t)nent * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return SPI_ERR_OOM;
        }
        od = staged;
    }
    // positions of every entry in its block's row-major output, uploaded once; a block's
    // key is group ga's indices followed (when gb != ga) by group gb's
    std::vector<int64_t> src((size_t)nent), dst((size_t)nent), bptr;
    std::vector<std::vector<int32_t>> keys;
    const int64_t nu = (int64_t)uniq.size();
    auto group_size = [&](int64_t g) { return std::min<int64_t>(kGroup, nu - g * kGroup); };
    int64_t e = 0;
    for (auto& kv : buckets) {
        const int64_t ga = kv.first.first, gb = kv.first.second;
        std::vector<int32_t> key(uniq.begin() + ga * kGroup, uniq.begin() + ga * kGroup + group_size(ga));
        if (gb != ga) key.insert(key.end(), uniq.begin() + gb * kGroup, uniq.begin() + gb * kGroup + group_size(gb));
        const int64_t m = (int64_t)key.size();
        auto local = [&](int64_t r) { return r / kGroup == ga ? r - ga * kGroup : group_size(ga) + (r - gb * kGroup); };
        bptr.push_back(e);
        for (int64_t t : kv.second) {
            src[(size_t)e] = local(rank[(size_t)ri[t]]) * m + local(rank[(size_t)ci[t]]);
            dst[(size_t)e] = t;
            ++e;
        }
        keys.push_back(std::move(key));
    }
    bptr.push_back(e);
    int64_t* d_idx = nullptr;
    int rc = SPI_OK;
    if (cudaMalloc(&d_idx, 2 * (size_t)nent * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        if (staged) cudaFree(staged);
        return SPI_ERR_OOM;
    }
    cudaError_t ce = cudaMemcpyAsync(d_idx, src.data(), (size_t)nent * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_idx + nent, dst.data(), (size_t)nent * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) rc = cuda_fail(ce);
    for (size_t q = 0; q < keys.size() && rc == SPI_OK; ++q) {
        rc = inverse_block_impl(c, keys[q], c->d_blk, st);
        if (rc == SPI_OK)
            launch_pick_entries(c->d_blk, d_idx + bptr[q], d_idx + nent + bptr[q], bptr[q + 1] - bptr[q], od, st);
    }
    if (rc == SPI_OK && !on_device) {
        ce = cudaMemcpyAsync(out, od, (size_t)nent * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce != cudaSuccess) rc = cuda_fail(ce);
    }
    ce = cudaStreamSynchronize(st);
    if (rc == SPI_OK && ce != cudaSuccess) rc = cuda_fail(ce);
    cudaFree(d_idx);
    if (staged) cudaFree(staged);
    if (rc) return rc;
    return finish(c, st);
}

int spi_normal_setup(spi_ctx* c, int64_t nrows, const int64_t* rowptr, const int32_t* colind) {
    if (!c || nrows < 0 || (nrows > 0 && (!rowptr || !colind))) return SPI_ERR_ARG;
    const int32_t n = c->S.n;
    if ((int64_t)c->in_colptr.size() != (int64_t)n + 1) return SPI_ERR_STATE;  // a single analysed pattern
    if (nrows > 0 && rowptr[0] != 0) return SPI_ERR_PATTERN;
    for (int64_t r = 0; r < nrows; ++r) {
        if (rowptr[r + 1] < rowptr[r]) return SPI_ERR_PATTERN;
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            if (colind[e] < 0 || colind[e] >= n) return SPI_ERR_PATTERN;
            if (e > rowptr[r] && colind[e] <= colind[e - 1]) return SPI_ERR_PATTERN;
        }
    }
    if (c->nrm.ready) return SPI_ERR_STATE;  // once per context
    int rc = ensure_device(c);
    if (rc) return rc;
    auto& N = c->nrm;
    N = spi_ctx::Normal();
    const int64_t nnzh = nrows ? rowptr[nrows] : 0;
    N.nrows = nrows;
    N.nnzh = nnzh;
    // row groups: consecutive rows while the union of their columns grows by at most
    // 32 beyond the first row's, at most 32 rows and 8,192 dense entries
    constexpr int kMaxRows = 32, kGrow = 32, kMaxDense = 8192;
    std::vector<int64_t> gcolptr{0};
    std::vector<int32_t> gcols, entpos((size_t)nnzh);
    std::vector<int32_t> uni, cand;
    int32_t max_rows = 1, max_dense = 0;
    N.row_grp.assign((size_t)nrows, 0);
    int64_t r = 0;
    while (r < nrows) {
        uni.assign(colind + rowptr[r], colind + rowptr[r + 1]);
        const size_t base = uni.size();
        int64_t R = 1;
        while (r + R < nrows && R < kMaxRows) {
            cand.clear();
            std::set_union(uni.begin(), uni.end(), colind + rowptr[r + R], colind + rowptr[r + R + 1],
                           std::back_inserter(cand));
            if (cand.size() > base + kGrow || (R + 1) * (int64_t)cand.size() > kMaxDense) break;
            uni.swap(cand);
            ++R;
        }
        const int32_t g = (int32_t)N.grp_row.size();
        N.grp_row.push_back(r);
        for (int64_t q = r; q < r + R; ++q) {
            N.row_grp[(size_t)q] = g;
            for (int64_t e = rowptr[q]; e < rowptr[q + 1]; ++e)
                entpos[(size_t)e] = (int32_t)(std::lower_bound(uni.begin(), uni.end(), colind[e]) - uni.begin());
        }
        gcols.insert(gcols.end(), uni.begin(), uni.end());
        gcolptr.push_back((int64_t)gcols.size());
        if (R > 1) {
            max_rows = std::max<int32_t>(max_rows, (int32_t)R);
            max_dense = std::max<int32_t>(max_dense, (int32_t)(R * (int64_t)uni.size()));
        }
        r += R;
    }
    N.grp_row.push_back(nrows);
    N.ngroups = (int32_t)N.grp_row.size() - 1;
    // H's pattern by columns (the rows of each column), for the column updates
    N.hcp.assign((size_t)n + 1, 0);
    for (int64_t e = 0; e < nnzh; ++e) N.hcp[(size_t)colind[e] + 1]++;
    for (int32_t j = 0; j < n; ++j) N.hcp[(size_t)j + 1] += N.hcp[(size_t)j];
    N.hri.resize((size_t)nnzh);
    {
        std::vector<int64_t> fill(N.hcp.begin(), N.hcp.end() - 1);
        for (int64_t q = 0; q < nrows; ++q)
            for (int64_t e = rowptr[q]; e < rowptr[q + 1]; ++e) N.hri[(size_t)fill[(size_t)colind[e]]++] = (int32_t)q;
    }
    // positions of every group's column pairs in N's pattern (b-major, a >= b), unless the
    // table would exceed 2^28 entries (the kernel then walks the pattern itself)
    std::vector<int64_t> pairptr((size_t)N.ngroups + 1, 0);
    for (int32_t g = 0; g < N.ngroups; ++g) {
        const int64_t cg = gcolptr[(size_t)g + 1] - gcolptr[(size_t)g];
        pairptr[(size_t)g + 1] = pairptr[(size_t)g] + cg * (cg + 1) / 2;
    }
    std::vector<int32_t> pairpos;
    const bool table = pairptr.back() <= (int64_t)1 << 28 && c->S.nnz_a < INT32_MAX;
    if (table) {
        pairpos.resize((size_t)pairptr.back());
        const std::vector<int64_t>& ncp = c->in_colptr;
        const std::vector<int32_t>& nri = c->in_rowind;
        for (int32_t g = 0; g < N.ngroups; ++g) {
            const int32_t* C = gcols.data() + gcolptr[(size_t)g];
            const int64_t cg = gcolptr[(size_t)g + 1] - gcolptr[(size_t)g];
            int64_t o = pairptr[(size_t)g];
            for (int64_t b = 0; b < cg; ++b) {
                int64_t q = ncp[(size_t)C[b]];
                const int64_t qend = ncp[(size_t)C[b] + 1];
                for (int64_t a = b; a < cg; ++a) {
                    while (q < qend && nri[(size_t)q] < C[a]) ++q;
                    pairpos[(size_t)o++] = (q < qend && nri[(size_t)q] == C[a]) ? (int32_t)q : -1;
                }
            }
        }
    }
    std::vector<int64_t> hrow(rowptr, rowptr + nrows + 1);
    std::vector<int32_t> hcol(colind, colind + nnzh);
    std::vector<int32_t> all((size_t)N.ngroups);
    for (int32_t g = 0; g < N.ngroups; ++g) all[(size_t)g] = g;
    int64_t *d_rowptr = nullptr, *d_grow = nullptr, *d_gcp = nullptr;
    int32_t *d_entpos = nullptr, *d_gcols = nullptr;
    CK(dev_upload(c, &d_rowptr, hrow));
    CK(dev_upload(c, &d_entpos, entpos));
    int32_t* d_hcol = nullptr;
    CK(dev_upload(c, &d_hcol, hcol));
    CK(dev_upload(c, &d_grow, N.grp_row));
    CK(dev_upload(c, &d_gcp, gcolptr));
    CK(dev_upload(c, &d_gcols, gcols));
    CK(dev_upload(c, &N.d_groups, all));
    CK(dev_alloc(c, &N.d_sel, (size_t)std::max<int32_t>(N.ngroups, 1)));
    CK(dev_alloc(c, &N.d_flag, 1));
    CK(dev_alloc(c, &N.d_mark, (size_t)std::max<int32_t>(n, 1)));
    CK(dev_alloc(c, &N.d_hv, (size_t)std::max<int64_t>(nnzh, 1)));
    CK(dev_alloc(c, &N.d_w, (size_t)std::max<int64_t>(nrows, 1)));
    CK(dev_alloc(c, &N.d_y, (size_t)std::max<int64_t>(nrows, 1)));
    CK(dev_alloc(c, &N.d_nv, (size_t)std::max<int64_t>(c->S.nnz_a, 1)));
    CK(dev_alloc(c, &N.d_b, (size_t)std::max<int32_t>(n, 1)));
    if (!c->d_cp) CK(dev_upload(c, &c->d_cp, c->in_colptr));
    if (!c->d_ri) CK(dev_upload(c, &c->d_ri, c->in_rowind));
    int64_t* d_pairptr = nullptr;
    int32_t* d_pairpos = nullptr;
    if (table) {
        CK(dev_upload(c, &d_pairptr, pairptr));
        CK(dev_upload(c, &d_pairpos, pairpos));
    }
    N.args = NormalArgs{d_rowptr, d_hcol, d_entpos, d_grow, d_gcp, d_gcols, c->d_cp, c->d_ri, d_pairptr, d_pairpos};
    int32_t max_cols = 1;
    for (int32_t g = 0; g < N.ngroups; ++g)
        max_cols = std::max<int32_t>(max_cols, (int32_t)(gcolptr[(size_t)g + 1] - gcolptr[(size_t)g]));
    N.smem = normal_smem_bytes(max_dense, max_rows, max_cols);
    if (N.smem > 200 * 1024) return SPI_ERR_ARG;  // a row with too many entries for one CTA's list
    CK(normal_kernel_setup(N.smem));
    N.ready = true;
    return SPI_OK;
}

namespace {
// Device copies of the caller's inputs (or the caller's own device buffers).
int normal_inputs(spi_ctx* c, const double* hvals, const double* w, const double* y, int on_device,
                  cudaStream_t st, const double** hv, const double** wd, const double** yd) {
    auto& N = c->nrm;
    if (on_device) {
        *hv = hvals; *wd = w; *yd = y;
        return SPI_OK;
    }
    CK(cudaMemcpyAsync(N.d_hv, hvals, (size_t)N.nnzh * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(N.d_w, w, (size_t)N.nrows * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(N.d_y, y, (size_t)N.nrows * sizeof(double), cudaMemcpyHostToDevice, st));
    *hv = N.d_hv; *wd = N.d_w; *yd = N.d_y;
    return SPI_OK;
}

int normal_finish(spi_ctx* c, double* nvals, double* b, int on_device, cudaStream_t st) {
    auto& N = c->nrm;
    int flag = 0;
    if (!on_device) {
        CK(cudaMemcpyAsync(nvals, N.d_nv, (size_t)c->S.nnz_a * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(b, N.d_b, (size_t)c->S.n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(&flag, N.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return flag ? SPI_ERR_PATTERN : SPI_OK;
}
}  // namespace

int spi_normal_assemble(spi_ctx* c, const double* hvals, const double* w, const double* y, double* nvals,
                        double* b, int on_device, void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->nrm.ready) return SPI_ERR_STATE;
    auto& N = c->nrm;
    if (!nvals || !b || (N.nnzh > 0 && !hvals) || (N.nrows > 0 && (!w || !y))) return SPI_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const double *hv, *wd, *yd;
    int rc = normal_inputs(c, hvals, w, y, on_device, st, &hv, &wd, &yd);
    if (rc) return rc;
    double* nv = on_device ? nvals : N.d_nv;
    double* bv = on_device ? b : N.d_b;
    CK(cudaMemsetAsync(nv, 0, (size_t)c->S.nnz_a * sizeof(double), st));
    CK(cudaMemsetAsync(bv, 0, (size_t)c->S.n * sizeof(double), st));
    CK(cudaMemsetAsync(N.d_flag, 0, sizeof(int), st));
    launch_normal(N.args, N.d_groups, N.ngroups, hv, wd, yd, nullptr, nullptr, false, nv, bv, N.d_flag, N.smem, st);
    return normal_finish(c, nvals, b, on_device, st);
}

int spi_normal_update(spi_ctx* c, int64_t ncols, const int32_t* cols, const double* hvals, const double* w,
                      const double* y, double* nvals, double* b, int on_device, void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->nrm.ready) return SPI_ERR_STATE;
    auto& N = c->nrm;
    const int32_t n = c->S.n;
    if (ncols < 0 || (ncols > 0 && !cols) || !nvals || !b || (N.nnzh > 0 && !hvals) || (N.nrows > 0 && (!w || !y)))
        return SPI_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uint8_t> mark((size_t)std::max<int32_t>(n, 1), 0);
    std::vector<char> gsel((size_t)N.ngroups, 0);
    std::vector<int32_t> sel;
    for (int64_t t = 0; t < ncols; ++t) {
        const int32_t j = cols[t];  // caller numbering, host memory
        if (j < 0 || j >= n) return SPI_ERR_ARG;
        if (mark[(size_t)j]) continue;
        mark[(size_t)j] = 1;
        for (int64_t p = N.hcp[(size_t)j]; p < N.hcp[(size_t)j + 1]; ++p) {
            const int32_t g = N.row_grp[(size_t)N.hri[(size_t)p]];
            if (!gsel[(size_t)g]) { gsel[(size_t)g] = 1; sel.push_back(g); }
        }
    }
    const double *hv, *wd, *yd;
    int rc = normal_inputs(c, hvals, w, y, on_device, st, &hv, &wd, &yd);
    if (rc) return rc;
    double* nv = on_device ? nvals : N.d_nv;
    double* bv = on_device ? b : N.d_b;
    if (!on_device) {  // the previous N and b are updated in place
        CK(cudaMemcpyAsync(nv, nvals, (size_t)c->S.nnz_a * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(bv, b, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(N.d_flag, 0, sizeof(int), st));
    if (!sel.empty()) {
        CK(cudaMemcpyAsync(N.d_mark, mark.data(), (size_t)n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(N.d_sel, sel.data(), sel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        launch_normal(N.args, N.d_sel, (int32_t)sel.size(), hv, wd, yd, nullptr, N.d_mark, true, nv, bv, N.d_flag,
                      N.smem, st);
        launch_normal(N.args, N.d_sel, (int32_t)sel.size(), hv, wd, yd, nullptr, N.d_mark, false, nv, bv, N.d_flag,
                      N.smem, st);
    }
    return normal_finish(c, nvals, b, on_device, st);
}

namespace {
// Newton's work vectors (spi_mle_newton, spi_background_fit)
struct MleWork {
    double *xc, *xt, *dx, *gx, *e, *w, *v, *acc;
};

int mle_work(spi_ctx* c, MleWork* W) {
    const int64_t n1 = std::max<int64_t>(c->S.n, 1), m1 = std::max<int64_t>(c->nrm.nrows, 1);
    if (!c->d_mle) CK(dev_alloc(c, &c->d_mle, (size_t)(4 * n1 + 3 * m1 + 2)));
    W->xc = c->d_mle;
    W->xt = W->xc + n1;
    W->dx = W->xt + n1;
    W->gx = W->dx + n1;
    W->e = W->gx + n1;
    W->w = W->e + m1;
    W->v = W->w + m1;
    W->acc = W->v + m1;
    return SPI_OK;
}

// e = H xs; hacc = {C(xs), rows with e <= 0}; with weights also w = y/e^2, v = y/e - 1
int mle_model(spi_ctx* c, const MleWork& W, const double* hv, const double* yd, const double* xs, bool weights,
              double* hacc, cudaStream_t st) {
    auto& N = c->nrm;
    launch_spmv_rows(N.nrows, N.args.rowptr, N.args.colind, hv, xs, W.e, st);
    CK(cudaMemsetAsync(W.acc, 0, 2 * sizeof(double), st));
    launch_mle_rows(N.nrows, W.e, yd, weights ? W.w : nullptr, W.v, W.acc, st);
    CK(cudaMemcpyAsync(hacc, W.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SPI_OK;
}

// the Hessian H^T diag(w) H into N's values and factored; H^T v into gx
int mle_hessian(spi_ctx* c, const MleWork& W, const double* hv, const double* yd, cudaStream_t st) {
    auto& N = c->nrm;
    CK(cudaMemsetAsync(N.d_nv, 0, (size_t)c->S.nnz_a * sizeof(double), st));
    CK(cudaMemsetAsync(W.gx, 0, (size_t)c->S.n * sizeof(double), st));
    CK(cudaMemsetAsync(N.d_flag, 0, sizeof(int), st));
    launch_normal(N.args, N.d_groups, N.ngroups, hv, W.w, yd, W.v, nullptr, false, N.d_nv, W.gx, N.d_flag, N.smem, st);
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, N.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) return SPI_ERR_PATTERN;
    return factor_impl(c, 1, N.d_nv, 1, st);
}

// Newton's method for the Cash statistic from W.xc, the fit left in W.xc
int mle_fit(spi_ctx* c, const MleWork& W, const double* hv, const double* yd, int max_iter, double tol,
            cudaStream_t st) {
    const int32_t n = c->S.n;
    double hacc[2];
    int rc = mle_model(c, W, hv, yd, W.xc, true, hacc, st);
    if (rc) return rc;
    if (hacc[1] != 0.0) return SPI_ERR_ARG;  // the model must be positive at the start
    double cx = hacc[0];
    c->mle_steps = 0;
    for (int it = 0; it < max_iter; ++it) {
        rc = mle_hessian(c, W, hv, yd, st);
        if (rc) return rc;
        rc = solve_impl(c, 1, W.gx, W.dx, 1, st);
        if (rc) return rc;
        double t = 1.0, ct = cx;
        bool ok = false;
        for (int h = 0; h < 60 && !ok; ++h, t *= 0.5) {
            launch_step(n, W.xc, W.dx, t, W.xt, st);
            rc = mle_model(c, W, hv, yd, W.xt, false, hacc, st);
            if (rc) return rc;
            ct = hacc[0];
            ok = hacc[1] == 0.0 && ct <= cx + 1e-12 * std::fabs(cx);  // C's rounding level
            if (ok) break;
        }
        if (!ok) break;  // no step keeps e > 0 and C from growing: stop at the current x
        CK(cudaMemsetAsync(W.acc, 0, 2 * sizeof(double), st));
        launch_norms2(n, W.dx, W.xt, W.acc, 1, st);
        CK(cudaMemcpyAsync(hacc, W.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(W.xc, W.xt, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
        cx = ct;
        c->mle_steps++;
        if (t * std::sqrt(hacc[0]) <= tol * std::sqrt(hacc[1])) break;
        rc = mle_model(c, W, hv, yd, W.xc, true, hacc, st);  // weights at the new point
        if (rc) return rc;
    }
    c->mle_cash = cx;
    return SPI_OK;
}

// diag(Hess^-1) at W.xc into var
int mle_variances(spi_ctx* c, const MleWork& W, const double* hv, const double* yd, double* var, int on_device,
                  cudaStream_t st) {
    double hacc[2];
    int rc = mle_model(c, W, hv, yd, W.xc, true, hacc, st);
    if (rc) return rc;
    rc = mle_hessian(c, W, hv, yd, st);
    if (rc) return rc;
    return diag_impl(c, 1, nullptr, 0, var, on_device, st);
}
}  // namespace

int spi_mle_newton(spi_ctx* c, const double* hvals, const double* y, double* x, int max_iter, double tol,
                   double* var, int on_device, void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->nrm.ready) return SPI_ERR_STATE;
    auto& N = c->nrm;
    const int32_t n = c->S.n;
    const int64_t M = N.nrows;
    if (max_iter < 0 || !x || (N.nnzh > 0 && !hvals) || (M > 0 && !y)) return SPI_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MleWork W;
    int rc = mle_work(c, &W);
    if (rc) return rc;
    const double *hv = hvals, *yd = y;
    if (!on_device) {
        CK(cudaMemcpyAsync(N.d_hv, hvals, (size_t)N.nnzh * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(N.d_y, y, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, st));
        hv = N.d_hv;
        yd = N.d_y;
    }
    CK(cudaMemcpyAsync(W.xc, x, (size_t)n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    rc = mle_fit(c, W, hv, yd, max_iter, tol, st);
    if (rc) return rc;
    if (var) {
        rc = mle_variances(c, W, hv, yd, var, on_device, st);
        if (rc) return rc;
    }
    CK(cudaMemcpyAsync(x, W.xc, (size_t)n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return finish(c, st);
}

// Newton's method inside each solve of spi_background_fit's likelihood form
constexpr int kFitNewtonSteps = 30;
constexpr double kFitNewtonTol = 1e-12;

int spi_background_fit(spi_ctx* c, int64_t k0, const int32_t* upat, const double* t, int32_t npat, double* hvals,
                       const double* w, const double* y, double* U, double* x, int mode, int max_iter, double tol,
                       double* stat, double* var, int on_device, void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->nrm.ready) return SPI_ERR_STATE;
    auto& N = c->nrm;
    const int32_t n = c->S.n;
    const int64_t M = N.nrows;
    if (k0 < 0 || k0 > n || npat < 1 || npat > SPI_PATTERN_MAX || (mode != SPI_FIT_LSQ && mode != SPI_FIT_MLE) ||
        max_iter < 1 || !(tol >= 0.0) || !U || !x || (N.nnzh > 0 && !hvals) ||
        (M > 0 && (!w || !y || !upat || !t)))
        return SPI_ERR_ARG;
    const bool mle = mode == SPI_FIT_MLE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t m1 = std::max<int64_t>(M, 1), n1 = std::max<int32_t>(n, 1);
    auto& B = c->bg;
    if (!B.pos) {
        CK(dev_alloc(c, &B.pos, (size_t)m1));
        CK(dev_alloc(c, &B.pat, (size_t)m1));
        CK(dev_alloc(c, &B.vec, (size_t)(m1 + 4 * SPI_PATTERN_MAX + n1 + 2)));
    }
    double* td = B.vec;                     // t (host inputs)
    double* Ud = td + m1;                   // the pattern in use
    double* Up = Ud + SPI_PATTERN_MAX;      // the previous solve's pattern
    double* sums = Up + SPI_PATTERN_MAX;    // [2 SPI_PATTERN_MAX]
    double* xp = sums + 2 * SPI_PATTERN_MAX;  // the previous solve's x
    double* acc = xp + n1;
    MleWork W;
    int rc = mle_work(c, &W);
    if (rc) return rc;
    double* xc = W.xc;  // the current solve's x
    // device views of the inputs (H's values are rewritten in place: the caller's
    // buffer on the device, the context's copy otherwise)
    double* hv = hvals;
    const double *wd = w, *yd = y, *tv = t;
    const int32_t* pv = upat;
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (!on_device) {
        CK(cudaMemcpyAsync(N.d_hv, hvals, (size_t)N.nnzh * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(N.d_w, w, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(N.d_y, y, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(td, t, (size_t)M * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(B.pat, upat, (size_t)M * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        hv = N.d_hv; wd = N.d_w; yd = N.d_y; tv = td; pv = B.pat;
    }
    CK(cudaMemcpyAsync(Ud, U, (size_t)npat * sizeof(double), in, st));
    // each row's background entry, checked against its pattern index
    CK(cudaMemsetAsync(N.d_flag, 0, sizeof(int), st));
    launch_bg_locate(M, N.args.rowptr, N.args.colind, (int32_t)k0, pv, npat, B.pos, N.d_flag, st);
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, N.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) return SPI_ERR_ARG;
    launch_bg_write(M, B.pos, pv, tv, Ud, hv, st);
    // the row groups that hold the background columns (their update after U changes)
    std::vector<uint8_t> mark((size_t)n1, 0);
    std::vector<char> gsel((size_t)std::max(N.ngroups, 1), 0);
    std::vector<int32_t> sel;
    for (int32_t j = 0; j < (int32_t)k0; ++j) {
        mark[(size_t)j] = 1;
        for (int64_t p = N.hcp[(size_t)j]; p < N.hcp[(size_t)j + 1]; ++p) {
            const int32_t g = N.row_grp[(size_t)N.hri[(size_t)p]];
            if (!gsel[(size_t)g]) { gsel[(size_t)g] = 1; sel.push_back(g); }
        }
    }
    if (!sel.empty()) {
        CK(cudaMemcpyAsync(N.d_mark, mark.data(), (size_t)n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(N.d_sel, sel.data(), sel.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    const size_t nvb = (size_t)c->S.nnz_a * sizeof(double), nb8 = (size_t)n * sizeof(double);
    // N and b of the current H: all of them, or the background columns' rows and columns
    auto normal = [&](bool full) -> int {
        CK(cudaMemsetAsync(N.d_flag, 0, sizeof(int), st));
        if (full) {
            CK(cudaMemsetAsync(N.d_nv, 0, nvb, st));
            CK(cudaMemsetAsync(N.d_b, 0, nb8, st));
            launch_normal(N.args, N.d_groups, N.ngroups, hv, wd, yd, nullptr, nullptr, false, N.d_nv, N.d_b,
                          N.d_flag, N.smem, st);
        } else if (!sel.empty()) {
            launch_normal(N.args, N.d_sel, (int32_t)sel.size(), hv, wd, yd, nullptr, N.d_mark, true, N.d_nv, N.d_b,
                          N.d_flag, N.smem, st);
            launch_normal(N.args, N.d_sel, (int32_t)sel.size(), hv, wd, yd, nullptr, N.d_mark, false, N.d_nv,
                          N.d_b, N.d_flag, N.smem, st);
        }
        int fl = 0;
        CK(cudaMemcpyAsync(&fl, N.d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return fl ? SPI_ERR_PATTERN : SPI_OK;
    };
    // N and b in the context's scratch: 0 = to assemble, 1 = to update after U
    // changed, 2 = those of the current H
    int nstate = 0;
    auto make_normal = [&]() -> int {
        if (nstate == 2) return SPI_OK;
        int r = normal(nstate == 0);
        if (r == SPI_OK) nstate = 2;
        return r;
    };
    // the weighted least-squares solution of the current H into xc
    auto lsq = [&]() -> int {
        int r = make_normal();
        if (r) return r;
        r = factor_impl(c, 1, N.d_nv, 1, st);
        if (r) return r;
        return solve_impl(c, 1, N.d_b, xc, 1, st);
    };
    // the statistic at (U, xc) (into hacc) and the pattern's sums (into sums)
    double hacc[2];
    auto statistic = [&]() -> int {
        CK(cudaMemsetAsync(sums, 0, 2 * (size_t)npat * sizeof(double), st));
        CK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
        launch_bg_sums(mle, M, N.args.rowptr, N.args.colind, hv, xc, (int32_t)k0, B.pos, pv, tv, yd, wd, npat, sums,
                       acc, st);
        CK(cudaMemcpyAsync(hacc, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return SPI_OK;
    };
    c->bg_iters = 0;
    bool restore = false, have_x = false;
    double prev = 0.0;
    for (int it = 0; it < max_iter; ++it) {
        if (!mle) {
            rc = lsq();
            if (rc) return rc;
        } else {
            // the Newton fit starts from the previous x where the model is positive
            // there, else from the least-squares solution
            bool start_ok = false;
            if (have_x) {
                rc = mle_model(c, W, hv, yd, xc, false, hacc, st);
                if (rc) return rc;
                start_ok = hacc[1] == 0.0;
            }
            if (!start_ok) {
                rc = lsq();
                if (rc) return rc;
            }
            rc = mle_fit(c, W, hv, yd, kFitNewtonSteps, kFitNewtonTol, st);
            nstate = 0;  // the Hessians overwrote N's values
            if (rc) return rc;
        }
        have_x = true;
        rc = statistic();
        if (rc) return rc;
        if (mle && hacc[1] != 0.0) return SPI_ERR_ARG;
        const double sv = hacc[0];
        if (stat) stat[it] = sv;
        c->bg_iters = it + 1;
        c->bg_stat = sv;
        if (it > 0 && sv >= prev - tol * std::fabs(prev)) {
            restore = sv > prev;
            break;
        }
        if (it == max_iter - 1) break;
        prev = sv;
        // keep this solve's pair, then the pattern from x and H's background entries
        CK(cudaMemcpyAsync(Up, Ud, (size_t)npat * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(xp, xc, nb8, cudaMemcpyDeviceToDevice, st));
        launch_bg_pattern(npat, sums, Ud, st);
        launch_bg_write(M, B.pos, pv, tv, Ud, hv, st);
        if (nstate == 2) nstate = 1;
    }
    if (restore) {  // the previous solve was the better one: its pair, H and factor
        CK(cudaMemcpyAsync(Ud, Up, (size_t)npat * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(xc, xp, nb8, cudaMemcpyDeviceToDevice, st));
        launch_bg_write(M, B.pos, pv, tv, Ud, hv, st);
        c->bg_stat = prev;
        if (!mle) {
            nstate = 1;
            rc = make_normal();
            if (rc) return rc;
            rc = factor_impl(c, 1, N.d_nv, 1, st);
            if (rc) return rc;
        }
    }
    if (var) {
        rc = mle ? mle_variances(c, W, hv, yd, var, on_device, st) : diag_impl(c, 1, nullptr, 0, var, on_device, st);
        if (rc) return rc;
    }
    const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(x, xc, nb8, out, st));
    CK(cudaMemcpyAsync(U, Ud, (size_t)npat * sizeof(double), out, st));
    if (!on_device)
        CK(cudaMemcpyAsync(hvals, N.d_hv, (size_t)N.nnzh * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return finish(c, st);
}

int spi_info(const spi_ctx* c, spi_stats* o) {
    if (!c || !o) return SPI_ERR_ARG;
    std::memset(o, 0, sizeof *o);
    const Symbolic& S = c->S;
    o->n = S.n;
    o->nnz_a = S.nnz_a;
    o->nnz_l = S.nnz_l;
    o->nnz_l_stored = S.nnz_l_stored;
    o->n_supernodes = S.ns;
    o->n_levels = S.nlevels;
    o->max_front = S.max_front;
    o->bad_pivot = c->bad_pivot;
    o->bad_band = c->bad_band;
    o->factor_flops = S.factor_flops;
    o->diag_flops = c->last_diag_flops;
    o->solve_flops = 4.0 * (double)S.nnz_l + (double)S.n;
    o->diag_flops_all = S.diag_flops_all;
    o->diag_work_flops = c->last_diag_work;
    o->device_bytes = c->device_bytes;
    o->launches_factor = 2 + c->FP.n_kernel_launches + (mixed_of(c) ? 1 : 0);
    o->launches_factor_fused = c->FP.n_fused_launches;
    o->launches_factor_tc = c->FP.n_tc_launches;
    o->tiles_factor_tc = c->FP.n_tc_tiles;
    o->factor_tc_flops = c->FP.tc_flops;
    o->factor_work_flops = c->FP.work_flops;
    o->factor_dag_tasks = (int64_t)c->FP.dag.size();
    o->factor_dag_levels = c->FP.dag_levels;
    o->tune_ms_launches = c->tune_dag_ms[0];
    o->tune_ms_dag = c->tune_dag_ms[1];
    o->solve_dag_tasks = c->solve_dag == 1 ? (int64_t)c->SP.dag.size() : 0;
    o->tune_solve_ms_launches = c->tune_solve_ms[0];
    o->tune_solve_ms_dag = c->tune_solve_ms[1];
    if (c->solve_dag == 1) o->launches_solve = S.n ? 4 : 0;
    o->pivots_2x2 = c->piv_2x2;
    o->pivot_delays = c->piv_delays;
    o->pivot_restarts = c->piv_restarts;
    o->diag_tc_supernodes = c->dtc.ntc;
    o->diag_tc_tiles = c->dtc.npt;
    o->diag_tc_flops = c->last_diag_tc_flops;
    o->tune_source = c->tune_source;
    o->tune_seconds = c->tune_seconds;
    o->tune_panel_buckets = c->tune_panel_buckets;
    o->tune_panel_fused = c->tune_panel_fused;
    o->tune_schur_buckets = c->tune_schur_buckets;
    o->tune_schur_tc = c->tune_schur_tc;
    int64_t ls = 0;
    for (const Launch& l : c->SP.fwd_launches) ls += l.count > 0;
    for (const Launch& l : c->SP.bwd_launches) ls += l.count > 0;
    o->launches_solve = S.n ? 2 + ls : 0;
    o->launches_diag = S.n ? 1 : 0;
    o->refine_steps = c->refine_steps;
    o->solve_relres = c->solve_relres;
    o->rhs_block = c->rhs_block_used > 0 ? c->rhs_block_used : c->opt.rhs_block;
    o->analyse_seconds = c->analyse_seconds;
    o->mle_steps = c->mle_steps;
    o->mle_cash = c->mle_cash;
    o->bg_iters = c->bg_iters;
    o->bg_stat = c->bg_stat;
    return SPI_OK;
}

int spi_sync(spi_ctx* c, void* stream) {
    if (!c) return SPI_ERR_ARG;
    if (!c->dev_ready) return SPI_OK;
    const int async = c->opt.async;
    c->opt.async = 0;
    int rc = finish(c, (cudaStream_t)stream);
    c->opt.async = async;
    return rc;
}

int spi_get_perm(const spi_ctx* c, int32_t* perm) {
    if (!c || (!perm && c->S.n)) return SPI_ERR_ARG;
    if (c->S.n) std::memcpy(perm, c->S.perm.data(), (size_t)c->S.n * sizeof(int32_t));
    return SPI_OK;
}

int spi_get_etree(const spi_ctx* c, int32_t* parent) {
    if (!c || (!parent && c->S.n)) return SPI_ERR_ARG;
    if (c->S.n) std::memcpy(parent, c->S.parent.data(), (size_t)c->S.n * sizeof(int32_t));
    return SPI_OK;
}

int spi_diag_inverse_noalloc(const spi_ctx* c, const int32_t* idx, int64_t nidx, double* out, void* stream) {
    if (!c || nidx < 0 || (nidx > 0 && (!idx || !out)) || c->opt.pivoting) return SPI_ERR_ARG;
    const int64_t n = c->S.n;
    const int64_t fixed = 1 + (n + 1) / 2;
    if (fixed + n > kNoAllocScratchDoubles) return SPI_ERR_SCRATCH;  // not even one work vector fits
    if (!c->factored) return SPI_ERR_STATE;
    if (nidx == 0 || n == 0) return SPI_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return SPI_ERR_CUDA;
    if (dev != c->device) return SPI_ERR_ARG;
    // An error the caller left pending is reported, and left pending for the caller,
    // rather than taken for one of these launches (cudaPeekAtLastError does not clear it).
    if (cudaPeekAtLastError() != cudaSuccess) return SPI_ERR_CUDA;
    // once per device, with that device current (this first call must not be inside a stream capture)
    double* scratch = noalloc_scratch(dev);
    if (!scratch) return SPI_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t slots = std::min<int64_t>({(kNoAllocScratchDoubles - fixed) / n, nidx, 1024});
    k_noalloc_prepare<<<256, 256, 0, st>>>(c->dsym.perm, (int32_t)n, scratch, slots * n);
    if (cudaGetLastError() != cudaSuccess) return SPI_ERR_CUDA;
    k_diag_inv_noalloc<<<(int)slots, 256, 0, st>>>(c->dsym, c->d_L, c->d_D, idx, nidx, out, scratch);
    if (cudaGetLastError() != cudaSuccess) return SPI_ERR_CUDA;
    double flag = 0.0;
    if (cudaMemcpyAsync(&flag, scratch, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SPI_ERR_CUDA;
    return flag != 0.0 ? SPI_ERR_ARG : SPI_OK;
}

void spi_destroy(spi_ctx* c) {
    if (!c) return;
    free_plan(c->plan_all);
    free_plan(c->plan_sub);
    free_plan(c->plan_blk);
    free_factor_plan(c->dfp);
    if (c->d_zg) cudaFree(c->d_zg);
    for (auto& kv : c->g_factor) cudaGraphExecDestroy(kv.second);
    for (auto& kv : c->g_solve) cudaGraphExecDestroy(kv.second);
    for (auto& kv : c->g_solve_dag) cudaGraphExecDestroy(kv.second);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (void* p : c->allocs) cudaFree(p);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_norm) cudaFreeHost(c->h_norm);
    delete c;
}

}  // extern "C"
