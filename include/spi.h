/*
 * spi.h -- C ABI of the GB300 sparse LDL^T / variance library.
 *
 * The library solves the weighted least-squares normal equations
 * N x = b, N = H^T W H (paper Sec. 2.4.1, Eq. 7), and returns the variances
 * diag(N^-1) (Eq. 8) without forming N^-1.  It follows the three phases of a
 * sparse direct solver (Sec. 3.2): analysis (ordering, elimination tree,
 * symbolic factorization), numerical factorization (multifrontal, in
 * postorder, Sec. 3.2.2) and solution (Sec. 3.2.3), plus the selected-
 * inverse step of Sec. 3.3.1: (N^-1)_ii = || D^-1/2 L^-1 e_i ||^2 computed
 * by forward solves pruned to the elimination-tree path i -> root, with the
 * right-hand sides grouped in blocks (Sec. 3.3.1, last paragraph).
 *
 * Conventions for every call:
 *   - Indices are 0-based and refer to the caller's (unpermuted) numbering.
 *   - Return value: SPI_OK (0) or one of the spi_status codes below; the
 *     message for a code is spi_strerror(code).  On error no output buffer is
 *     guaranteed to hold meaningful data.
 *   - Pointers passed in are borrowed for the duration of the call only; the
 *     library keeps no caller pointer.  Host pointers are ordinary CPU memory;
 *     device pointers are CUDA global memory of the context's device.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it; every call returns after checking the device
 *     status word, i.e. after the stream has drained, unless the context was
 *     created with spi_options.async = 1 (then only the final call of a
 *     sequence reports device-side errors; see spi_sync).
 *   - The numeric path runs only in this library's CUDA kernels (sm_103a);
 *     there is no CPU fallback.  Without a usable GPU, calls that need one
 *     return SPI_ERR_CUDA.
 */
#ifndef SPI_H
#define SPI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spi_status {
    SPI_OK = 0,
    SPI_ERR_ARG = 1,      /* NULL pointer, negative size, index out of range, bad option */
    SPI_ERR_PATTERN = 2,  /* pattern not lower CSC with sorted rows, no duplicate, full diagonal */
    SPI_ERR_NOT_SPD = 3,  /* non-positive pivot; spi_info().bad_pivot holds the column */
    SPI_ERR_OOM = 4,      /* host or device allocation failed */
    SPI_ERR_CUDA = 5,     /* CUDA runtime error (no device, launch failure, ...) */
    SPI_ERR_TIMEOUT = 6,  /* a bounded device-side wait gave up */
    SPI_ERR_STATE = 7,    /* call out of order (factor before analyse, solve before factor) */
    SPI_ERR_SCRATCH = 8   /* problem too large for the fixed scratch of spi_diag_inverse_noalloc */
} spi_status;

typedef enum spi_precision {
    SPI_PREC_FP64 = 0,      /* every step in FP64 */
    SPI_PREC_MIXED_FP32 = 1 /* FP64 diagonal blocks, FP32 panels / Schur updates / variance
                               solves with FP64 variance accumulation, FP64 refinement of x */
} spi_precision;

typedef enum spi_ordering {
    SPI_ORDER_ND = 0,       /* nested dissection (default; Sec. 3.2.1 uses nested dissection) */
    SPI_ORDER_NATURAL = 1   /* the caller's order */
} spi_ordering;

typedef struct spi_options {
    int precision;   /* spi_precision */
    int ordering;    /* spi_ordering */
    int rhs_block;   /* right-hand sides per block in spi_diag_inverse, 1..512 (rounded up to a
                        multiple of 8 in mixed precision); 0 = automatic: the first variance call
                        times a few candidate sizes on the factor and keeps the fastest (32 in
                        FP64, 64-128 in mixed precision on the SPI workloads; Sec. 4.3 groups 128
                        right-hand sides on a CPU core) */
    int relax;       /* supernode amalgamation: max explicit zeros per parent-child merge as a
                        percentage of the merged panel, plus merges of very small supernodes and
                        grouping of sibling leaf fronts; 0 = fundamental supernodes only;
                        default 1 (explicit zeros are paid again by every variance path that
                        crosses them) */
    int refine_max;  /* max iterative-refinement steps of spi_solve in mixed precision */
    double refine_tol; /* stop refining when ||b - N x||_2 <= refine_tol * ||b||_2 */
    int async;       /* 1: do not drain the stream at the end of each call */
    int nd_leaf;     /* nested-dissection leaf size (vertices); 0 = default */
    int batch;       /* maximum number of same-pattern bands of the *_batch calls (device memory
                        is sized for it at the first factorization); 0 or 1 = single problem */
    int wait_limit;  /* polls allowed to each bounded device wait of spi_factor: the pipeline
                        waits of the tensor-core kernels (mixed form; default 2^20) and the
                        dependency waits of the dependency-driven launch (default 2^25, about
                        100 ns apart): 0 = those defaults, > 0 = that many, < 0 = none, so every
                        such wait gives up at once and spi_factor returns SPI_ERR_TIMEOUT (a
                        test of that path).  After giving up, a tensor-core kernel still waits,
                        with the default limit, for its own MMAs in flight before it frees its
                        tensor memory; the dependency-driven launch skips its remaining tasks */
    int diag_ctas_per_sm;  /* 0 = the variance kernels of spi_diag_inverse take every SM
                        slot they fit in; k > 0: at most k of their CTAs per
                        SM (their shared memory is padded to enforce it), so that work on
                        another stream -- a spi_solve running concurrently -- keeps room
                        on every SM instead of waiting for variance CTAs to finish */
    int diag_unpruned;   /* 0 = pruned solves (the method); 1 = the pruning ablation: every
                            variance from a full forward solve over all supernodes (32 per
                            pass, FP64 panels), var_i = sum_k z_k^2 / d_k, so that the gain
                            of pruning can be measured (the paper's brute-force comparison,
                            Table 5); spi_diag_inverse only, band 0 only */
    int autotune;    /* how the first spi_factor / spi_factor_batch of a context chooses, per
                        front-size bucket (floor(log2) of a front's rows and pivots), between the
                        panel of a front processed whole by one CTA of a persistent per-level
                        kernel and the tiled chain of 32-column block-step launches, and (mixed
                        precision) between the SIMT and tensor-core Schur complement:
                        0 = time both candidates of every bucket on the caller's values when the
                        factorization is large enough (>= 2e8 flops), else built-in rules;
                        1 = always time; -1 = never time (built-in rules).  Buckets found in
                        tune_cache are not timed again.  The timing costs two extra
                        factorizations, once per context */
    int force_panel; /* 0 = as chosen above; 1 = every panel on the block-step chain; 2 = every
                        panel whose work allows it in the persistent per-level kernel */
    int force_schur; /* 0 = as chosen above; 1 = no tensor-core launch at all (SIMT Schur
                        complements and panel updates); 2 = Schur complements on the tensor
                        cores wherever legal (mixed precision, at least 256 trailing rows and
                        32 pivots) */
    int dag;         /* 0 = as chosen by the autotuner (timed: one dependency-driven launch against
                        launches level by level, for spi_factor at the first factorization and for
                        spi_solve at the first solve), else on; 1 = launches level by level; 2 = the
                        dependency-driven form: spi_factor runs every level below the first one
                        with a tensor-core launch as one persistent kernel whose CTAs take the tasks
                        (pivot tiles, panel-solve chunks, update and Schur tiles, whole small
                        fronts) in a topological order and wait, bounded, for the tasks each
                        depends on; spi_solve runs both sweeps so (forward steps, backward passes
                        over 32 columns, backward steps) */
    const char* tune_cache; /* path of a text file keeping the autotuner's choices across
                        processes (one line per device, precision, batch class and bucket, plus
                        one line each for the factor's and the solve's form and for the
                        variance right-hand-side block), or NULL; each choice is read before it
                        would be timed and the file rewritten after a timing */
    int pivoting;    /* 0 = symmetric positive definite (the pivot-free LDL^T; a non-positive pivot
                        is SPI_ERR_NOT_SPD).  1 = symmetric indefinite (paper Sec. 5): every front
                        factored with restricted Bunch-Kaufman pivoting -- 1x1 and 2x2 pivots
                        chosen among its fully-summed columns, symmetric swaps within them -- and
                        a front that finds no stable pivot there has its pivots delayed to its
                        parent (the analysis is redone with the front merged into its parent's,
                        where its columns are fully summed, and the factorization restarts);
                        only a singular matrix then returns SPI_ERR_NOT_SPD.  D is block
                        diagonal; spi_solve applies it block by block and spi_diag_inverse sums
                        z^T D^-1 z with its 2x2 blocks.  FP64, one problem (batch 1), launches
                        level by level; spi_inverse_block, spi_inverse_entries and
                        spi_diag_inverse_noalloc return SPI_ERR_ARG in this form */
    int diag_tc_min_pivots; /* mixed precision: the variances of the supernodes with at least this
                        many pivots, and of all their ancestors, run on the tensor cores (3 x TF32
                        products of TMA-staged operand tiles prepared at each factorization); the
                        rest of every path on the SIMT kernel; their inverted 128 x 128 diagonal
                        tiles also let the mixed solve take 128 columns per step there.  0 = the
                        default (32); < 0 = none (SIMT variances, 32-column solve steps).
                        Variance blocks of more than 128 right-hand sides (rhs_block > 128) stay
                        on the SIMT kernel */
} spi_options;

typedef struct spi_stats {
    int64_t n;              /* order of N */
    int64_t nnz_a;          /* stored entries of the lower triangle of N */
    int64_t nnz_l;          /* entries of L (strictly lower), exact column counts */
    int64_t nnz_l_stored;   /* entries of the supernodal panels incl. explicit zeros */
    int64_t n_supernodes;
    int64_t n_levels;       /* elimination-tree levels of the supernodal tree */
    int64_t max_front;      /* largest front order m */
    int64_t bad_pivot;      /* column (caller numbering) of the first non-positive pivot, or -1 */
    int64_t bad_band;       /* band of that pivot in a batched factorization, or -1 */
    double factor_flops;    /* sum over pivots j of (c_j^2 - 1), c_j = entries of column j of L
                               including the diagonal (exact counts, no amalgamation zeros) */
    double diag_flops;      /* algorithmic flops of the last spi_diag_inverse call:
                               sum over requested i, over j on path(i), of 2 c_j (0 after a
                               call with spi_options.diag_unpruned) */
    double solve_flops;     /* 4 * nnz_l + n (one forward + one backward sweep) */
    double diag_flops_all;  /* algorithmic flops of spi_diag_inverse over all n indices */
    double diag_work_flops; /* flops the blocked kernel executes for the last spi_diag_inverse
                               (dense over each block's active range, amalgamation zeros; with
                               diag_unpruned, 2 x stored panel entries per index) */
    int64_t device_bytes;   /* device memory held by the context */
    int64_t launches_factor;/* kernels this library launches per spi_factor */
    int64_t launches_solve; /* ... per spi_solve */
    int64_t launches_diag;  /* ... per spi_diag_inverse */
    int64_t refine_steps;   /* refinement steps taken by the last spi_solve (mixed precision) */
    double solve_relres;    /* ||b - N x||_2 / ||b||_2 after the last mixed-precision spi_solve
                               (largest over the bands of a batch) */
    int64_t rhs_block;      /* right-hand sides per block in use (chosen by the autotuner when
                               spi_options.rhs_block = 0) */
    double analyse_seconds; /* host time of spi_analyse */
    int64_t mle_steps;      /* Newton steps of the last spi_mle_newton */
    double mle_cash;        /* its final Cash statistic sum (e - y ln e) */
    int64_t bg_iters;       /* solves made by the last spi_background_fit */
    double bg_stat;         /* the statistic of the pair it returned (chi^2 or Cash) */
    int64_t launches_factor_fused; /* launches of the persistent per-level panel kernel per spi_factor */
    int64_t launches_factor_tc;    /* tensor-core (tcgen05) launches per spi_factor (mixed precision) */
    int64_t tiles_factor_tc;       /* 128 x 128 tensor-core tiles per spi_factor */
    int64_t tune_source;    /* where the factorization's bucket choices came from: 0 built-in rules,
                               1 timed by this context, 2 the tune cache */
    double tune_seconds;    /* host time the timing took */
    int64_t tune_panel_buckets;  /* panel buckets of this tree with a choice to make ... */
    int64_t tune_panel_fused;    /* ... and how many of them run in the persistent kernel */
    int64_t tune_schur_buckets;  /* Schur buckets that may use the tensor cores ... */
    int64_t tune_schur_tc;       /* ... and how many of them do */
    double factor_tc_flops;      /* TF32 flops the tensor cores execute per spi_factor: 2 x 128 x 128 x K
                                    per tile and MMA, 6 MMAs per product (split precision) */
    double factor_work_flops;    /* flops the SIMT kernels of spi_factor execute: whole 32 x 32 tiles
                                    and explicit zeros included (compare factor_flops) */
    int64_t factor_dag_tasks;    /* tasks of the dependency-driven launch (0: none) ... */
    int64_t factor_dag_levels;   /* ... covering the tree levels [0, factor_dag_levels) */
    double tune_ms_launches;     /* the timed factorization with launches level by level ... */
    double tune_ms_dag;          /* ... and with the dependency-driven launch (-1: not timed) */
    int64_t solve_dag_tasks;     /* tasks of the solve's dependency-driven launch, when it is in use */
    double tune_solve_ms_launches; /* the first solve timed with launches level by level ... */
    double tune_solve_ms_dag;      /* ... and with the dependency-driven launch (-1: not timed) */
    int64_t pivots_2x2;     /* 2x2 pivots of the last factorization (spi_options.pivoting) */
    int64_t pivot_delays;   /* fronts whose pivots were delayed to their parents ... */
    int64_t pivot_restarts; /* ... and the factorizations restarted after merging them */
    int64_t diag_tc_supernodes; /* supernodes whose variances run on the tensor cores
                                   (spi_options.diag_tc_min_pivots) */
    int64_t diag_tc_tiles;      /* 128 x 32 operand tiles prepared for them per band */
    double diag_tc_flops;       /* TF32 MMA flops issued by the last spi_diag_inverse (three
                                   products per output, padded tiles) */
} spi_stats;

typedef struct spi_ctx spi_ctx;

/* Fill *opt with the defaults (FP64, nested dissection, automatic RHS block,
 * relax 1, refine_max 10, refine_tol 1e-13, synchronous, batch 1). */
void spi_default_options(spi_options* opt);

/* Analysis phase (Sec. 3.2.1): validate the pattern, order it (nested
 * dissection or natural), build the elimination tree and its postorder,
 * exact column counts, relaxed supernodes, the multifrontal assembly maps
 * and the level schedule.  Host work only; device memory is allocated at the
 * first spi_factor.
 *   n       order of N (>= 0)
 *   colptr  host, int64[n+1]: CSC column pointers of the LOWER triangle
 *           (including the diagonal), colptr[0] = 0
 *   rowind  host, int32[colptr[n]]: row indices, strictly increasing in each
 *           column, each column starting with its diagonal entry
 *   opt     host, may be NULL (defaults)
 *   out     receives the new context (owned by the caller; spi_destroy)
 * Errors: SPI_ERR_ARG (NULL out, n < 0, an option out of range: rhs_block
 * outside 0..512, precision or ordering unknown, relax, refine_max, nd_leaf
 * or diag_ctas_per_sm negative, diag_unpruned not 0 or 1), SPI_ERR_PATTERN,
 * SPI_ERR_OOM. */
int spi_analyse(int64_t n, const int64_t* colptr, const int32_t* rowind,
                const spi_options* opt, spi_ctx** out);

/* Numerical factorization (Sec. 3.2.2): N = P^T L D L^T P with the values of
 * the pattern given to spi_analyse.
 *   values  float64[colptr[n]] in the order of rowind; host memory when
 *           values_on_device = 0, device memory otherwise
 * May be called again with new values on the same pattern (energy bands,
 * Newton steps).  Errors: SPI_ERR_STATE, SPI_ERR_NOT_SPD (spi_info().bad_pivot
 * gives the column; the factor is unusable), SPI_ERR_CUDA, SPI_ERR_OOM. */
int spi_factor(spi_ctx* ctx, const double* values, int values_on_device, void* stream);

/* Solution phase (Sec. 3.2.3): x = N^-1 b by z = L^-1 P b (bottom-up over the
 * tree), w = D^-1 z, x = P^T L^-T w (top-down).  In mixed precision the
 * result is refined in FP64 against the FP64 values of N: x += solve(b - N x)
 * until ||b - N x||_2 <= opt.refine_tol ||b||_2 or opt.refine_max steps.  A
 * call after a converged one first runs as many steps as that one took, with no
 * residual check between them, then checks after every further step.
 *   b, x    float64[n]; host when on_device = 0, device otherwise; x may
 *           alias b.
 * Errors: SPI_ERR_STATE, SPI_ERR_ARG, SPI_ERR_CUDA. */
int spi_solve(spi_ctx* ctx, const double* b, double* x, int on_device, void* stream);

/* Selected inverse entries (Sec. 3.3.1, Sec. 4.3): out[t] = (N^-1)_{idx[t], idx[t]}
 * computed as sum_k z_k^2 / d_k with z = L^-1 P e_idx[t], each forward solve
 * pruned to the elimination-tree path of idx[t]; the requested indices are
 * sorted in postorder and grouped in blocks of opt.rhs_block right-hand
 * sides, every block solved by one CTA over the union of its paths.
 *   idx     int32[nidx] (host when on_device = 0, else device), or NULL for
 *           all n indices (then out[i] = (N^-1)_ii)
 *   out     float64[nidx] (or [n] when idx == NULL), host or device as above
 * Errors: SPI_ERR_STATE, SPI_ERR_ARG (index out of range), SPI_ERR_CUDA. */
int spi_diag_inverse(spi_ctx* ctx, const int32_t* idx, int64_t nidx, double* out,
                     int on_device, void* stream);

/* Uneven independent problems as one batch: problems p = 0..nprob-1, each given
 * like spi_analyse (n[p], colptr[p], rowind[p], host memory), are analysed as
 * the block-diagonal matrix diag(N_0, ..., N_{nprob-1}).  Its elimination
 * tree is the forest of the problems' trees, so every level launch of the
 * factorization, the solves and the variance solves covers all problems at
 * once.  All later calls use the concatenated numbering: values are the
 * problems' value arrays one after another, b, x and the variances likewise.
 * The paper runs many such sequential computations side by side (Sec. 6).
 * Errors: as spi_analyse. */
int spi_analyse_multi(int32_t nprob, const int64_t* n, const int64_t* const* colptr,
                      const int32_t* const* rowind, const spi_options* opt, spi_ctx** out);

/* Same-pattern batch (energy bands of one observation, Sec. 6: the analysis is
 * repeated for 24 energy bands): nbatch <= spi_options.batch value sets of the
 * analysed pattern, factored together; each tree level / block step is one
 * launch over all bands (the band is the second grid dimension), replayed
 * from a CUDA graph.
 *   values  float64[nbatch * nnz], band b at offset b * nnz (host or device)
 * Errors: as spi_factor; SPI_ERR_ARG when nbatch is out of range;
 * spi_info().bad_band names the band of a non-positive pivot. */
int spi_factor_batch(spi_ctx* ctx, int32_t nbatch, const double* values, int values_on_device, void* stream);

/* spi_solve for the first nbatch factored bands: b and x are float64[nbatch * n]. */
int spi_solve_batch(spi_ctx* ctx, int32_t nbatch, const double* b, double* x, int on_device, void* stream);

/* spi_diag_inverse for the first nbatch factored bands: out is
 * float64[nbatch * m] with m = nidx (or n when idx == NULL), band b at b * m. */
int spi_diag_inverse_batch(spi_ctx* ctx, int32_t nbatch, const int32_t* idx, int64_t nidx, double* out,
                           int on_device, void* stream);

/* Most indices of one spi_inverse_block call. */
#define SPI_INVERSE_BLOCK_MAX 512

/* A block of the inverse: out[s * nidx + t] = (N^-1)_{idx[s], idx[t]} (both
 * triangles, row-major), the covariances of the selected unknowns -- "any set
 * of entries" of the inverse (paper Sec. 3.3.1), here a dense index block.
 * Since N^-1 = P^T L^-T D^-1 L^-1 P, entry (s, t) is sum_k z_s[k] z_t[k] / d_k
 * with z_s = L^-1 e_(pivot of idx[s]); the nidx vectors are the pruned
 * forward solves of spi_diag_inverse, in blocks of consecutive pivots along
 * the union of their elimination-tree paths (FP64, also in a mixed-precision
 * context, whose factor is stored in FP64), gathered into one matrix over the
 * union of all their paths, followed by their FP64 Gram product.  No backward
 * pass is needed for a symmetric matrix.  Device memory: that matrix, rows of
 * the union x nidx doubles (at most n x nidx), kept for the next call.
 *   idx   int32[nidx], caller numbering, distinct, 0 <= nidx <= SPI_INVERSE_BLOCK_MAX
 *   out   float64[nidx * nidx]
 * on_device: idx and out are device pointers.  Band 0 of a batched context.
 * The plan is cached per index set.  Errors: SPI_ERR_STATE (not factored),
 * SPI_ERR_ARG (NULL buffer, nidx out of range, an index out of range or
 * repeated), SPI_ERR_OOM, SPI_ERR_CUDA. */
int spi_inverse_block(spi_ctx* ctx, const int32_t* idx, int64_t nidx, double* out, int on_device, void* stream);

/* Variances of a mixed-precision factorization with its first-order error
 * removed, for selected unknowns: out[t] = 2 e_i^T v - v^T N v with i = idx[t]
 * and v = F^-1 e_i computed by full (unpruned) forward and backward sweeps of
 * the factor F (FP32 panels converted to FP64, FP64 arithmetic), N the FP64
 * input matrix.  The quadratic form peaks at v = N^-1 e_i with value
 * (N^-1)_ii, so an error d = O(delta) in v leaves an error -d^T N d = O(delta^2)
 * in the variance (never above the exact one), against O(delta) for
 * spi_diag_inverse.  Cost: one full solve and one product with N per index
 * (32 indices per pass), far more than the pruned solves: meant for the
 * unknowns whose variances matter most, e.g. the sources' fluxes.  An FP64
 * context returns spi_diag_inverse's values.
 *   idx   int32[nidx], caller numbering (repeats allowed)
 *   out   float64[nidx]
 * on_device: idx and out are device pointers.  Band 0 of a batched context.
 * Device memory: about 5 x 32 x n doubles for the call.  Errors: SPI_ERR_STATE
 * (not factored), SPI_ERR_ARG (NULL buffer, an index out of range),
 * SPI_ERR_OOM, SPI_ERR_CUDA. */
int spi_diag_inverse_refined(spi_ctx* ctx, const int32_t* idx, int64_t nidx, double* out, int on_device,
                             void* stream);

/* Scattered entries of the inverse: out[t] = (N^-1)_{rows[t], cols[t]} for any
 * list of index pairs -- "any set of entries" of the inverse (paper
 * Sec. 3.3.1).  The distinct indices of the list, in elimination order, are
 * cut into groups of SPI_INVERSE_BLOCK_MAX / 2; every pair of groups holding a
 * requested entry is computed as one spi_inverse_block of the two groups'
 * indices (the same pruned forward solves and Gram product, FP64), and the
 * entries are picked from it on the device.  Cost: one block per group pair
 * present in the list, so a list concentrated on a few hundred unknowns costs
 * one block, while covariances spread over all n unknowns cost up to
 * (n / 256)^2 / 2 blocks.
 *   rows, cols  int32[nent], caller numbering (pairs may repeat, in either order)
 *   out         float64[nent]
 * on_device: rows, cols and out are device pointers.  Band 0 of a batched
 * context; the block plan cache of spi_inverse_block is reused and replaced.
 * Errors: SPI_ERR_STATE (not factored), SPI_ERR_ARG (NULL buffer, nent < 0, an
 * index out of range), SPI_ERR_OOM, SPI_ERR_CUDA. */
int spi_inverse_entries(spi_ctx* ctx, const int32_t* rows, const int32_t* cols, int64_t nent, double* out,
                        int on_device, void* stream);

/* The normal equations on the device (paper Sec. 4.1, Eq. 7): N = H^T W H on
 * the pattern this context was analysed with, and b = H^T W y, from the design
 * matrix H (rows = observations) -- the step before spi_factor, and its update
 * after the values of some columns of H changed (paper Table 3).
 *
 * spi_normal_setup records H's pattern (host CSR: rowptr int64[nrows + 1],
 * colind int32[rowptr[nrows]], columns ascending within a row, caller
 * numbering of N's unknowns) and groups consecutive rows with nearly the same
 * columns (for SPI, the detectors of one pointing) and tables the positions of
 * their column pairs in N's pattern.  Once per context, made by spi_analyse
 * (one pattern).  Errors: SPI_ERR_ARG, SPI_ERR_PATTERN (bad CSR), SPI_ERR_STATE
 * (a multi-problem context, or a second call), SPI_ERR_OOM, SPI_ERR_CUDA. */
int spi_normal_setup(spi_ctx* ctx, int64_t nrows, const int64_t* rowptr, const int32_t* colind);

/* N's lower-CSC values in the order of the analysed pattern (the values
 * spi_factor takes) and b = H^T W y:
 *   hvals float64[nnz(H)] in the CSR order of spi_normal_setup, w and y
 *   float64[nrows] (weights and observations), nvals float64[nnz(N)],
 *   b float64[n].
 * on_device: every buffer is a device pointer.  FP64 throughout; entries of N
 * are sums of per-group products added with FP64 atomics (their order, and so
 * their last bits, may vary from call to call).  Returns after the stream has
 * drained.  Errors: SPI_ERR_STATE (no setup), SPI_ERR_ARG, SPI_ERR_PATTERN (a
 * nonzero product of H has no place in N's pattern), SPI_ERR_CUDA. */
int spi_normal_assemble(spi_ctx* ctx, const double* hvals, const double* w, const double* y, double* nvals,
                        double* b, int on_device, void* stream);

/* Update nvals and b (as returned by spi_normal_assemble, in place) after the
 * values of H in the columns cols[0..ncols) (host int32, caller numbering)
 * changed: every entry of N in a row or column of those unknowns, and their
 * entries of b, are recomputed from hvals, w, y (the complete new values);
 * only the row groups that hold those columns are visited.  Other arguments
 * and errors as spi_normal_assemble. */
int spi_normal_update(spi_ctx* ctx, int64_t ncols, const int32_t* cols, const double* hvals, const double* w,
                      const double* y, double* nvals, double* b, int on_device, void* stream);

/* Poisson maximum-likelihood fit (the paper's appendix on low counts): minimise
 * the Cash statistic C(x) = sum_i (e_i - y_i ln e_i), e = H x, by Newton's
 * method on the design matrix recorded by spi_normal_setup.  Each step: e = H x
 * on the device, the Hessian H^T diag(y/e^2) H assembled there, factored (in
 * the context's precision) and solved for dx with right-hand side
 * H^T (y/e - 1); the step is halved (at most 60 times) until every e stays
 * positive and C does not increase by more than 1e-12 |C| (its rounding level).  Stops when ||step|| <= tol ||x|| (2-norms)
 * or after max_iter steps; spi_info().mle_steps / mle_cash report them.
 *   hvals float64[nnz(H)] (CSR order of spi_normal_setup), y float64[nrows]
 *   x     float64[n]: in, the start (the least-squares solution is a good one:
 *         e must be positive there); out, the fit
 *   var   float64[n] or NULL: diag(Hess^-1) at the fit (one more assembly,
 *         factorization and spi_diag_inverse)
 * on_device: every buffer is a device pointer.  The factor of the context is
 * the last Hessian's afterwards.  Returns after the stream has drained.
 * Errors: SPI_ERR_STATE (no spi_normal_setup), SPI_ERR_ARG (e <= 0 at the
 * start, max_iter < 0, NULL buffer), and those of spi_normal_assemble,
 * spi_factor and spi_solve. */
int spi_mle_newton(spi_ctx* ctx, const double* hvals, const double* y, double* x, int max_iter, double tol,
                   double* var, int on_device, void* stream);

/* Algorithm 1 of the appendix on the "empty-field" pattern: the background
 * B_dp = U^d I_p^bg t_dp (Eq. A4) has a pattern U that is fitted with the
 * solution.  The first k0 columns of H are the background normalisations
 * (I_p^bg, one per pointing); each row i has at most one entry in them, whose
 * value is U[upat[i]] t[i].  Starting from U, each iteration
 *   1. solves for x with the current H: weighted least squares (mode
 *      SPI_FIT_LSQ: N = H^T W H assembled -- after the first iteration only
 *      its rows and columns of the first k0 unknowns are recomputed --,
 *      factored and solved), or the Poisson likelihood fit (SPI_FIT_MLE:
 *      Newton's method as spi_mle_newton with at most 30 steps and tol 1e-12,
 *      started from the previous x where H x > 0, else from the least-squares
 *      solution);
 *   2. computes the statistic at (U, x): sum w (y - Hx)^2, or the Cash
 *      statistic sum (e - y ln e) = -L/2 + const; stat[it] receives it;
 *   3. stops when it is not below the previous iteration's by more than
 *      tol |previous| (the previous pair is restored when it is above it), or
 *      after max_iter solves;
 *   4. re-estimates each pattern value from x: with y^S the counts of the
 *      columns from k0 on and a_i = t_i x_c(i) (c(i): row i's background
 *      column), U_k = sum (y - y^S) a w / sum a^2 w (least squares) or
 *      sum (y - y^S) / sum a (likelihood, the paper's simplified form), sums
 *      over the rows with upat = k; a value whose denominator is not positive
 *      is kept; then the background entries of H are rewritten.
 * The test follows each solve, before U changes, so the returned U and x are
 * the pair that solve used.
 *   k0      number of background columns (caller numbering 0 .. k0-1)
 *   upat    int32[nrows]: the row's pattern index in 0 .. npat-1 (a detector,
 *           or a detector and an interval of pointings), -1 for a row with no
 *           entry in the first k0 columns
 *   t       float64[nrows]: t_dp of the row (unused where upat = -1)
 *   npat    1 .. SPI_PATTERN_MAX
 *   hvals   float64[nnz(H)], CSR order of spi_normal_setup: in, H (its
 *           background entries are overwritten from U at the start); out, H
 *           at the returned U
 *   w, y    float64[nrows]: least-squares weights (also those of the
 *           likelihood form's least-squares start) and counts
 *   U       float64[npat]: in, U_0; out, the returned pattern
 *   x       float64[n]: out, the returned solution
 *   stat    HOST float64[max_iter] or NULL: the statistic of each solve
 *   var     float64[n] or NULL: diag(Hess^-1) at the returned pair (N, or
 *           H^T diag(y/e^2) H)
 * on_device: hvals, w, y, upat, t, U, x, var are device pointers (stat stays
 * on the host).  The context's factor is that of the returned pair's N (least
 * squares) or of its Hessian (likelihood, with var).  spi_info().bg_iters and
 * bg_stat report the solves made and the returned statistic.  Returns after
 * the stream has drained.  Errors: SPI_ERR_STATE (no spi_normal_setup),
 * SPI_ERR_ARG (k0 outside 0..n, npat outside 1..SPI_PATTERN_MAX, bad mode,
 * max_iter < 1, tol < 0 or NaN, NULL buffer, a row with two entries in the
 * first k0 columns or a pattern index that does not match its row, H x <= 0
 * where the likelihood needs it positive), and those of spi_normal_assemble,
 * spi_factor and spi_solve.  After an error the background entries of hvals
 * (device form) may hold any pattern the loop had reached, and U, x, var are
 * not written. */
#define SPI_PATTERN_MAX 2048
#define SPI_FIT_LSQ 0
#define SPI_FIT_MLE 1
int spi_background_fit(spi_ctx* ctx, int64_t k0, const int32_t* upat, const double* t, int32_t npat,
                       double* hvals, const double* w, const double* y, double* U, double* x, int mode,
                       int max_iter, double tol, double* stat, double* var, int on_device, void* stream);

/* Variances without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need variances -- a host thread that must not enter the CUDA allocator (a
 * real-time loop, a callback of another runtime) or a process whose device
 * memory is already handed out by another allocator.  It computes the same
 * out[t] = (N^-1)_{idx[t], idx[t]} as spi_diag_inverse, one right-hand side
 * per CTA along its elimination-tree path, with its workspace in one fixed
 * 16 MiB array in device memory that every GPU loading this library holds
 * until the process exits; it calls no allocation routine.
 *   ctx     a factored context (spi_factor, or band 0 of spi_factor_batch) whose
 *           device is the current device
 *   idx     device int32[nidx], caller numbering
 *   out     device float64[nidx]
 * Limit: the inverse permutation and one length-n work vector must fit, i.e.
 * n <= 1,398,100; larger problems get SPI_ERR_SCRATCH (checked before any
 * device work).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Host threads may make that first call at
 * the same time (the lookup is serialised).  A CUDA error already pending
 * when the call starts makes it return SPI_ERR_CUDA before any device work and
 * is left pending for the caller.  Every call clears the part of the array it
 * uses before use; calls that overlap on the GPU (other streams, other
 * contexts) share the array and race.  The call returns after the stream has
 * drained.  Errors: SPI_ERR_ARG (NULL buffer, index out of range -- its out[t]
 * is NaN -- or another device current), SPI_ERR_STATE (not factored),
 * SPI_ERR_SCRATCH, SPI_ERR_CUDA. */
int spi_diag_inverse_noalloc(const spi_ctx* ctx, const int32_t* idx, int64_t nidx, double* out, void* stream);

/* Measured throughput of one arithmetic unit of the current device, in
 * TFLOP/s (a multiply-add counts 2), for the roofline denominators of the
 * benchmark; not a step of the method.  unit: 0 FP64 FMA, 1 FP64 mma.sync
 * m8n8k4 (DMMA), 2 FP32 FMA, 3 tcgen05.mma kind::tf32 (M 128, N 256), 4
 * tcgen05.mma kind::f16 with BF16 inputs and FP32 accumulation.  Each probe
 * runs independent operations on every SM for tens of milliseconds; *tflops
 * receives the best of `reps` timed runs after one warm-up run.  The tensor-
 * core probes wait for their MMAs with a bounded wait.  Allocates and frees a
 * small device buffer.  Errors: SPI_ERR_ARG, SPI_ERR_OOM, SPI_ERR_CUDA,
 * SPI_ERR_TIMEOUT. */
int spi_measure_peak(int unit, int reps, double* tflops);

/* Statistics of the analysis and of the last calls.  Errors: SPI_ERR_ARG. */
int spi_info(const spi_ctx* ctx, spi_stats* out);

/* Drain the context's last stream and report any device-side error. */
int spi_sync(spi_ctx* ctx, void* stream);

/* Export the permutation: perm[k] = caller index of the k-th pivot
 * (host int32[n]).  Errors: SPI_ERR_ARG. */
int spi_get_perm(const spi_ctx* ctx, int32_t* perm);

/* Export the elimination tree of the permuted matrix: parent[k] = pivot
 * index of the parent of pivot k, -1 at a root (host int32[n]). */
int spi_get_etree(const spi_ctx* ctx, int32_t* parent);

/* Static message for a status code. */
const char* spi_strerror(int status);

/* Free the context and all its device memory.  NULL is allowed. */
void spi_destroy(spi_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SPI_H */
