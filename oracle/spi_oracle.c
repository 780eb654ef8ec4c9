/*
 * spi_oracle.c -- plain, slow, obviously correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that the tests, the smoke check and the
 * benchmark's CPU-baseline leg can compare the GPU path against an
 * independent computation.  It shares no code, header or table with the
 * CUDA library.
 *
 * What it computes (paper Sec. 2.4.1 Eq. 7-8, Sec. 3.2, Sec. 4.3):
 *   A = N (symmetric, given as its lower triangle in CSC, natural order)
 *   A = L D L^T, L unit lower triangular, D diagonal      (Sec. 3.2)
 *   x = A^{-1} b by z = L^{-1} b, w = D^{-1} z, x = L^{-T} w  (Sec. 3.2.3)
 *   (A^{-1})_ii = sum_k (1/d_kk) (l^{-1}_ki)^2                 (Sec. 4.3)
 *
 * Factorization: left-looking, column by column, in the manner of the
 * sequential LDL package the paper compares against (Sec. 4.3): column j
 * gathers A(j:n, j) into a dense accumulator and subtracts
 * L(:,k) d_k L(j,k) for every earlier column k with L(j,k) != 0.  Those k
 * are found with one linked list per row: a finished column k sits on the
 * list of the next row of its pattern not yet reached.  No ordering is done
 * (natural order); no pivoting is done: a pivot d_j <= 0, or
 * d_j <= 1e-14 * A_jj, stops the factorization and reports column j
 * (the matrices here are SPD by construction; the paper's MUMPS runs use
 * numerical pivoting, which is not part of this path).
 *
 * Inverse diagonal: for each requested i, solve L z = e_i with a dense
 * length-n vector (z_i = 1; the nonzeros of z lie on the elimination-tree
 * path from i to the root, parent(k) = smallest row index > k in L(:,k),
 * Sec. 3.2.1), then (A^{-1})_ii = sum over that path, in ascending k, of
 * z_k^2 / d_k.  The requested indices are split over POSIX threads; this is
 * the only parallelism.
 *
 * Inverse block: for a set I of indices, A^{-1} = L^{-T} D^{-1} L^{-1} gives
 * (A^{-1})_ij = sum_k z_i[k] z_j[k] / d_k with z_i = L^{-1} e_i as above, so
 * the block A^{-1}(I, I) (covariances of the selected unknowns, Sec. 3.3.1:
 * any set of entries of the inverse) is the FP64 sum, over ascending k, of
 * products of the |I| solved vectors.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct oracle_factor {
    int64_t n;
    int64_t *Lp;    /* [n+1] column pointers of strictly-lower L */
    int32_t *Li;    /* row indices, ascending within a column */
    double *Lx;     /* values */
    double *D;      /* [n] */
    int32_t *parent;/* [n] elimination tree, -1 at a root */
    double flops;   /* multiply-adds * 2 spent in the column updates */
} oracle_factor;

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_NOT_SPD = 2, ORACLE_ERR_OOM = 3 };

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

void oracle_free(oracle_factor *f) {
    if (!f) return;
    free(f->Lp); free(f->Li); free(f->Lx); free(f->D); free(f->parent);
    free(f);
}

/* Left-looking LDL^T.  Returns ORACLE_OK or an error; *bad_col receives the
 * column of a non-positive pivot. */
int oracle_ldlt(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                oracle_factor **out, int64_t *bad_col) {
    *out = NULL;
    if (bad_col) *bad_col = -1;
    if (n < 0 || (n > 0 && (!colptr || !rowind || !val))) return ORACLE_ERR_ARG;
    oracle_factor *f = calloc(1, sizeof *f);
    if (!f) return ORACLE_ERR_OOM;
    f->n = n;
    int64_t cap = colptr[n] > 16 ? colptr[n] : 16;
    f->Lp = malloc((size_t)(n + 1) * sizeof(int64_t));
    f->Li = malloc((size_t)cap * sizeof(int32_t));
    f->Lx = malloc((size_t)cap * sizeof(double));
    f->D = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    f->parent = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    double *acc = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    char *mark = calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t *pat = malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t *head = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)); /* list head per row */
    int64_t *next = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t)); /* list link per column */
    int64_t *pos = malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));  /* next unread entry per column */
    if (!f->Lp || !f->Li || !f->Lx || !f->D || !f->parent || !acc || !mark || !pat || !head ||
        !next || !pos) {
        free(acc); free(mark); free(pat); free(head); free(next); free(pos); oracle_free(f);
        return ORACLE_ERR_OOM;
    }
    for (int64_t j = 0; j < n; ++j) head[j] = -1;
    f->Lp[0] = 0;
    int rc = ORACLE_OK;
    for (int64_t j = 0; j < n; ++j) {
        /* gather A(j:n, j); the first stored entry of a lower-CSC column is its diagonal */
        int64_t np = 0;
        double ajj = 0.0;
        for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
            int32_t i = rowind[p];
            if (i < j) continue;
            if (i == j) ajj += val[p];
            if (!mark[i]) { mark[i] = 1; pat[np++] = i; }
            acc[i] += val[p];
        }
        /* subtract the contributions of every column k < j with L(j,k) != 0 */
        int64_t k = head[j];
        head[j] = -1;
        while (k != -1) {
            int64_t knext = next[k];
            int64_t p = pos[k];               /* Li[p] == j */
            double ljk = f->Lx[p];
            double s = ljk * f->D[k];
            for (int64_t q = p; q < f->Lp[k + 1]; ++q) {
                int32_t i = f->Li[q];
                if (!mark[i]) { mark[i] = 1; pat[np++] = i; }
                acc[i] -= f->Lx[q] * s;
            }
            f->flops += 2.0 * (double)(f->Lp[k + 1] - p);
            /* move column k to the list of its next row */
            if (p + 1 < f->Lp[k + 1]) {
                pos[k] = p + 1;
                int64_t r = f->Li[p + 1];
                next[k] = head[r];
                head[r] = k;
            }
            k = knext;
        }
        double dj = acc[j];
        if (!mark[j] || !(dj > 0.0) || dj <= 1e-14 * fabs(ajj)) {
            if (bad_col) *bad_col = j;
            rc = ORACLE_ERR_NOT_SPD;
            break;
        }
        f->D[j] = dj;
        /* sort the pattern and write column j of L */
        qsort(pat, (size_t)np, sizeof(int32_t), cmp_i32);
        int64_t need = f->Lp[j] + np;
        if (need > cap) {
            while (cap < need) cap *= 2;
            int32_t *li = realloc(f->Li, (size_t)cap * sizeof(int32_t));
            double *lx = realloc(f->Lx, (size_t)cap * sizeof(double));
            if (li) f->Li = li;
            if (lx) f->Lx = lx;
            if (!li || !lx) { rc = ORACLE_ERR_OOM; break; }
        }
        int64_t w = f->Lp[j];
        for (int64_t t = 0; t < np; ++t) {
            int32_t i = pat[t];
            if (i > j) { f->Li[w] = i; f->Lx[w] = acc[i] / dj; ++w; }
            acc[i] = 0.0;
            mark[i] = 0;
        }
        f->Lp[j + 1] = w;
        f->parent[j] = (w > f->Lp[j]) ? f->Li[f->Lp[j]] : -1;
        if (w > f->Lp[j]) {
            pos[j] = f->Lp[j];
            int64_t r = f->Li[f->Lp[j]];
            next[j] = head[r];
            head[r] = j;
        }
    }
    free(acc); free(mark); free(pat); free(head); free(next); free(pos);
    if (rc != ORACLE_OK) { oracle_free(f); return rc; }
    *out = f;
    return ORACLE_OK;
}

int64_t oracle_n(const oracle_factor *f) { return f->n; }
int64_t oracle_nnz_l(const oracle_factor *f) { return f->Lp[f->n]; }
double oracle_flops(const oracle_factor *f) { return f->flops; }

/* Copy out L (strictly lower CSC), D and the elimination tree. */
void oracle_get(const oracle_factor *f, int64_t *Lp, int32_t *Li, double *Lx, double *D,
                int32_t *parent) {
    int64_t n = f->n, nz = f->Lp[n];
    if (Lp) memcpy(Lp, f->Lp, (size_t)(n + 1) * sizeof(int64_t));
    if (Li) memcpy(Li, f->Li, (size_t)nz * sizeof(int32_t));
    if (Lx) memcpy(Lx, f->Lx, (size_t)nz * sizeof(double));
    if (D) memcpy(D, f->D, (size_t)n * sizeof(double));
    if (parent) memcpy(parent, f->parent, (size_t)n * sizeof(int32_t));
}

/* x = A^{-1} b: forward z = L^{-1} b, w = D^{-1} z, backward x = L^{-T} w (Sec. 3.2.3). */
void oracle_solve(const oracle_factor *f, const double *b, double *x) {
    int64_t n = f->n;
    if (x != b) memcpy(x, b, (size_t)n * sizeof(double));
    for (int64_t j = 0; j < n; ++j)                       /* forward, bottom-up */
        for (int64_t p = f->Lp[j]; p < f->Lp[j + 1]; ++p) x[f->Li[p]] -= f->Lx[p] * x[j];
    for (int64_t j = 0; j < n; ++j) x[j] /= f->D[j];
    for (int64_t j = n - 1; j >= 0; --j) {                /* backward, top-down */
        double s = x[j];
        for (int64_t p = f->Lp[j]; p < f->Lp[j + 1]; ++p) s -= f->Lx[p] * x[f->Li[p]];
        x[j] = s;
    }
}

typedef struct {
    const oracle_factor *f;
    const int32_t *idx;
    double *out;
    int64_t lo, hi;
    int err;
} inv_job;

static void *inv_worker(void *arg) {
    inv_job *jb = arg;
    const oracle_factor *f = jb->f;
    int64_t n = f->n;
    double *z = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!z) { jb->err = 1; return NULL; }
    for (int64_t t = jb->lo; t < jb->hi; ++t) {
        int64_t i = jb->idx[t];
        /* L z = e_i: z is zero above i and off the path i -> root */
        z[i] = 1.0;
        double var = 0.0;
        for (int64_t k = i; k != -1; k = f->parent[k]) {
            double zk = z[k];
            for (int64_t p = f->Lp[k]; p < f->Lp[k + 1]; ++p) z[f->Li[p]] -= f->Lx[p] * zk;
            var += zk * zk / f->D[k];
            z[k] = 0.0;
        }
        jb->out[t] = var;
    }
    free(z);
    return NULL;
}

/* out[t] = (A^{-1})_{idx[t], idx[t]} for t < m, using up to nthreads threads. */
int oracle_inv_diag(const oracle_factor *f, const int32_t *idx, int64_t m, double *out,
                    int nthreads) {
    for (int64_t t = 0; t < m; ++t)
        if (idx[t] < 0 || idx[t] >= f->n) return ORACLE_ERR_ARG;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (m < nthreads) nthreads = m > 0 ? (int)m : 1;
    pthread_t th[256];
    inv_job jobs[256];
    for (int w = 0; w < nthreads; ++w) {
        jobs[w].f = f; jobs[w].idx = idx; jobs[w].out = out; jobs[w].err = 0;
        jobs[w].lo = m * w / nthreads; jobs[w].hi = m * (w + 1) / nthreads;
    }
    int started[256] = {0};
    for (int w = 1; w < nthreads; ++w)
        started[w] = pthread_create(&th[w], NULL, inv_worker, &jobs[w]) == 0;
    inv_worker(&jobs[0]);
    int err = jobs[0].err;
    for (int w = 1; w < nthreads; ++w) {
        if (started[w]) pthread_join(th[w], NULL);
        else inv_worker(&jobs[w]);
        err |= jobs[w].err;
    }
    return err ? ORACLE_ERR_OOM : ORACLE_OK;
}

/* Algorithmic flops of the pruned forward solves behind oracle_inv_diag:
 * sum over requested i of sum over k on path(i) of 2 * (|L(:,k)| + 1). */
double oracle_inv_diag_flops(const oracle_factor *f, const int32_t *idx, int64_t m) {
    double s = 0.0;
    for (int64_t t = 0; t < m; ++t)
        for (int64_t k = idx[t]; k != -1; k = f->parent[k])
            s += 2.0 * (double)(f->Lp[k + 1] - f->Lp[k] + 1);
    return s;
}

/* out[s * m + t] = (A^{-1})_{idx[s], idx[t]} for s, t < m (row-major, both
 * triangles).  Every z = L^{-1} e_i is kept as a dense length-n vector. */
int oracle_inv_block(const oracle_factor *f, const int32_t *idx, int64_t m, double *out) {
    const int64_t n = f->n;
    for (int64_t t = 0; t < m; ++t)
        if (idx[t] < 0 || idx[t] >= n) return ORACLE_ERR_ARG;
    if (m == 0) return ORACLE_OK;
    double *Zm = calloc((size_t)m * (size_t)n, sizeof(double));
    if (!Zm) return ORACLE_ERR_OOM;
    for (int64_t t = 0; t < m; ++t) {
        double *z = Zm + t * n;
        z[idx[t]] = 1.0;
        for (int64_t k = idx[t]; k != -1; k = f->parent[k])
            for (int64_t p = f->Lp[k]; p < f->Lp[k + 1]; ++p) z[f->Li[p]] -= f->Lx[p] * z[k];
    }
    for (int64_t s = 0; s < m; ++s)
        for (int64_t t = 0; t <= s; ++t) {
            const double *zs = Zm + s * n, *zt = Zm + t * n;
            double acc = 0.0;
            for (int64_t k = 0; k < n; ++k) acc += zs[k] * zt[k] / f->D[k];
            out[s * m + t] = acc;
            out[t * m + s] = acc;
        }
    free(Zm);
    return ORACLE_OK;
}
