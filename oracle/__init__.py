"""FP64 CPU oracle for the sparse LDL^T / solve / diag(N^-1) path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package.  The path's arithmetic lives in spi_oracle.c (plain C, natural
ordering, left-looking LDL^T, column-by-column inverse diagonal and inverse
blocks; paper Sec. 3.2, Sec. 3.3.1 and Sec. 4.3), which this module compiles
and calls.  The steps around the path are written here in plain NumPy/SciPy:
the normal equations (Sec. 4.1, Eq. 7), the Poisson fit of the appendix on
low counts, Algorithm 1 of the appendix on the "empty-field" pattern, and a
dense LDL^T with two-by-two pivots for indefinite matrices (Sec. 5).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ORACLE_OK, ORACLE_ERR_ARG, ORACLE_ERR_NOT_SPD, ORACLE_ERR_OOM = 0, 1, 2, 3


class NotSPD(RuntimeError):
    def __init__(self, col: int):
        super().__init__(f"non-positive pivot at column {col}")
        self.col = col


def build(force: bool = False) -> str:
    """Compile spi_oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.oracle_ldlt.argtypes = [I64, P, P, P, ctypes.POINTER(P), ctypes.POINTER(I64)]
    lib.oracle_ldlt.restype = ctypes.c_int
    lib.oracle_n.argtypes = [P]; lib.oracle_n.restype = I64
    lib.oracle_nnz_l.argtypes = [P]; lib.oracle_nnz_l.restype = I64
    lib.oracle_flops.argtypes = [P]; lib.oracle_flops.restype = D
    lib.oracle_get.argtypes = [P, P, P, P, P, P]; lib.oracle_get.restype = None
    lib.oracle_solve.argtypes = [P, P, P]; lib.oracle_solve.restype = None
    lib.oracle_inv_diag.argtypes = [P, P, I64, P, ctypes.c_int]
    lib.oracle_inv_diag.restype = ctypes.c_int
    lib.oracle_inv_diag_flops.argtypes = [P, P, I64]
    lib.oracle_inv_diag_flops.restype = D
    lib.oracle_inv_block.argtypes = [P, P, I64, P]
    lib.oracle_inv_block.restype = ctypes.c_int
    lib.oracle_free.argtypes = [P]; lib.oracle_free.restype = None
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleFactor:
    """A = L D L^T of a symmetric matrix given by its lower CSC (natural order)."""

    def __init__(self, n, colptr, rowind, values, lib=None):
        lib = _load() if lib is None else lib
        self._lib = lib
        self._cp = np.ascontiguousarray(colptr, dtype=np.int64)
        self._ri = np.ascontiguousarray(rowind, dtype=np.int32)
        self._va = np.ascontiguousarray(values, dtype=np.float64)
        h = ctypes.c_void_p()
        bad = ctypes.c_int64(-1)
        rc = lib.oracle_ldlt(int(n), _ptr(self._cp), _ptr(self._ri), _ptr(self._va),
                             ctypes.byref(h), ctypes.byref(bad))
        if rc == ORACLE_ERR_NOT_SPD:
            raise NotSPD(bad.value)
        if rc != ORACLE_OK:
            raise RuntimeError(f"oracle_ldlt failed with code {rc}")
        self._h = h
        self.n = int(n)

    @classmethod
    def from_problem(cls, pb, lib=None):
        return cls(pb.n, pb.colptr, pb.rowind, pb.values, lib=lib)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None:
            self._lib.oracle_free(h)
            self._h = None

    @property
    def nnz_l(self) -> int:
        return int(self._lib.oracle_nnz_l(self._h))

    @property
    def flops(self) -> float:
        return float(self._lib.oracle_flops(self._h))

    def factors(self):
        """(Lp, Li, Lx, D, parent): strictly-lower L in CSC, D, elimination tree."""
        nz = self.nnz_l
        Lp = np.empty(self.n + 1, np.int64); Li = np.empty(nz, np.int32)
        Lx = np.empty(nz, np.float64); D = np.empty(self.n, np.float64)
        par = np.empty(self.n, np.int32)
        self._lib.oracle_get(self._h, _ptr(Lp), _ptr(Li), _ptr(Lx), _ptr(D), _ptr(par))
        return Lp, Li, Lx, D, par

    def solve(self, b) -> np.ndarray:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        self._lib.oracle_solve(self._h, _ptr(b), _ptr(x))
        return x

    def inv_diag(self, idx=None, nthreads: int | None = None) -> np.ndarray:
        """(A^-1)_ii for i in idx (all i if None)."""
        idx = np.arange(self.n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, np.int32)
        out = np.empty(len(idx), np.float64)
        nt = nthreads if nthreads is not None else (os.cpu_count() or 1)
        rc = self._lib.oracle_inv_diag(self._h, _ptr(idx), len(idx), _ptr(out), int(nt))
        if rc != ORACLE_OK:
            raise RuntimeError(f"oracle_inv_diag failed with code {rc}")
        return out

    def inv_block(self, idx) -> np.ndarray:
        """The dense block (A^-1)[idx, idx] (m x m)."""
        idx = np.ascontiguousarray(idx, np.int32)
        out = np.empty((len(idx), len(idx)), np.float64)
        rc = self._lib.oracle_inv_block(self._h, _ptr(idx), len(idx), _ptr(out))
        if rc:
            raise RuntimeError(f"oracle_inv_block failed with code {rc}")
        return out

    def inv_diag_flops(self, idx=None) -> float:
        idx = np.arange(self.n, dtype=np.int32) if idx is None else np.ascontiguousarray(idx, np.int32)
        return float(self._lib.oracle_inv_diag_flops(self._h, _ptr(idx), len(idx)))


def normal_equations(H, w, y, colptr, rowind):
    """The normal equations of the weighted least-squares problem (Eq. 7):
    N = H^T W H and b = H^T W y with W = diag(w), H any scipy sparse matrix
    (rows = observations).  N is returned as values on the given lower CSC
    pattern (0 where the pattern holds a structural zero of N), b densely.
    The product is a plain sparse matrix product (the paper's Sec. 4.1 is
    about computing it efficiently; this is the definition)."""
    import scipy.sparse as sp
    Hc = sp.csc_matrix(H)
    N = (Hc.T @ sp.diags(np.asarray(w, dtype=np.float64)) @ Hc).tocsc()
    N.sort_indices()
    colptr = np.asarray(colptr, dtype=np.int64)
    rowind = np.asarray(rowind, dtype=np.int32)
    vals = np.zeros(len(rowind), dtype=np.float64)
    for j in range(len(colptr) - 1):
        rows = N.indices[N.indptr[j]:N.indptr[j + 1]]
        data = N.data[N.indptr[j]:N.indptr[j + 1]]
        want = rowind[colptr[j]:colptr[j + 1]]
        pos = np.searchsorted(rows, want)
        ok = (pos < len(rows)) & (rows[np.minimum(pos, max(len(rows) - 1, 0))] == want) if len(rows) else np.zeros(len(want), bool)
        vals[colptr[j]:colptr[j + 1]][ok] = data[pos[ok]]
    b = Hc.T @ (np.asarray(w, dtype=np.float64) * np.asarray(y, dtype=np.float64))
    return vals, np.asarray(b).ravel()


def cash(H, y, x):
    """The Cash statistic C(x) = sum_i (e_i - y_i ln e_i), e = H x (the
    likelihood of the appendix on Poisson fitting, up to the factor -2 and a
    constant); terms with y_i = 0 are e_i."""
    e = np.asarray(H @ x).ravel()
    yy = np.asarray(y, dtype=np.float64)
    t = e.copy()
    pos = yy > 0
    t[pos] -= yy[pos] * np.log(e[pos])
    return float(t.sum())


def mle_newton(H, y, x0, max_iter=30, tol=1e-12):
    """Poisson maximum-likelihood fit by Newton's method, as the paper's
    appendix states it: minimise C(x) = sum (e - y ln e), e = H x, with
    gradient H^T (1 - y/e) and Hessian H^T diag(y/e^2) H; each step solves
    Hess dx = H^T (y/e - 1) (a dense solve here), halving the step until
    every e stays positive and C does not increase beyond 1e-12 |C| (the
    rounding level of the sum: near the fit the decrease is below it);
    stops when
    ||dx|| <= tol ||x|| (2-norms) or after max_iter steps.  Returns
    (x, diag(Hess^-1) at x, steps taken)."""
    import scipy.sparse as sp
    Hs = sp.csr_matrix(H)
    yy = np.asarray(y, dtype=np.float64)
    x = np.array(x0, dtype=np.float64)
    steps = 0
    for it in range(max_iter):
        e = np.asarray(Hs @ x).ravel()
        if np.any(e <= 0):
            raise ValueError("the model must be positive at the starting point")
        Hess = (Hs.T @ sp.diags(yy / e ** 2) @ Hs).toarray()
        g = np.asarray(Hs.T @ (yy / e - 1.0)).ravel()
        dx = np.linalg.solve(Hess, g)
        c0, t = cash(Hs, yy, x), 1.0
        for _ in range(60):
            xt = x + t * dx
            et = np.asarray(Hs @ xt).ravel()
            if np.all(et > 0) and cash(Hs, yy, xt) <= c0 + 1e-12 * abs(c0):
                break
            t *= 0.5
        x = x + t * dx
        steps += 1
        if np.linalg.norm(t * dx) <= tol * np.linalg.norm(x):
            break
    e = np.asarray(Hs @ x).ravel()
    Hess = (Hs.T @ sp.diags(yy / e ** 2) @ Hs).toarray()
    return x, np.diag(np.linalg.inv(Hess)).copy(), steps


def set_background(H, k0, upat, t, U):
    """H with the entry of each row i in the first k0 columns (its background
    column: the pointing's normalisation I_p^bg) set to U[upat_i] t_i, the
    background model B_dp = U^d I_p^bg t_dp of Eq. A4 with upat_i the pattern
    index of the row (its detector, or its detector and time interval) and
    t_i its t_dp.  Rows with upat_i < 0 have no background entry."""
    import scipy.sparse as sp
    Hs = sp.csr_matrix(H, copy=True)
    Hs.sort_indices()
    upat = np.asarray(upat)
    for i in range(Hs.shape[0]):
        lo, hi = Hs.indptr[i], Hs.indptr[i + 1]
        bg = [p for p in range(lo, hi) if Hs.indices[p] < k0]
        if len(bg) > 1 or (len(bg) == 1) != (upat[i] >= 0):
            raise ValueError(f"row {i}: background entries {len(bg)}, pattern index {upat[i]}")
        if bg:
            Hs.data[bg[0]] = U[upat[i]] * t[i]
    return Hs


def _background_terms(Hs, x, k0, upat, t):
    """Per row: y^S_i (the counts of the columns after the first k0), the
    background column c(i) and a_i = t_i x_c(i) (= I_p^bg t_dp); rows
    without a background entry get a_i = 0."""
    nrow = Hs.shape[0]
    ys = np.zeros(nrow)
    a = np.zeros(nrow)
    for i in range(nrow):
        for p in range(Hs.indptr[i], Hs.indptr[i + 1]):
            j = Hs.indices[p]
            if j < k0:
                a[i] = t[i] * x[j]
            else:
                ys[i] += Hs.data[p] * x[j]
    return ys, a


def background_pattern(H, x, y, w, k0, upat, t, U, mode="lsq"):
    """One re-estimation of the "empty-field" pattern (the appendix on its
    auto-computation): with the solution x known, the counts split into the
    sources' y^S and the background U^d a_i, a_i = I_p^bg t_dp, and each
    pattern value minimises its own statistic:
      least squares:  U_k = sum (y_i - y^S_i) a_i w_i / sum a_i^2 w_i,
      likelihood:     U_k = sum (y_i - y^S_i) / sum a_i  (the paper's
                      simplified form; the exact maximiser when y^S = 0),
    sums over the rows of pattern index k (a detector over all pointings, or
    over one interval of pointings).  A pattern index whose denominator is
    not positive keeps its value."""
    import scipy.sparse as sp
    Hs = sp.csr_matrix(H)
    upat = np.asarray(upat)
    ys, a = _background_terms(Hs, np.asarray(x, float), k0, upat, t)
    r = np.asarray(y, float) - ys
    U = np.array(U, dtype=np.float64)
    num = np.zeros(len(U))
    den = np.zeros(len(U))
    for i in range(Hs.shape[0]):
        k = upat[i]
        if k < 0:
            continue
        if mode == "lsq":
            num[k] += r[i] * a[i] * w[i]
            den[k] += a[i] * a[i] * w[i]
        else:
            num[k] += r[i]
            den[k] += a[i]
    ok = den > 0
    U[ok] = num[ok] / den[ok]
    return U


def chi2(H, y, w, x):
    """sum_i w_i (y_i - (H x)_i)^2, the weighted least-squares statistic."""
    r = np.asarray(y, float) - np.asarray(H @ x).ravel()
    return float(np.sum(np.asarray(w, float) * r * r))


def background_fit(H, y, w, k0, upat, t, U0, mode="lsq", max_iter=20, tol=1e-9,
                   variances=True, mle_iter=30, mle_tol=1e-12):
    """Algorithm 1 of the appendix on the "empty-field" pattern: starting
    from the pattern U0, repeat {solve for x with the current H (weighted
    least squares, or the Poisson likelihood fit by Newton's method started
    from the previous x when the model is positive there, else from the
    least-squares solution); re-estimate U from x (background_pattern); set
    the background entries of H} and stop when the statistic (chi^2, or the
    Cash statistic C = -L/2 + const) of a solve is not below the previous
    solve's by more than tol times its size, or after max_iter solves.
    The statistic is tested right after each solve, before U changes, so
    that the returned (U, x) are the pair that solve used; when the last
    solve's statistic is above the previous one, the previous pair is
    returned.  Then the variances diag(Hess^-1) at the returned pair (N for
    least squares, H^T diag(y/e^2) H for the likelihood).
    Returns (x, U, [statistic per solve], var or None)."""
    import scipy.sparse as sp
    yy = np.asarray(y, dtype=np.float64)
    ww = np.asarray(w, dtype=np.float64)
    U = np.array(U0, dtype=np.float64)
    x = None
    stats = []
    prev = None
    for it in range(max_iter):
        Hc = set_background(H, k0, upat, t, U)
        Nd = (Hc.T @ sp.diags(ww) @ Hc).toarray()
        if mode == "lsq":
            x = np.linalg.solve(Nd, Hc.T @ (ww * yy))
            stat = chi2(Hc, yy, ww, x)
        else:
            if x is None or np.any(np.asarray(Hc @ x).ravel() <= 0):
                x = np.linalg.solve(Nd, Hc.T @ (ww * yy))
            x, _, _ = mle_newton(Hc, yy, x, max_iter=mle_iter, tol=mle_tol)
            stat = cash(Hc, yy, x)
        stats.append(stat)
        if it > 0 and stat >= stats[-2] - tol * abs(stats[-2]):
            if stat > stats[-2]:
                U, x = prev
            break
        if it == max_iter - 1:
            break
        prev = (U.copy(), x.copy())
        U = background_pattern(Hc, x, yy, ww, k0, upat, t, U, mode)
    var = None
    if variances:
        Hc = set_background(H, k0, upat, t, U)
        if mode == "lsq":
            Hess = (Hc.T @ sp.diags(ww) @ Hc).toarray()
        else:
            e = np.asarray(Hc @ x).ravel()
            Hess = (Hc.T @ sp.diags(yy / e ** 2) @ Hc).toarray()
        var = np.diag(np.linalg.inv(Hess)).copy()
    return x, U, stats, var


BK_ALPHA = (1.0 + 17.0 ** 0.5) / 8.0  # Bunch-Kaufman growth-balancing constant


def ldlt_pivoted(A):
    """Symmetric indefinite LDL^T with 1x1 and 2x2 pivots (Sec. 5 of the
    paper notes that its matrices need 2x2 pivots for stability), in the
    Bunch-Kaufman partial-pivoting form: for the active column k with
    largest off-diagonal |a_rk| = lam,
      |a_kk| >= alpha lam            -> 1x1 pivot a_kk;
      else with sig = max_{i != r} |a_ir|:
      |a_kk| sig >= alpha lam^2      -> 1x1 pivot a_kk;
      |a_rr| >= alpha sig            -> swap k, r; 1x1 pivot;
      otherwise                      -> swap k+1, r; 2x2 pivot on (k, k+1);
    alpha = (1 + sqrt 17) / 8.  Dense FP64 on a copy of A (small problems).
    Returns (p, L, D, blocks): A[p][:, p] = L D L^T, L unit lower triangular,
    D block diagonal, blocks = list of (start, size) of D's pivots."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    p = np.arange(n)
    L = np.eye(n)
    D = np.zeros((n, n))
    blocks = []

    def swap(i, j):
        if i == j:
            return
        A[[i, j], :] = A[[j, i], :]
        A[:, [i, j]] = A[:, [j, i]]
        L[[i, j], :] = L[[j, i], :]  # rows of the finished columns follow their unknowns
        L[:, [i, j]] = L[:, [j, i]]
        p[[i, j]] = p[[j, i]]

    k = 0
    while k < n:
        col = np.abs(A[k + 1:, k])
        lam = col.max() if col.size else 0.0
        size = 1
        if lam == 0.0:
            if A[k, k] == 0.0:
                raise NotSPD(k)  # a zero column: singular
        elif abs(A[k, k]) >= BK_ALPHA * lam:
            pass
        else:
            r = k + 1 + int(np.argmax(col))
            row_r = np.abs(np.concatenate([A[r, k:r], A[r + 1:, r]]))
            sig = row_r.max()
            if abs(A[k, k]) * sig >= BK_ALPHA * lam * lam:
                pass
            elif abs(A[r, r]) >= BK_ALPHA * sig:
                swap(k, r)
            else:
                swap(k + 1, r)
                size = 2
        E = A[k:k + size, k:k + size].copy()
        C = A[k + size:, k:k + size].copy()
        if size == 1 and E[0, 0] == 0.0:
            raise NotSPD(k)
        Einv = np.linalg.inv(E)
        D[k:k + size, k:k + size] = E
        L[k + size:, k:k + size] = C @ Einv
        A[k + size:, k + size:] -= C @ Einv @ C.T
        blocks.append((k, size))
        k += size
    # the swaps above also permuted the unit diagonal of columns not yet reached; restore it
    L[np.diag_indices(n)] = 1.0
    return p, np.tril(L), D, blocks


def inv_diag_pivoted(A):
    """diag(A^-1) from the pivoted factorization: with A[p][:, p] = L D L^T,
    (A^-1)_{p_i p_i} = z^T D^-1 z, z = L^-1 e_i, D^-1 taken block by block
    (1x1 and 2x2) -- the diagonal of the inverse of an indefinite matrix by
    forward solves, as in the SPD case."""
    p, L, D, blocks = ldlt_pivoted(A)
    n = len(p)
    out = np.empty(n)
    Linv = np.linalg.inv(L)  # columns z_i = L^-1 e_i (dense: small problems)
    for i in range(n):
        z = Linv[:, i]
        s = 0.0
        for (k, size) in blocks:
            zb = z[k:k + size]
            s += float(zb @ np.linalg.solve(D[k:k + size, k:k + size], zb))
        out[p[i]] = s
    return out
