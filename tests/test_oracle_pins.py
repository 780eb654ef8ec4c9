"""Pins for the FP64 CPU oracle: each check ties the oracle to something other
than itself (a dense Gauss-Jordan inverse written here, a library routine,
a closed form, an identity, or the worked elimination-tree example of
Sec. 3.2.1 / Fig. 3-4).  A final test plants mistakes in copies of the
oracle's C source and checks that the pins catch every one."""
import json
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from spigen import TINY, generate, random_spd, scaled

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lower_csc(A):
    low = sp.tril(sp.csc_matrix(A)).tocsc()
    low.sum_duplicates(); low.sort_indices()
    return low.shape[0], low.indptr.astype(np.int64), low.indices.astype(np.int32), low.data


def gauss_jordan_inverse(A):
    """Dense Gauss-Jordan elimination with partial pivoting on [A | I]."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    M = np.hstack([A, np.eye(n)])
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] /= M[c, c]
        f = M[:, c].copy(); f[c] = 0.0
        M -= np.outer(f, M[c])
    return M[:, n:]


def takahashi_diag(Lp, Li, Lx, D):
    """Selected inverse on the pattern of L (Takahashi 1973 / Campbell 1995,
    cited in Sec. 3.3): Z = D^-1 L^-1 + (I - L^T) Z, swept from the last
    column; returns diag(Z)."""
    n = len(D)
    Z = np.zeros((n, n))
    for j in range(n - 1, -1, -1):
        S = Li[Lp[j]:Lp[j + 1]]
        l = Lx[Lp[j]:Lp[j + 1]]
        if len(S):
            zs = -(Z[np.ix_(S, S)] @ l)
            Z[S, j] = zs
            Z[j, S] = zs
            Z[j, j] = 1.0 / D[j] - l @ zs
        else:
            Z[j, j] = 1.0 / D[j]
    return np.diag(Z).copy()


def scaled_condition(A):
    d = np.sqrt(np.diag(A))
    ev = np.linalg.eigvalsh(A / d[:, None] / d[None, :])
    return ev[-1] / ev[0]


def small_cases():
    pbs = [generate(TINY), random_spd(40, 0.15, 1), random_spd(120, 0.05, 2, dominance=0.3)]
    return [(pb.full_matrix().toarray(), pb.b) for pb in pbs]


def run_pins(lib=None):
    """Run the numeric pins against an oracle library; return failures."""
    fails = []
    for A, b in small_cases():
        n, cp, ri, va = lower_csc(A)
        try:
            f = oracle.OracleFactor(n, cp, ri, va, lib=lib)
        except Exception as e:  # a planted mistake may stop the factorization
            fails.append(f"factor: {e}")
            continue
        kappa = scaled_condition(A)
        Ainv = gauss_jordan_inverse(A)
        tol = 64 * np.finfo(float).eps * max(kappa, 10.0)
        x = f.solve(b)
        if np.abs(x - Ainv @ b).max() > tol * np.abs(Ainv @ b).max():
            fails.append("x vs Gauss-Jordan")
        if np.linalg.norm(A @ x - b) > 1e-12 * np.linalg.norm(b):
            fails.append("residual")
        v = f.inv_diag()
        # per entry: the variances of one problem span decades (pointing columns against
        # source bins), so an error confined to the small ones must not hide under the
        # largest one's scale
        vg = np.diag(Ainv)
        if not np.all(np.abs(v - vg) <= tol * vg):
            fails.append("diag vs Gauss-Jordan")
        # a block of the inverse (covariances of selected unknowns) against Gauss-Jordan,
        # on the scale sqrt(v_s v_t) of each entry
        sel = np.unique(np.linspace(0, n - 1, min(n, 12)).astype(np.int32))
        G = f.inv_block(sel)
        Gref = Ainv[np.ix_(sel, sel)]
        sc = np.sqrt(np.outer(np.diag(Gref), np.diag(Gref)))
        if np.abs(G - Gref).max() > tol * sc.max() or not np.all(np.abs(G - Gref) <= tol * sc + 1e-300):
            fails.append("inverse block vs Gauss-Jordan")
        Lp, Li, Lx, D, par = f.factors()
        tk = takahashi_diag(Lp, Li, Lx, D)
        if not np.all(np.abs(v - tk) <= 1e-12 * np.abs(tk)):
            fails.append("diag vs Takahashi")
        # elimination tree: parent = smallest row > j of L(:, j)
        Ldense = np.zeros((n, n))
        for j in range(n):
            Ldense[Li[Lp[j]:Lp[j + 1]], j] = 1
        for j in range(n):
            rows = np.nonzero(Ldense[:, j])[0]
            if (par[j] if len(rows) else -1) != (rows[0] if len(rows) else -1):
                fails.append("etree"); break
    return fails


# ---------------------------------------------------------------- the pins
def test_pins_hold_for_the_oracle():
    assert run_pins() == []


def test_inverse_block_properties():
    """The block of the inverse is symmetric positive definite, its diagonal
    is the inverse diagonal, and |cov| <= sqrt(v_s v_t) (a principal block of
    an SPD inverse)."""
    pb = generate(scaled(TINY, 200, seed=4))
    f = oracle.OracleFactor.from_problem(pb)
    sel = np.random.default_rng(3).choice(pb.n, 40, replace=False).astype(np.int32)
    G = f.inv_block(sel)
    assert np.array_equal(G, G.T)
    assert np.allclose(np.diag(G), f.inv_diag(sel), rtol=1e-14, atol=0)
    np.linalg.cholesky(G)
    v = np.diag(G)
    assert np.all(np.abs(G) <= np.sqrt(np.outer(v, v)) * (1 + 1e-12))


def test_paper_etree_example():
    g = json.load(open(os.path.join(GOLDEN, "etree_fig3.json")))
    n = g["n"]
    A = np.eye(n) * 4.0
    for i, j in g["offdiagonal_pattern_lower"]:
        A[i - 1, j - 1] = A[j - 1, i - 1] = -1.0
    f = oracle.OracleFactor(*lower_csc(A))
    _, _, _, _, par = f.factors()
    par1 = {j + 1: (int(p) + 1 if p >= 0 else None) for j, p in enumerate(par)}
    roots = [k for k, v in par1.items() if v is None]
    assert roots == [g["root"]]
    assert {k: v for k, v in par1.items() if v is not None} == {int(k): v for k, v in g["parent"].items()}
    assert sorted(k for k, v in par1.items() if v == 5) == g["children_of_5"]
    internal = set(v for v in par1.values() if v is not None)
    assert sorted(set(range(1, n + 1)) - internal) == g["leaves"]
    desc5 = sorted(k for k in range(1, n + 1) if k != 5 and _is_ancestor(par1, 5, k))
    assert desc5 == g["descendants_of_5"]
    # the printed order is a postorder: parents after children, subtrees contiguous
    po = g["postorder"]
    pos = {v: i for i, v in enumerate(po)}
    assert all(pos[k] < pos[v] for k, v in par1.items() if v is not None)
    for v in range(1, n + 1):
        sub = sorted(pos[k] for k in range(1, n + 1) if k == v or _is_ancestor(par1, v, k))
        assert sub == list(range(sub[0], sub[0] + len(sub)))
    # a^-1_23: L z = e_3 is nonzero only on the path 3 -> 6; nodes 1 and 4 are never touched
    Lp, Li, Lx, D, _ = f.factors()
    L = np.eye(n)
    for j in range(n):
        L[Li[Lp[j]:Lp[j + 1]], j] = Lx[Lp[j]:Lp[j + 1]]
    z = np.linalg.solve(L, np.eye(n)[:, 2])
    assert [k + 1 for k in np.nonzero(z)[0]] == g["entry_a23"]["forward_path"]
    path = []
    k = 2
    while k != -1:
        path.append(k + 1); k = par[k]
    assert path == g["entry_a23"]["forward_path"]
    assert list(reversed(path)) + [2] == g["entry_a23"]["backward_path"]
    assert not set(g["entry_a23"]["not_visited"]) & set(g["entry_a23"]["backward_path"])
    # and the entry itself: (L^-T D^-1 z)_2 against the dense inverse
    a23 = np.linalg.solve(L.T, z / D)[1]
    assert abs(a23 - np.linalg.inv(A)[1, 2]) < 1e-14


def _is_ancestor(par1, a, k):
    while par1.get(k) is not None:
        k = par1[k]
        if k == a:
            return True
    return False


def test_residual_and_positivity_on_a_larger_spi_problem():
    pb = generate(scaled(TINY, 1200, seed=3))
    A = pb.full_matrix()
    f = oracle.OracleFactor.from_problem(pb)
    x = f.solve(pb.b)
    assert np.linalg.norm(A @ x - pb.b) <= 1e-12 * np.linalg.norm(pb.b)
    v = f.inv_diag()
    assert np.all(v > 0)
    # Cauchy-Schwarz for SPD: (A^-1)_ii >= 1 / A_ii
    assert np.all(v * A.diagonal() >= 1.0 - 1e-12)
    # last eliminated column: L^-1 e_{n-1} = e_{n-1}, so the variance is 1/d_{n-1}
    _, _, _, D, _ = f.factors()
    assert v[-1] == 1.0 / D[-1]


def test_noise_free_closed_form():
    """With y = H x_true exactly the least-squares solution is x_true (Eq. 6-7)."""
    pb = generate(TINY, noise=False)
    f = oracle.OracleFactor.from_problem(pb)
    x = f.solve(pb.b)
    kappa = scaled_condition(pb.full_matrix().toarray())
    assert np.abs(x - pb.x_true).max() <= 1e-13 * kappa * np.abs(pb.x_true).max() * 100


def test_trace_identity():
    """sum_i (A^-1)_ii = ||D^-1/2 L^-1||_F^2 with L^-1 from a library triangular solve."""
    pb = generate(TINY)
    f = oracle.OracleFactor.from_problem(pb)
    Lp, Li, Lx, D, _ = f.factors()
    n = pb.n
    L = np.eye(n)
    for j in range(n):
        L[Li[Lp[j]:Lp[j + 1]], j] = Lx[Lp[j]:Lp[j + 1]]
    Linv = sla.solve_triangular(L, np.eye(n), lower=True, unit_diagonal=True)
    tr = np.sum(Linv ** 2 / D[:, None])
    assert abs(f.inv_diag().sum() - tr) <= 1e-12 * tr


def test_ordering_invariance():
    pb = generate(TINY)
    A = pb.full_matrix().toarray()
    v = oracle.OracleFactor.from_problem(pb).inv_diag()
    x = oracle.OracleFactor.from_problem(pb).solve(pb.b)
    rng = np.random.default_rng(7)
    for perm in (rng.permutation(pb.n), np.arange(pb.n)[::-1].copy()):
        Ap = A[np.ix_(perm, perm)]
        f = oracle.OracleFactor(*lower_csc(Ap))
        vp = f.inv_diag()
        assert np.abs(vp - v[perm]).max() <= 1e-10 * np.abs(v).max()
        xp = f.solve(pb.b[perm])
        assert np.abs(xp - x[perm]).max() <= 1e-10 * np.abs(x).max()


def test_block_diagonal_special_cases():
    """Diagonal N (pointing columns alone): var = 1/N_ii exactly.
    2x2 blocks: (A^-1)_11 = a22 / (a11 a22 - a12^2)."""
    rng = np.random.default_rng(5)
    d = rng.uniform(0.5, 3.0, 50)
    f = oracle.OracleFactor(*lower_csc(np.diag(d)))
    assert np.array_equal(f.inv_diag(), 1.0 / d)
    B = np.zeros((40, 40))
    for k in range(0, 40, 2):
        a, c = rng.uniform(2, 3, 2)
        bb = rng.uniform(-1, 1)
        B[k:k + 2, k:k + 2] = [[a, bb], [bb, c]]
    v = oracle.OracleFactor(*lower_csc(B)).inv_diag()
    ref = np.empty(40)
    for k in range(0, 40, 2):
        a, bb, c = B[k, k], B[k + 1, k], B[k + 1, k + 1]
        ref[k], ref[k + 1] = c / (a * c - bb * bb), a / (a * c - bb * bb)
    assert np.abs(v - ref).max() <= 4 * np.finfo(float).eps * np.abs(ref).max()


def test_not_spd_reports_column():
    A = np.diag([2.0, 3.0, -1.0, 4.0])
    A[1, 0] = A[0, 1] = 0.5
    with pytest.raises(oracle.NotSPD) as e:
        oracle.OracleFactor(*lower_csc(A))
    assert e.value.col == 2


# ------------------------------------------------- planted mistakes (CPU only)
MUTATIONS = {
    "variance without 1/d": ("var += zk * zk / f->D[k];", "var += zk * zk;"),
    "update sign flipped": ("acc[i] -= f->Lx[q] * s;", "acc[i] += f->Lx[q] * s;"),
    "update misses d_k": ("double s = ljk * f->D[k];", "double s = ljk;"),
    "forward solve sign": ("x[f->Li[p]] -= f->Lx[p] * x[j];", "x[f->Li[p]] += f->Lx[p] * x[j];"),
    "diagonal solve multiplies": ("x[j] /= f->D[j];", "x[j] *= f->D[j];"),
    "backward solve transposed": ("s -= f->Lx[p] * x[f->Li[p]];", "s -= f->Lx[p] * x[j];"),
    "pruned solve drops z_k": ("z[f->Li[p]] -= f->Lx[p] * zk;", "z[f->Li[p]] -= f->Lx[p];"),
    "etree parent = last row": ("f->parent[j] = (w > f->Lp[j]) ? f->Li[f->Lp[j]] : -1;",
                                "f->parent[j] = (w > f->Lp[j]) ? f->Li[w - 1] : -1;"),
    "L scaled by wrong pivot": ("f->Lx[w] = acc[i] / dj;", "f->Lx[w] = acc[i] / ajj;"),
    "inverse block without 1/d": ("acc += zs[k] * zt[k] / f->D[k];", "acc += zs[k] * zt[k];"),
    "inverse block from one vector": ("acc += zs[k] * zt[k] / f->D[k];", "acc += zs[k] * zs[k] / f->D[k];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    src = open(oracle._SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o",
                           str(so), str(mutated), "-lm"])
    lib = oracle.load_library(str(so))
    assert run_pins(lib) != [], f"planted mistake '{name}' was not caught"


def test_mle_oracle_pins():
    """The Poisson maximum-likelihood oracle: noise-free counts give x_true
    back; at its fit the gradient H^T (1 - y/e) vanishes and C did not grow
    from the start; its gradient and Hessian formulas agree with finite
    differences of C itself."""
    import scipy.sparse as sp
    pb = generate(TINY, sparse_design=True, noise=False)
    x0 = np.linalg.solve(pb.full_matrix().toarray(), pb.b)
    x, v, _ = oracle.mle_newton(pb.H, pb.y, x0)
    assert np.abs(x - pb.x_true).max() <= 1e-10 * np.abs(pb.x_true).max()
    pb = generate(TINY, sparse_design=True)
    x0 = np.linalg.solve(pb.full_matrix().toarray(), pb.b)
    x, v, _ = oracle.mle_newton(pb.H, pb.y, x0)
    e = pb.H @ x
    g = pb.H.T @ (1.0 - pb.y / e)
    assert np.abs(g).max() <= 1e-9 * np.abs(pb.H.T @ np.ones_like(e)).max()
    assert oracle.cash(pb.H, pb.y, x) <= oracle.cash(pb.H, pb.y, x0)
    assert np.all(v > 0)
    # finite differences of C along two coordinates, at a point off the optimum
    H = sp.csr_matrix(pb.H)
    xp = x * 1.01
    ep = H @ xp
    grad = H.T @ (1.0 - pb.y / ep)
    hess = (H.T @ sp.diags(pb.y / ep ** 2) @ H).tocsc()
    for j in (3, pb.n - 2):
        h = 1e-6 * max(1.0, abs(xp[j]))
        d = np.zeros(pb.n); d[j] = h
        fd = (oracle.cash(H, pb.y, xp + d) - oracle.cash(H, pb.y, xp - d)) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-5 * max(1.0, abs(grad[j]))
        h2 = 1e-3 * max(1.0, abs(xp[j]))  # wider step: the second difference cancels more
        d2 = np.zeros(pb.n); d2[j] = h2
        fd2 = (oracle.cash(H, pb.y, xp + d2) - 2 * oracle.cash(H, pb.y, xp) + oracle.cash(H, pb.y, xp - d2)) / h2 ** 2
        assert abs(fd2 - hess[j, j]) <= 1e-3 * hess[j, j]
