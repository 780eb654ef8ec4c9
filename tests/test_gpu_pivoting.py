"""Symmetric indefinite matrices on the GPU (spi_options.pivoting; paper Sec. 5:
the paper's matrices are symmetric indefinite and need two-by-two pivots):
restricted Bunch-Kaufman pivoting inside each front, pivots delayed to the
parent front when none of a front's fully-summed columns gives a stable
pivot.  x and the inverse diagonal are compared element by element with the
oracle's dense Bunch-Kaufman factorization (oracle.ldlt_pivoted,
oracle.inv_diag_pivoted), at a tolerance scaled by the matrix's condition
number (the pivot sequences differ: the GPU may only pivot inside a front)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle
from spigen import TINY, generate, random_spd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def lower(A):
    low = sp.tril(sp.csc_matrix(A)).tocsc()
    # the pattern keeps explicit zeros on the diagonal (a KKT block has none stored)
    low = (low + sp.diags(np.zeros(A.shape[0]), format="csc")).tocsc()
    low.sum_duplicates()
    low.sort_indices()
    n = A.shape[0]
    cp = low.indptr.astype(np.int64)
    ri = low.indices.astype(np.int32)
    va = low.data.astype(np.float64)
    # every column must start with its diagonal entry, stored even when zero
    cols, rows, vals = [], [], []
    for j in range(n):
        r, v = ri[cp[j]:cp[j + 1]], va[cp[j]:cp[j + 1]]
        if len(r) == 0 or r[0] != j:
            r, v = np.concatenate([[j], r]), np.concatenate([[0.0], v])
        rows.append(r); vals.append(v)
    cp2 = np.zeros(n + 1, np.int64)
    cp2[1:] = np.cumsum([len(r) for r in rows])
    return n, cp2, np.concatenate(rows).astype(np.int32), np.concatenate(vals)


def oracle_solve_pivoted(A, b):
    """x = A^-1 b through the oracle's pivoted factorization A[p][:, p] = L D L^T."""
    p, L, D, _ = oracle.ldlt_pivoted(A)
    y = sla.solve_triangular(L, b[p], lower=True, unit_diagonal=True)
    w = np.linalg.solve(D, y)
    z = sla.solve_triangular(L.T, w, lower=False, unit_diagonal=True)
    x = np.empty_like(b)
    x[p] = z
    return x


def kkt(n1, n2, seed):
    rng = np.random.default_rng(seed)
    Bm = sp.random(n1, n1, density=4.0 / n1, random_state=rng, format="csr")
    A = (Bm @ Bm.T + sp.identity(n1)).toarray()
    C = np.zeros((n2, n1))
    for i in range(n2):  # full row rank: each constraint touches a few primal unknowns
        cols = rng.choice(n1, 3, replace=False)
        C[i, cols] = rng.uniform(0.5, 1.5, 3) * rng.choice([-1.0, 1.0], 3)
    K = np.zeros((n1 + n2, n1 + n2))
    K[:n1, :n1] = A
    K[n1:, :n1] = C
    K[:n1, n1:] = C.T
    return K


def indefinite(n, seed, density=0.05):
    rng = np.random.default_rng(seed)
    S = sp.random(n, n, density=density, random_state=rng).toarray()
    S = S + S.T
    S[np.diag_indices(n)] = rng.uniform(-1.0, 1.0, n)
    return S


def check(P, A, ordering=0):
    n, cp, ri, va = lower(A)
    b = np.random.default_rng(n).standard_normal(n)
    s = P.Solver(n, cp, ri, pivoting=True, ordering=ordering)
    s.factor(va)
    x = s.solve(b)
    v = s.diag_inverse()
    x_ref = oracle_solve_pivoted(A, b)
    v_ref = oracle.inv_diag_pivoted(A)
    kappa = np.linalg.cond(A)
    tol = 64 * np.finfo(float).eps * max(kappa, 10.0)
    ex = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    ev = np.abs(v - v_ref).max() / np.abs(v_ref).max()
    info = s.info()
    print(f"n={n} kappa={kappa:.1e} x_err={ex:.2e} var_err={ev:.2e} tol={tol:.1e} 2x2={info['pivots_2x2']} "
          f"delays={info['pivot_delays']} restarts={info['pivot_restarts']} supernodes={info['n_supernodes']}")
    assert ex <= tol and ev <= tol
    # each variance against its own scale, too (they have both signs here)
    assert np.all(np.abs(v - v_ref) <= tol * np.maximum(np.abs(v_ref), np.abs(v_ref).max() * 1e-3))
    return s, info


@pytest.mark.parametrize("n1,n2,seed", [(30, 10, 1), (120, 40, 2), (400, 90, 3)])
@pytest.mark.parametrize("ordering", [0, 1])
def test_kkt_saddle_point(P, n1, n2, seed, ordering):
    """[[A, C^T], [C, 0]]: the zero diagonal block has no 1x1 pivot of its own; leaf
    fronts holding only constraint columns delay their pivots to their parents,
    where 1x1 or 2x2 pivots pair them with primal unknowns."""
    _, info = check(P, kkt(n1, n2, seed), ordering)
    if ordering == 0:
        # nested dissection eliminates the constraints (few neighbours) first, as leaf
        # fronts whose only fully-summed column has a zero diagonal: they must delay
        assert info["pivot_delays"] > 0 and info["pivot_restarts"] > 0


@pytest.mark.parametrize("n,seed,density", [(20, 4, 0.3), (150, 5, 0.04), (600, 6, 0.01)])
def test_random_indefinite(P, n, seed, density):
    check(P, indefinite(n, seed, density))


def test_spd_through_the_pivoting_path(P):
    """An SPD matrix takes 1x1 pivots only and gives the plain path's results."""
    pb = generate(TINY)
    A = pb.full_matrix().toarray()
    s, info = check(P, A)
    assert info["pivots_2x2"] == 0 and info["pivot_delays"] == 0
    plain = P.Solver.for_problem(pb)
    plain.factor(pb.values)
    assert np.allclose(plain.diag_inverse(), s.diag_inverse(), rtol=1e-10, atol=0)


def test_shifted_spd_matrix(P):
    """A sparse SPD matrix shifted into indefiniteness (A - sigma I, sigma between
    two of its eigenvalues): mixed-sign pivots on an SPD matrix's structure."""
    pb = random_spd(200, 0.03, 7)
    A = pb.full_matrix().toarray()
    ev = np.linalg.eigvalsh(A)
    sigma = 0.5 * (ev[40] + ev[41])
    check(P, A - sigma * np.eye(A.shape[0]))


def test_singular_reported(P):
    """A singular symmetric matrix (a zero row and column) ends in SPI_ERR_NOT_SPD
    once no front can pivot, root included."""
    A = indefinite(30, 8, 0.2)
    A[7, :] = 0.0
    A[:, 7] = 0.0
    n, cp, ri, va = lower(A)
    s = P.Solver(n, cp, ri, pivoting=True)
    with pytest.raises(P.SpiError) as e:
        s.factor(va)
    assert e.value.code == 3


def test_pivoting_restrictions(P):
    pb = random_spd(40, 0.2, 9)
    with pytest.raises(P.SpiError):
        P.Solver.for_problem(pb, pivoting=True, precision=P.SPI_PREC_MIXED_FP32)
    s = P.Solver.for_problem(pb, pivoting=True)
    s.factor(pb.values)
    with pytest.raises(P.SpiError):
        s.inverse_block(np.arange(5, dtype=np.int32))
