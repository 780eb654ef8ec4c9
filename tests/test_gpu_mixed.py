"""Mixed-precision form (FP64 pivot tiles, FP32 panel/Schur updates and
variance solves, FP64 variance accumulation, FP64 refinement of x) against
the FP64 oracle.  Bounds: x after refinement <= 1e-8 relative (the stated
bound of the mixed form is 1e-6); variances within MIXED_VAR_TOL relative
(first order in the FP32 factor error; they are not refined)."""
import numpy as np
import pytest

import oracle
from spigen import SCALE, TINY, generate, random_spd, scaled, sky_scaled

pytestmark = pytest.mark.gpu
X_TOL = 1e-8
MIXED_VAR_TOL = 3e-5  # measured: at most 2.3e-5 on the P = 20,000 workload, the largest problem


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def run(P, pb, **kw):
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32, **kw)
    s.factor(pb.values)
    x = s.solve(pb.b)
    v = s.diag_inverse()
    x_ref, v_ref = f.solve(pb.b), f.inv_diag()
    ex = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    ev = (np.abs(v - v_ref) / v_ref).max()
    return s, ex, ev


@pytest.mark.parametrize("make", [lambda: generate(TINY), lambda: generate(scaled(SCALE, 2000, seed=5)),
                                  lambda: random_spd(300, 0.01, 6)])
def test_mixed_against_oracle(P, make):
    pb = make()
    s, ex, ev = run(P, pb)
    info = s.info()
    print(f"n={pb.n} x_err={ex:.2e} var_err={ev:.2e} refine_steps={info['refine_steps']} "
          f"relres={info['solve_relres']:.2e}")
    assert info["solve_relres"] <= 1e-13
    assert ex <= X_TOL
    assert ev <= MIXED_VAR_TOL


def test_repeated_solves_plan_their_corrections(P):
    """A solve after a converged one first runs as many correction steps as that one
    needed, back to back, then checks the residual after every further step: new
    right-hand sides and a new factorization (values scaled) still end below the
    refinement tolerance, and never with fewer steps than planned."""
    pb = generate(scaled(SCALE, 2000, seed=5))
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    s.factor(pb.values)
    rng = np.random.default_rng(3)
    steps = []
    for k, scale in enumerate((1.0, 1.0, 1.0, 4.0, 1.0)):
        if k >= 3:  # a new factorization: values x 4, then back
            s.factor(pb.values * scale)
        b = rng.standard_normal(pb.n)
        x = s.solve(b)
        info = s.info()
        x_ref = f.solve(b) / scale
        ex = np.abs(x - x_ref).max() / np.abs(x_ref).max()
        steps.append(info["refine_steps"])
        print(f"solve {k}: scale={scale} refine_steps={info['refine_steps']} relres={info['solve_relres']:.2e} "
              f"x_err={ex:.2e}")
        assert info["solve_relres"] <= 1e-13 and ex <= X_TOL
        if k:
            assert steps[k] >= steps[k - 1]  # the planned steps run first
    assert steps[0] >= 1


@pytest.mark.parametrize("rhs_block", [1, 32, 128])
def test_mixed_blocking(P, rhs_block):
    pb = generate(TINY)
    _, ex, ev = run(P, pb, rhs_block=rhs_block)
    assert ex <= X_TOL and ev <= MIXED_VAR_TOL


def test_mixed_not_spd(P):
    pb = random_spd(40, 0.2, 3)
    vals = pb.values.copy()
    vals[pb.colptr[7]] = -2.0
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    with pytest.raises(P.SpiError) as e:
        s.factor(vals)
    assert e.value.code == 3 and s.info()["bad_pivot"] == 7


def test_mixed_device_buffers_and_alias(P):
    import torch
    pb = generate(TINY)
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    dev = torch.device("cuda:0")
    s.factor(torch.from_numpy(pb.values).to(dev))
    xb = torch.from_numpy(pb.b).to(dev)
    s.solve(xb, xb)
    torch.cuda.synchronize()
    x_ref = f.solve(pb.b)
    assert np.abs(xb.cpu().numpy() - x_ref).max() <= X_TOL * np.abs(x_ref).max()


def arrowhead(n_leaf=400, n_tail=2100, seed=0):
    """SPD arrowhead: independent leading columns, each coupled to every column
    of a dense tail, so the grouped leaf fronts have k = 32 pivots and
    n_tail rows below them (wide Schur updates)."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    n = n_leaf + n_tail
    A = np.zeros((n, n))
    A[:n_leaf, :n_leaf] = np.diag(rng.uniform(400.0, 600.0, n_leaf))
    C = rng.uniform(-0.5, 0.5, (n_tail, n_leaf))
    A[n_leaf:, :n_leaf] = C
    A[:n_leaf, n_leaf:] = C.T
    R = rng.uniform(-1.0, 1.0, (n_tail, n_tail))
    A[n_leaf:, n_leaf:] = R @ R.T / n_tail + 5.0 * np.eye(n_tail)
    low = sp.tril(sp.csc_matrix(A)).tocsc()
    low.sort_indices()
    return n, low.indptr.astype(np.int64), low.indices.astype(np.int32), low.data, rng.standard_normal(n)


def test_tensor_core_schur_fronts(P):
    """Fronts with >= 2048 rows below their pivots take the tcgen05 Schur path
    in the mixed form; the result must match the oracle like the SIMT path."""
    n, cp, ri, va, b = arrowhead()
    f = oracle.OracleFactor(n, cp, ri, va)
    x_ref, v_ref = f.solve(b), f.inv_diag()
    s = P.Solver(n, cp, ri, precision=P.SPI_PREC_MIXED_FP32, ordering=P.SPI_ORDER_NATURAL)
    s.factor(va)
    x = s.solve(b)
    v = s.diag_inverse()
    ex = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    ev = (np.abs(v - v_ref) / v_ref).max()
    print(f"tensor-core fronts: x_err={ex:.2e} var_err={ev:.2e}")
    info = s.info()
    assert info["launches_factor_tc"] > 0 and info["tiles_factor_tc"] > 0  # the tcgen05 path ran
    assert ex <= X_TOL and ev <= MIXED_VAR_TOL


@pytest.mark.parametrize("dag", [1, 2])
@pytest.mark.parametrize("force_schur", [1, 2])
@pytest.mark.parametrize("force_panel", [1, 2])
def test_mixed_paths_against_oracle(P, force_panel, force_schur, dag):
    """Every combination of the factorization's paths in mixed precision: panels on
    the block-step chain or in the persistent per-level kernel, Schur complements
    on the SIMT kernel with no tensor-core launch at all, or on the tensor cores
    (all fronts with >= 256 trailing rows and >= 32 pivots); each combination must
    meet the mixed bounds against the
    oracle, and the counters must show that the forced path ran."""
    pb = generate(sky_scaled(1500, 1.2, 40))  # fronts of up to ~3,000 rows
    s, ex, ev = run(P, pb, force_panel=force_panel, force_schur=force_schur, dag=dag)
    info = s.info()
    print(f"panel={force_panel} schur={force_schur} dag={dag} x_err={ex:.2e} var_err={ev:.2e} "
          f"fused={info['launches_factor_fused']} tc={info['launches_factor_tc']} tiles={info['tiles_factor_tc']} "
          f"dag_tasks={info['factor_dag_tasks']} dag_levels={info['factor_dag_levels']}")
    if dag == 1:
        assert (info["launches_factor_fused"] > 0) == (force_panel == 2)
    elif force_schur == 1:  # no tensor-core level: every level in the dependency-driven launch
        assert info["factor_dag_tasks"] > 0 and info["factor_dag_levels"] == info["n_levels"]
    else:  # the levels below the first one with a tensor-core launch
        assert info["factor_dag_levels"] < info["n_levels"]
    if force_schur == 1:
        assert info["launches_factor_tc"] == 0
    else:
        assert info["tiles_factor_tc"] > 0
    assert info["solve_relres"] <= 1e-13
    assert ex <= X_TOL and ev <= MIXED_VAR_TOL


def test_bounded_wait_timeout_reported(P):
    """wait_limit < 0 makes every bounded pipeline wait of the tcgen05 Schur
    kernel give up at once.  The kernel then drains its own MMAs, frees its
    tensor memory and raises the timeout flag: spi_factor returns
    SPI_ERR_TIMEOUT, the context refuses to solve, and the device stays usable
    (a fresh context on it factors the same matrix to the oracle's result).
    No wait is left unbounded and nothing faults."""
    n, cp, ri, va, b = arrowhead()
    s = P.Solver(n, cp, ri, precision=P.SPI_PREC_MIXED_FP32, ordering=P.SPI_ORDER_NATURAL, wait_limit=-1)
    with pytest.raises(P.SpiError) as e:
        s.factor(va)
    assert e.value.code == 6
    with pytest.raises(P.SpiError) as e:
        s.solve(b)
    assert e.value.code == 7
    # launched level by level, the FP64 form waits nowhere: the same option leaves it untouched
    s64 = P.Solver(n, cp, ri, ordering=P.SPI_ORDER_NATURAL, wait_limit=-1, dag=1)
    s64.factor(va)
    x_ref = oracle.OracleFactor(n, cp, ri, va).solve(b)
    assert np.abs(s64.solve(b) - x_ref).max() <= 1e-10 * np.abs(x_ref).max()
    ok = P.Solver(n, cp, ri, precision=P.SPI_PREC_MIXED_FP32, ordering=P.SPI_ORDER_NATURAL)
    ok.factor(va)
    assert np.abs(ok.solve(b) - x_ref).max() <= X_TOL * np.abs(x_ref).max()


def test_refined_variances(P):
    """spi_diag_inverse_refined: 2 e^T v - v^T N v with v from the mixed factor
    removes the first-order error of the mixed variances (O(delta^2) left, never
    above the exact variance); an FP64 context returns spi_diag_inverse's values."""
    import torch
    pb = generate(scaled(SCALE, 2000, seed=5))
    f = oracle.OracleFactor.from_problem(pb)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(pb.n, 70, replace=False), [0, pb.n - 1, 5, 5]]).astype(np.int32)
    ref = f.inv_diag(idx)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    s.factor(pb.values)
    plain = s.diag_inverse(idx)
    refined = s.diag_inverse_refined(idx)
    e_plain = (np.abs(plain - ref) / ref).max()
    e_ref = (np.abs(refined - ref) / ref).max()
    print(f"mixed variances: plain {e_plain:.2e}, refined {e_ref:.2e}")
    assert e_ref <= 1e-9
    assert e_ref <= 1e-2 * e_plain
    assert ((refined - ref) / ref).max() <= 1e-12  # a lower bound up to rounding
    d = s.diag_inverse_refined(torch.from_numpy(idx).cuda())
    torch.cuda.synchronize()
    assert np.allclose(d.cpu().numpy(), refined, rtol=1e-12, atol=0)  # atomics: last bits may differ
    s64 = P.Solver.for_problem(pb)
    s64.factor(pb.values)
    assert np.allclose(s64.diag_inverse_refined(idx), s64.diag_inverse(idx), rtol=1e-13, atol=0)
    with pytest.raises(P.SpiError) as e:
        s.diag_inverse_refined(np.array([pb.n], np.int32))
    assert e.value.code == 1
