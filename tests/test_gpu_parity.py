"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bar (FP64 form): relative error <= 1e-10 for x (max-norm relative) and for
every variance (max_i |v_i - v_i^oracle| / v_i^oracle)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from spigen import SCALE, TINY, generate, random_spd, scaled

pytestmark = pytest.mark.gpu
TOL = 1e-10


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
    low.sum_duplicates(); low.sort_indices()
    return low.shape[0], low.indptr.astype(np.int64), low.indices.astype(np.int32), low.data.astype(np.float64)


def check(P, n, cp, ri, va, b, **opts):
    f = oracle.OracleFactor(n, cp, ri, va)
    x_ref, v_ref = f.solve(b), f.inv_diag()
    s = P.Solver(n, cp, ri, **opts)
    s.factor(va)
    x = s.solve(b)
    v = s.diag_inverse()
    ex = np.abs(x - x_ref).max() / max(np.abs(x_ref).max(), 1e-300)
    ev = (np.abs(v - v_ref) / v_ref).max() if n else 0.0
    assert ex <= TOL, f"x rel err {ex:.3e}"
    assert ev <= TOL, f"variance rel err {ev:.3e}"
    return s, f


@pytest.mark.parametrize("ordering", [0, 1])
def test_tiny_spi(P, ordering):
    pb = generate(TINY)
    check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, ordering=ordering)


@pytest.mark.parametrize("n,dens,seed", [(1, 1.0, 0), (2, 1.0, 1), (31, 0.3, 2), (33, 0.2, 3),
                                         (97, 0.05, 4), (257, 0.02, 5), (300, 0.01, 6)])
@pytest.mark.parametrize("ordering", [0, 1])
def test_random_spd(P, n, dens, seed, ordering):
    pb = random_spd(n, dens, seed)
    check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, ordering=ordering)


@pytest.mark.parametrize("n", [32, 64, 65, 130])
def test_dense_single_front(P, n):
    """A dense SPD matrix is one front: several block columns and a ragged tail."""
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    check(P, *lower(A), rng.standard_normal(n), ordering=1)


def test_diagonal_matrix(P):
    d = np.linspace(1.0, 5.0, 77)
    n, cp, ri, va = lower(np.diag(d))
    s, _ = check(P, n, cp, ri, va, np.ones(77))
    assert np.array_equal(s.diag_inverse(), 1.0 / d)


@pytest.mark.parametrize("relax", [0, 10, 60])
@pytest.mark.parametrize("rhs_block", [1, 7, 32, 128])
def test_blocking_and_amalgamation(P, relax, rhs_block):
    pb = generate(scaled(TINY, 600, seed=11))
    check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, relax=relax, rhs_block=rhs_block)


def test_index_subset_and_order(P):
    pb = generate(TINY)
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    rng = np.random.default_rng(3)
    for m in (0, 1, 5, 200):
        idx = rng.permutation(pb.n)[:m].astype(np.int32)
        v = s.diag_inverse(idx)
        if m:
            ref = f.inv_diag(idx)
            assert (np.abs(v - ref) / ref).max() <= TOL
    # repeated call with the same set reuses the plan
    idx = rng.permutation(pb.n)[:50].astype(np.int32)
    v1 = s.diag_inverse(idx); v2 = s.diag_inverse(idx)
    assert np.array_equal(v1, v2)


def test_device_buffers(P):
    import torch
    pb = generate(TINY)
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    dev = torch.device("cuda:0")
    st = torch.cuda.current_stream()
    s.factor(torch.from_numpy(pb.values).to(dev), stream=st)
    xb = torch.from_numpy(pb.b).to(dev)
    x = s.solve(xb, stream=st)
    v = s.diag_inverse(device=dev, stream=st)
    idx = torch.arange(0, pb.n, 3, dtype=torch.int32, device=dev)
    vs = s.diag_inverse(idx, stream=st)
    torch.cuda.synchronize()
    x_ref, v_ref = f.solve(pb.b), f.inv_diag()
    assert np.abs(x.cpu().numpy() - x_ref).max() <= TOL * np.abs(x_ref).max()
    assert (np.abs(v.cpu().numpy() - v_ref) / v_ref).max() <= TOL
    assert (np.abs(vs.cpu().numpy() - v_ref[::3]) / v_ref[::3]).max() <= TOL
    # x may alias b
    s.solve(xb, xb, stream=st)
    torch.cuda.synchronize()
    assert np.abs(xb.cpu().numpy() - x_ref).max() <= TOL * np.abs(x_ref).max()


def test_refactor_same_pattern(P):
    pb = generate(TINY)
    s = P.Solver.for_problem(pb)
    rng = np.random.default_rng(1)
    for scale in (1.0, 2.5):
        vals = pb.values * scale
        vals[pb.colptr[:-1]] += rng.uniform(0, 1, pb.n)  # perturb the diagonal
        f = oracle.OracleFactor(pb.n, pb.colptr, pb.rowind, vals)
        s.factor(vals)
        v = s.diag_inverse()
        assert (np.abs(v - f.inv_diag()) / f.inv_diag()).max() <= TOL


def test_not_spd_reports_column(P):
    pb = random_spd(60, 0.1, 9)
    vals = pb.values.copy()
    bad = 23
    vals[pb.colptr[bad]] = -1.0
    s = P.Solver.for_problem(pb)
    with pytest.raises(P.SpiError) as e:
        s.factor(vals)
    assert e.value.code == 3
    assert s.info()["bad_pivot"] == bad
    with pytest.raises(P.SpiError) as e:
        s.diag_inverse()
    assert e.value.code == 7  # no usable factor
    s.factor(pb.values)  # recovers with good values
    s.diag_inverse()


def test_spi_mid_size_nd(P):
    pb = generate(scaled(SCALE, 2000, seed=5))
    check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b)


def test_full_size_sampled():
    """The benchmark workload (P = 20,000, full diag(N^-1) in FP64, the
    launch configuration the benchmark times): every variance is positive and
    >= 1/N_ii, x meets the residual bound, and 256 sampled variances plus x
    match the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    pb = generate(SCALE)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    x = s.solve(pb.b)
    v = s.diag_inverse()
    A = pb.full_matrix()
    assert np.linalg.norm(A @ x - pb.b) <= 1e-12 * np.linalg.norm(pb.b)
    assert np.all(v > 0) and np.all(v * A.diagonal() >= 1 - 1e-12)
    f = oracle.OracleFactor.from_problem(pb)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(pb.n, 250, replace=False), [0, pb.n - 1, pb.n_pointing,
                          pb.n_pointing - 1, pb.n_pointing + pb.n_detcol, pb.n // 2]]).astype(np.int32)
    ref = f.inv_diag(idx)
    assert (np.abs(v[idx] - ref) / ref).max() <= TOL
    x_ref = f.solve(pb.b)
    assert np.abs(x - x_ref).max() <= TOL * np.abs(x_ref).max()


def test_unpruned_ablation_matches_pruned(P):
    """spi_options.diag_unpruned (full forward solves, no pruning) gives the
    pruned variances: same values up to rounding, for a subset and for all."""
    pb = generate(scaled(SCALE, 2000, seed=5))
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    u = P.Solver.for_problem(pb, diag_unpruned=True)
    u.factor(pb.values)
    idx = np.random.default_rng(9).choice(pb.n, 100, replace=False).astype(np.int32)
    vu, vp = u.diag_inverse(idx), s.diag_inverse(idx)
    assert (np.abs(vu - vp) / vp).max() <= 1e-12
    assert (np.abs(vu - f.inv_diag(idx)) / vp).max() <= 1e-10
    allu, allp = u.diag_inverse(), s.diag_inverse()
    assert (np.abs(allu - allp) / allp).max() <= 1e-12
    assert u.info()["diag_work_flops"] > 10 * s.info()["diag_work_flops"]


@pytest.mark.parametrize("dag", [1, 2])
@pytest.mark.parametrize("force_panel", [1, 2])
@pytest.mark.parametrize("make", [lambda: generate(TINY), lambda: generate(scaled(SCALE, 2000, seed=5)),
                                  lambda: random_spd(300, 0.02, 11), lambda: random_spd(700, 0.01, 12)])
def test_panel_paths(P, make, force_panel, dag):
    """The ways of running the factorization, each against the oracle at the FP64
    bar: launches level by level (dag 1) with every front's panel on the chain of
    32-column block-step launches or in the persistent per-level kernel (one CTA
    runs all block steps of a front), and the same two panel forms as tasks of
    the single dependency-driven launch (dag 2)."""
    pb = make()
    s, _ = check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, force_panel=force_panel, dag=dag)
    info = s.info()
    if dag == 1:
        assert info["factor_dag_tasks"] == 0
        assert (info["launches_factor_fused"] > 0) == (force_panel == 2)
        if force_panel == 2:
            assert info["launches_factor"] < 2 + 3 * info["n_levels"] + 64  # about one panel launch per level
    else:
        assert info["factor_dag_tasks"] > 0 and info["factor_dag_levels"] == info["n_levels"]
        assert info["launches_factor"] == 3  # status reset, assembly, the one dependency-driven launch


def test_dag_batched_bands(P):
    """The dependency-driven launch over a batch of same-pattern bands (one set of
    counters per band) against the oracle band by band."""
    from spigen import BAND, generate_bands
    bands = generate_bands(scaled(BAND, 600, seed=4), 3)
    n = bands.n
    s = P.Solver(n, bands.colptr, bands.rowind, batch=bands.nbands, dag=2)
    s.factor_batch(bands.values)
    x = s.solve_batch(bands.b)
    v = s.diag_inverse_batch()
    assert s.info()["factor_dag_tasks"] > 0
    for k in range(bands.nbands):
        pb = bands.band(k)
        f = oracle.OracleFactor.from_problem(pb)
        xr, vr = f.solve(pb.b), f.inv_diag()
        assert np.abs(x[k * n:(k + 1) * n] - xr).max() <= TOL * np.abs(xr).max(), k
        assert (np.abs(v[k * n:(k + 1) * n] - vr) / vr).max() <= TOL, k


def test_dag_timeout_reported(P):
    """wait_limit < 0 makes every bounded wait give up at once: the dependency-
    driven launch raises the timeout flag at its first dependent task, every CTA
    skips the rest, spi_factor returns SPI_ERR_TIMEOUT, and a fresh context on the
    device still factors correctly.  No wait is unbounded; nothing faults."""
    pb = generate(TINY)
    s = P.Solver.for_problem(pb, dag=2, wait_limit=-1)
    with pytest.raises(P.SpiError) as e:
        s.factor(pb.values)
    assert e.value.code == 6
    check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, dag=2)


def test_autotuner_and_tune_cache(P, tmp_path):
    """autotune = 1 times both candidates of every bucket on the first factorization
    (tune_source 1) and writes the table; a second context with the same cache
    reads it (tune_source 2) and builds the same plan; both match the oracle."""
    pb = generate(scaled(SCALE, 2000, seed=5))
    cache = tmp_path / "tune.txt"
    s1, _ = check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, autotune=1, tune_cache=str(cache))
    i1 = s1.info()
    assert i1["tune_source"] == 1 and i1["tune_seconds"] > 0 and i1["tune_panel_buckets"] > 0
    lines = [l.split() for l in cache.read_text().splitlines() if not l.startswith("#")]
    assert sum(l[3] in "PS" for l in lines) == i1["tune_panel_buckets"] + i1["tune_schur_buckets"]
    assert sum(l[3] == "D" for l in lines) == 1  # launches level by level against the dependency-driven launch
    # the same for the solve, timed at the first solve
    assert sum(l[3] == "V" for l in lines) == (1 if i1["tune_solve_ms_launches"] > 0 else 0)
    assert i1["tune_ms_launches"] > 0 and i1["tune_ms_dag"] > 0
    s2, _ = check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, autotune=1, tune_cache=str(cache))
    i2 = s2.info()
    assert i2["tune_source"] == 2
    for k in ("launches_factor", "launches_factor_fused", "tune_panel_fused", "factor_dag_tasks"):
        assert i1[k] == i2[k], k
    # the rules alone (no timing) are a valid plan too
    s3, _ = check(P, pb.n, pb.colptr, pb.rowind, pb.values, pb.b, autotune=-1)
    assert s3.info()["tune_source"] == 0
