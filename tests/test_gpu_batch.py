"""Batched forms against the oracle, band by band / problem by problem:
same-pattern energy bands (one launch per level over all bands) and uneven
independent problems (one block-diagonal forest)."""
import numpy as np
import pytest

import oracle
from spigen import BAND, generate_bands, generate_uneven, random_spd, scaled

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


@pytest.fixture(scope="module")
def bands():
    return generate_bands(scaled(BAND, 600, seed=4), 5)


def test_same_pattern_bands_fp64(P, bands):
    nb, n = bands.nbands, bands.n
    s = P.Solver(n, bands.colptr, bands.rowind, batch=nb)
    s.factor_batch(bands.values)
    x = s.solve_batch(bands.b)
    v = s.diag_inverse_batch()
    for k in range(nb):
        pb = bands.band(k)
        f = oracle.OracleFactor.from_problem(pb)
        xr, vr = f.solve(pb.b), f.inv_diag()
        assert np.abs(x[k * n:(k + 1) * n] - xr).max() <= TOL * np.abs(xr).max(), k
        assert (np.abs(v[k * n:(k + 1) * n] - vr) / vr).max() <= TOL, k


def test_batch_matches_single_calls(P, bands):
    nb, n = bands.nbands, bands.n
    sb = P.Solver(n, bands.colptr, bands.rowind, batch=nb)
    sb.factor_batch(bands.values)
    vb = sb.diag_inverse_batch()
    ss = P.Solver(n, bands.colptr, bands.rowind)
    for k in range(nb):
        ss.factor(bands.band(k).values)
        vs = ss.diag_inverse()
        assert np.abs(vb[k * n:(k + 1) * n] - vs).max() <= 1e-13 * np.abs(vs).max()
    # fewer bands than the context holds
    sb.factor_batch(bands.values[: 2 * bands.nnz], nbatch=2)
    v2 = sb.diag_inverse_batch(nbatch=2)
    assert np.abs(v2 - vb[: 2 * n]).max() <= 1e-13 * np.abs(vb).max()


def test_same_pattern_bands_mixed(P, bands):
    nb, n = bands.nbands, bands.n
    s = P.Solver(n, bands.colptr, bands.rowind, batch=nb, precision=P.SPI_PREC_MIXED_FP32)
    s.factor_batch(bands.values)
    x = s.solve_batch(bands.b)
    v = s.diag_inverse_batch()
    assert s.info()["solve_relres"] <= 1e-13
    for k in range(nb):
        pb = bands.band(k)
        f = oracle.OracleFactor.from_problem(pb)
        xr, vr = f.solve(pb.b), f.inv_diag()
        assert np.abs(x[k * n:(k + 1) * n] - xr).max() <= 1e-8 * np.abs(xr).max(), k
        assert (np.abs(v[k * n:(k + 1) * n] - vr) / vr).max() <= 3e-5, k


def test_bad_band_reported(P, bands):
    vals = bands.values.copy()
    bad_band, bad_col = 3, 11
    vals[bad_band * bands.nnz + bands.colptr[bad_col]] = -5.0
    s = P.Solver(bands.n, bands.colptr, bands.rowind, batch=bands.nbands)
    with pytest.raises(P.SpiError) as e:
        s.factor_batch(vals)
    assert e.value.code == 3
    info = s.info()
    assert info["bad_band"] == bad_band and info["bad_pivot"] == bad_col


def test_uneven_problems_as_one_forest(P):
    probs = generate_uneven(6) + [random_spd(50, 0.1, 2), random_spd(1, 1.0, 3)]
    s = P.Solver.for_problems(probs)
    vals = np.concatenate([p.values for p in probs])
    b = np.concatenate([p.b for p in probs])
    s.factor(vals)
    x = s.solve(b)
    v = s.diag_inverse()
    off = 0
    for p in probs:
        f = oracle.OracleFactor.from_problem(p)
        xr, vr = f.solve(p.b), f.inv_diag()
        assert np.abs(x[off:off + p.n] - xr).max() <= TOL * np.abs(xr).max()
        assert (np.abs(v[off:off + p.n] - vr) / vr).max() <= TOL
        off += p.n
    assert off == s.n


def test_autotuned_block_size(P):
    pb = generate_bands(scaled(BAND, 1500, seed=2), 1).band(0)
    s = P.Solver.for_problem(pb)  # rhs_block = 0: the autotuner picks it
    s.factor(pb.values)
    v1 = s.diag_inverse()
    B = s.info()["rhs_block"]
    assert B in (16, 32, 64)
    v2 = s.diag_inverse()
    assert np.array_equal(v1, v2)
    vr = oracle.OracleFactor.from_problem(pb).inv_diag()
    assert (np.abs(v1 - vr) / vr).max() <= TOL


def test_shard_solve_share_matches_oracle(P):
    """One rank's share of independent problems, as the multi-GPU path runs
    it on each GPU (here: every share in turn on this one)."""
    from paper_1305_5683_gb300 import shard
    probs = generate_uneven(4) + [random_spd(60, 0.1, 5)]
    parts = shard.assign(shard.problem_costs(probs), 2)
    for idx in parts:
        xs, vs = shard.solve_share(probs, idx)
        for i, x, v in zip(idx, xs, vs):
            f = oracle.OracleFactor.from_problem(probs[i])
            xr, vr = f.solve(probs[i].b), f.inv_diag()
            assert np.abs(x - xr).max() <= TOL * np.abs(xr).max()
            assert (np.abs(v - vr) / vr).max() <= TOL
