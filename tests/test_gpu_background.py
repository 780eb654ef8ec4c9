"""Algorithm 1 (the empty-field pattern fitted with the solution) on the
device against the oracle's loop: the statistic of every solve, the pattern,
the solution, the variances and the rewritten design matrix."""
import numpy as np
import pytest

import oracle
from spigen import SCALE, TINY, generate, scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def perturbed(u, seed=1):
    rng = np.random.default_rng(seed)
    return u * (1 + 0.2 * rng.uniform(-1, 1, len(u)))


def check_against_oracle(P, pb, upat, U0, mode, max_iter, tol, precision=None, rel=1e-8):
    k0 = pb.n_pointing
    xr, Ur, sr, vr = oracle.background_fit(pb.H, pb.y, pb.w, k0, upat, pb.bg_t, U0, mode=mode,
                                           max_iter=max_iter, tol=tol)
    kw = {} if precision is None else {"precision": precision}
    s = P.Solver.for_problem(pb, **kw).normal_setup(pb.H)
    hv = pb.H.data.copy()
    x, U, st, v = s.background_fit(k0, upat, pb.bg_t, hv, pb.w, pb.y, U0, mode=mode, max_iter=max_iter, tol=tol)
    print(f"{mode} n={pb.n} solves gpu={len(st)} oracle={len(sr)} stat {st[0]:.9e} -> {st[-1]:.9e}")
    assert len(st) == len(sr)
    assert np.abs(st - sr).max() <= rel * np.abs(sr).max()
    assert np.abs(U - Ur).max() <= rel * np.abs(Ur).max()
    assert np.abs(x - xr).max() <= rel * np.abs(xr).max()
    assert (np.abs(v - vr) / vr).max() <= max(rel, 1e-8)
    assert s.info()["bg_stat"] == pytest.approx(sr[-1] if sr[-1] <= sr[max(len(sr) - 2, 0)] else sr[-2], rel=rel)
    # H comes back with the returned pattern in its background entries
    Hr = oracle.set_background(pb.H, k0, upat, pb.bg_t, Ur)
    assert np.abs(hv - Hr.data).max() <= rel * np.abs(Hr.data).max()
    return s


@pytest.mark.parametrize("cfg", [TINY, scaled(SCALE, 1500, seed=7)])
def test_least_squares_loop_matches_oracle(P, cfg):
    pb = generate(cfg, sparse_design=True)
    check_against_oracle(P, pb, pb.bg_pat, perturbed(pb.bg_u), "lsq", 4, 0.0)


def test_likelihood_loop_matches_oracle(P):
    pb = generate(TINY, sparse_design=True)
    check_against_oracle(P, pb, pb.bg_pat, perturbed(pb.bg_u), "mle", 3, 0.0)


def test_interval_pattern_and_stop_rule(P):
    """A pattern per detector and interval of 100 pointings (U(d, k)); a
    tolerance of 1 stops after the second solve."""
    pb = generate(TINY, sparse_design=True)
    p = np.arange(pb.H.shape[0]) // 19
    upat = (pb.bg_pat + 19 * (p // 100)).astype(np.int32)
    U0 = np.tile(perturbed(pb.bg_u), 3)
    check_against_oracle(P, pb, upat, U0, "lsq", 3, 0.0)
    s = check_against_oracle(P, pb, upat, U0, "lsq", 10, 1.0)
    assert s.info()["bg_iters"] == 2


def test_noise_free_fixed_point_device_buffers_and_mixed(P):
    import torch
    pb = generate(scaled(SCALE, 1500, seed=8), sparse_design=True, noise=False)
    k0 = pb.n_pointing
    dev = torch.device("cuda:0")
    for prec in (P.SPI_PREC_FP64, P.SPI_PREC_MIXED_FP32):
        s = P.Solver.for_problem(pb, precision=prec).normal_setup(pb.H)
        hv = torch.tensor(pb.H.data, device=dev)
        args = [torch.tensor(a, device=dev) for a in (pb.bg_pat, pb.bg_t)]
        w, y = torch.tensor(pb.w, device=dev), torch.tensor(pb.y, device=dev)
        x, U, st, v = s.background_fit(k0, args[0], args[1], hv, w, y, pb.bg_u, max_iter=3)
        x, U = x.cpu().numpy(), U.cpu().numpy()
        assert np.abs(x - pb.x_true).max() <= 1e-7 * np.abs(pb.x_true).max()
        assert np.abs(U - pb.bg_u).max() <= 1e-7 * pb.bg_u.max()
        assert bool((v > 0).all())


def test_mixed_precision_loop_follows_fp64(P):
    pb = generate(TINY, sparse_design=True)
    U0 = perturbed(pb.bg_u)
    res = []
    for prec in (P.SPI_PREC_FP64, P.SPI_PREC_MIXED_FP32):
        s = P.Solver.for_problem(pb, precision=prec).normal_setup(pb.H)
        res.append(s.background_fit(pb.n_pointing, pb.bg_pat, pb.bg_t, pb.H.data.copy(), pb.w, pb.y, U0,
                                    max_iter=4, tol=0.0))
    (x0, U0_, s0, v0), (x1, U1, s1, v1) = res
    assert np.abs(U1 - U0_).max() <= 1e-7 * U0_.max()
    assert np.abs(s1 - s0).max() <= 1e-8 * s0.max()
    assert (np.abs(v1 - v0) / v0).max() <= 1e-4


def test_rejects_a_pattern_index_that_does_not_match(P):
    pb = generate(TINY, sparse_design=True)
    s = P.Solver.for_problem(pb).normal_setup(pb.H)
    upat = pb.bg_pat.copy()
    upat[5] = -1  # row 5 has a background entry
    with pytest.raises(P.SpiError) as e:
        s.background_fit(pb.n_pointing, upat, pb.bg_t, pb.H.data.copy(), pb.w, pb.y, pb.bg_u)
    assert e.value.code == 1
    upat[5] = 19  # beyond npat
    with pytest.raises(P.SpiError) as e:
        s.background_fit(pb.n_pointing, upat, pb.bg_t, pb.H.data.copy(), pb.w, pb.y, pb.bg_u)
    assert e.value.code == 1
