"""The Poisson maximum-likelihood Newton loop on the device (Hessian
H^T diag(y/e^2) H assembled, factored and solved every step) against the
oracle's loop: same fit and Hessian-inverse diagonal."""
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


def lsq_start(P, pb):
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    return s.solve(pb.b)


@pytest.mark.parametrize("cfg", [TINY, scaled(SCALE, 1500, seed=7)])
def test_mle_matches_oracle(P, cfg):
    pb = generate(cfg, sparse_design=True)
    x0 = lsq_start(P, pb)
    xr, vr, kr = oracle.mle_newton(pb.H, pb.y, x0)
    s = P.Solver.for_problem(pb).normal_setup(pb.H)
    x, v = s.mle_newton(pb.H.data, pb.y, x0)
    info = s.info()
    print(f"n={pb.n} steps gpu={info['mle_steps']} oracle={kr} cash={info['mle_cash']:.6e}")
    assert np.abs(x - xr).max() <= 1e-9 * np.abs(xr).max()
    assert (np.abs(v - vr) / vr).max() <= 1e-8
    assert info["mle_cash"] == pytest.approx(oracle.cash(pb.H, pb.y, xr), rel=1e-12)


def test_mle_noise_free_returns_the_truth_and_mixed_agrees(P):
    pb = generate(scaled(SCALE, 1500, seed=8), sparse_design=True, noise=False)
    x0 = lsq_start(P, pb)
    for prec in (P.SPI_PREC_FP64, P.SPI_PREC_MIXED_FP32):
        s = P.Solver.for_problem(pb, precision=prec).normal_setup(pb.H)
        x, _ = s.mle_newton(pb.H.data, pb.y, x0, variances=False)
        assert np.abs(x - pb.x_true).max() <= 1e-8 * np.abs(pb.x_true).max()


def test_mle_rejects_a_nonpositive_start(P):
    pb = generate(TINY, sparse_design=True)
    s = P.Solver.for_problem(pb).normal_setup(pb.H)
    with pytest.raises(P.SpiError) as e:
        s.mle_newton(pb.H.data, pb.y, -np.ones(pb.n))
    assert e.value.code == 1
