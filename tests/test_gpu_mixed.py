"""Mixed-precision form (FP64 pivot tiles, FP32 panel/Schur updates and
variance solves, FP64 variance accumulation, FP64 refinement of x) against
the FP64 oracle.  Bounds: x after refinement <= 1e-8 relative (the stated
bound of the mixed form is 1e-6); variances within MIXED_VAR_TOL relative
(first order in the FP32 factor error; they are not refined)."""
import numpy as np
import pytest

import oracle
from spigen import SCALE, TINY, generate, random_spd, scaled

pytestmark = pytest.mark.gpu
X_TOL = 1e-8
MIXED_VAR_TOL = 1e-4


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
