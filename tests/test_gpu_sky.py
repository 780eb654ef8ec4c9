"""Diffuse-sky problems (point sources plus a pixel grid, pointings on a
target grid) against the oracle: the FP64 form element by element, the
mixed form within its bounds, variances requested for the sky columns only.
The second problem has a dense sky front of more than 2,048 rows, so the
mixed form runs its tensor-core trailing updates there."""
import numpy as np
import pytest

import oracle
from spigen import generate, sky_scaled

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


def test_sky_fp64_against_oracle(P):
    pb = generate(sky_scaled(3000, 2.0, 60))
    f = oracle.OracleFactor.from_problem(pb)
    x_ref, v_ref = f.solve(pb.b), f.inv_diag()
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    x = s.solve(pb.b)
    v = s.diag_inverse()
    vs = s.diag_inverse(pb.sky_columns)
    assert np.abs(x - x_ref).max() <= TOL * np.abs(x_ref).max()
    assert (np.abs(v - v_ref) / v_ref).max() <= TOL
    assert np.array_equal(vs, v[pb.sky_columns])


def test_sky_mixed_with_tensor_core_fronts(P):
    pb = generate(sky_scaled(1500, 1.2, 40))
    f = oracle.OracleFactor.from_problem(pb)
    x_ref, v_ref = f.solve(pb.b), f.inv_diag(pb.sky_columns)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    s.factor(pb.values)
    info = s.info()
    assert info["max_front"] >= 2048
    assert info["launches_factor_tc"] > 0 and info["tiles_factor_tc"] > 0  # the tcgen05 path ran
    x = s.solve(pb.b)
    v = s.diag_inverse(pb.sky_columns)
    ex = np.abs(x - x_ref).max() / np.abs(x_ref).max()
    ev = (np.abs(v - v_ref) / v_ref).max()
    print(f"sky mixed n={pb.n} sky={pb.n_sky} max_front={info['max_front']} x_err={ex:.2e} var_err={ev:.2e}")
    assert s.info()["solve_relres"] <= 1e-13
    assert ex <= 1e-8
    assert ev <= 3e-5
