"""Blocks of the inverse (covariances of selected unknowns) through the C ABI
against the oracle, entry by entry on the scale sqrt(v_s v_t) of each entry:
FP64 bar 1e-10; in a mixed-precision context the same bound as its variances."""
import numpy as np
import pytest

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


def rel_err(G, Gref):
    v = np.diag(Gref)
    return (np.abs(G - Gref) / np.sqrt(np.outer(v, v))).max()


def test_whole_inverse_of_a_tiny_problem(P):
    pb = generate(TINY)  # n = 463 <= SPI_INVERSE_BLOCK_MAX: the whole inverse
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    idx = np.arange(pb.n, dtype=np.int32)
    G = s.inverse_block(idx)
    Gref = f.inv_block(idx)
    assert rel_err(G, Gref) <= TOL
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("mixed", [False, True])
def test_random_index_sets(P, mixed):
    pb = generate(scaled(SCALE, 2000, seed=5))
    f = oracle.OracleFactor.from_problem(pb)
    prec = P.SPI_PREC_MIXED_FP32 if mixed else P.SPI_PREC_FP64
    s = P.Solver.for_problem(pb, precision=prec)
    s.factor(pb.values)
    rng = np.random.default_rng(7)
    for m in (1, 37, 300, 512):
        idx = rng.choice(pb.n, m, replace=False).astype(np.int32)
        G = s.inverse_block(idx)
        err = rel_err(G, f.inv_block(idx))
        assert err <= (1e-4 if mixed else TOL), (m, err)
        # its diagonal is the variances of the same unknowns
        v = s.diag_inverse(idx)
        assert np.abs(np.diag(G) - v).max() <= (1e-4 if mixed else 1e-12) * v.max()


def test_device_buffers_and_errors(P):
    import torch
    pb = random_spd(300, 0.02, 9)
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    idx = torch.tensor([5, 250, 17, 99], dtype=torch.int32, device="cuda")
    G = s.inverse_block(idx)
    torch.cuda.synchronize()
    assert rel_err(G.cpu().numpy(), f.inv_block(idx.cpu().numpy())) <= TOL
    for bad in ([3, 3], [0, 300], [-1]):
        with pytest.raises(P.SpiError) as e:
            s.inverse_block(np.array(bad, np.int32))
        assert e.value.code == 1
    with pytest.raises(P.SpiError) as e:
        s.inverse_block(np.arange(513, dtype=np.int32) % 300)
    assert e.value.code == 1
