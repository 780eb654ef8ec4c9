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


def test_scattered_entries_across_groups(P):
    """spi_inverse_entries: pairs over 700 distinct unknowns (three groups of
    256 in elimination order, so several blocks), repeated pairs, both
    orders and diagonal entries, against the oracle's block of those
    unknowns, each entry on the scale sqrt(v_i v_j)."""
    pb = generate(scaled(SCALE, 2000, seed=5))
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    rng = np.random.default_rng(3)
    U = rng.choice(pb.n, 700, replace=False).astype(np.int32)
    Gref = f.inv_block(U)
    pos = {int(u): t for t, u in enumerate(U)}
    a = rng.integers(0, 700, 3000)
    b = rng.integers(0, 700, 3000)
    a[:50] = b[:50]                         # diagonal entries
    a[50:60], b[50:60] = b[60:70], a[60:70]  # both orders of a few pairs
    a[70:80], b[70:80] = a[60:70], b[60:70]  # repeats
    rows, cols = U[a], U[b]
    out = s.inverse_entries(rows, cols)
    ref = Gref[a, b]
    scale = np.sqrt(np.diag(Gref)[a] * np.diag(Gref)[b])
    assert (np.abs(out - ref) / scale).max() <= TOL
    assert [pos[int(r)] for r in rows[:3]] == list(a[:3])


def test_entries_on_device_and_errors(P):
    import torch
    pb = random_spd(300, 0.02, 9)
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    r = torch.tensor([5, 250, 17, 99, 5], dtype=torch.int32, device="cuda")
    c = torch.tensor([250, 5, 17, 3, 5], dtype=torch.int32, device="cuda")
    out = s.inverse_entries(r, c)
    torch.cuda.synchronize()
    U = np.array([3, 5, 17, 99, 250], np.int32)
    G = f.inv_block(U)
    k = {int(u): t for t, u in enumerate(U)}
    ref = np.array([G[k[int(i)], k[int(j)]] for i, j in zip(r.cpu().numpy(), c.cpu().numpy())])
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL * np.abs(np.diag(G)).max()
    assert s.inverse_entries(np.zeros(0, np.int32), np.zeros(0, np.int32)).shape == (0,)
    with pytest.raises(P.SpiError) as e:
        s.inverse_entries(np.array([0, 300], np.int32), np.array([1, 2], np.int32))
    assert e.value.code == 1
