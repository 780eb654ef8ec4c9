"""spi_diag_inverse_noalloc: variances for callers that cannot allocate
device memory (a thread that must stay out of the CUDA allocator, or a
process whose device memory belongs to another allocator).  Its output must
match the ordinary spi_diag_inverse on the same factor and the FP64 oracle,
on two calls in a row (the fixed scratch array keeps the previous call's
contents, which the call must clear), and it must accept a mixed-precision
context and band 0 of a batched one, as its header says.  This file is
collected last on purpose."""
import numpy as np
import pytest

import oracle
from spigen import BAND, TINY, generate, generate_bands, random_spd, scaled, SCALE

TOL = 1e-10
# a mixed-precision factor's variances carry its FP32 error to first order (the
# bound used by every mixed-precision test of this suite)
MIXED_VAR_TOL = 3e-5


def _torch_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(P, s, idx, stream=None):
    torch = _torch_or_skip()
    out = torch.full((idx.numel(),), -1.0, dtype=torch.float64, device=idx.device)
    P.spi_diag_inverse_noalloc(s._h, idx, out, stream=stream)
    return out.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_diag_inverse_twice():
    torch = _torch_or_skip()
    import paper_1305_5683_gb300 as P
    P.build.build()
    dev = torch.device("cuda:0")
    for pb in (generate(TINY), generate(scaled(SCALE, 1500, seed=9)), random_spd(200, 0.03, 4)):
        s = P.Solver.for_problem(pb)
        s.factor(pb.values)
        f = oracle.OracleFactor.from_problem(pb)
        rng = np.random.default_rng(pb.n)
        sel = rng.permutation(pb.n)[: min(300, pb.n)].astype(np.int32)
        idx = torch.from_numpy(sel).to(dev)
        ref = s.diag_inverse(idx).cpu().numpy()
        orc = f.inv_diag(sel)
        st = torch.cuda.current_stream(dev)
        for _ in range(2):
            o = _noalloc(P, s, idx, stream=st)
            assert (np.abs(o - ref) / ref).max() <= TOL
            assert (np.abs(o - orc) / orc).max() <= TOL
        # a second, different index set after the first (stale scratch contents)
        idx2 = torch.arange(pb.n - 1, -1, -1, dtype=torch.int32, device=dev)
        full = f.inv_diag()
        o2 = _noalloc(P, s, idx2, stream=st)
        assert (np.abs(o2 - full[::-1]) / full[::-1]).max() <= TOL


@pytest.mark.gpu
def test_noalloc_mixed_context():
    """A mixed-precision context: the call reads the FP64 copy of the factor's
    FP32 panels, so its variances carry the FP32 factor error, like those of
    spi_diag_inverse in that context."""
    torch = _torch_or_skip()
    import paper_1305_5683_gb300 as P
    dev = torch.device("cuda:0")
    pb = generate(scaled(SCALE, 1500, seed=9))
    f = oracle.OracleFactor.from_problem(pb)
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32)
    s.factor(pb.values)
    sel = np.random.default_rng(7).permutation(pb.n)[:400].astype(np.int32)
    idx = torch.from_numpy(sel).to(dev)
    orc = f.inv_diag(sel)
    for _ in range(2):
        o = _noalloc(P, s, idx)
        err = (np.abs(o - orc) / orc).max()
        print(f"noalloc mixed context: var_err={err:.2e}")
        assert err <= MIXED_VAR_TOL


@pytest.mark.gpu
def test_noalloc_band0_of_batch():
    """Band 0 of a same-pattern batch: the variances of band 0's factor."""
    torch = _torch_or_skip()
    import paper_1305_5683_gb300 as P
    dev = torch.device("cuda:0")
    bands = generate_bands(scaled(BAND, 400, seed=2), 3)
    s = P.Solver(bands.n, bands.colptr, bands.rowind, batch=bands.nbands)
    s.factor_batch(bands.values)
    pb0 = bands.band(0)
    orc = oracle.OracleFactor.from_problem(pb0).inv_diag()
    idx = torch.arange(bands.n, dtype=torch.int32, device=dev)
    for _ in range(2):
        o = _noalloc(P, s, idx)
        assert (np.abs(o - orc) / orc).max() <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_bad_index():
    torch = _torch_or_skip()
    import paper_1305_5683_gb300 as P
    pb = random_spd(50, 0.1, 1)
    s = P.Solver.for_problem(pb)
    s.factor(pb.values)
    idx = torch.tensor([3, 50, 7], dtype=torch.int32, device="cuda:0")
    out = torch.empty(3, dtype=torch.float64, device="cuda:0")
    with pytest.raises(P.SpiError) as e:
        P.spi_diag_inverse_noalloc(s._h, idx, out)
    assert e.value.code == 1


def test_noalloc_rejects_oversized_problem_before_device_work():
    """n above the scratch capacity is refused on the host (no GPU needed)."""
    import ctypes
    import paper_1305_5683_gb300 as P
    P.build.build()
    n = 1_398_101
    cp = np.arange(n + 1, dtype=np.int64)
    ri = np.arange(n, dtype=np.int32)
    o = P.spi_default_options()
    o.ordering = P.SPI_ORDER_NATURAL
    h = P.spi_analyse(n, cp, ri, o)
    try:
        rc = P.spi.lib().spi_diag_inverse_noalloc(h, ctypes.c_void_p(16), 1, ctypes.c_void_p(16), None)
        assert rc == P.spi.SPI_ERR_SCRATCH
        assert "scratch" in P.spi_strerror(rc)
    finally:
        P.spi_destroy(h)
