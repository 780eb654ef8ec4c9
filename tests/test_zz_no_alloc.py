"""spi_diag_inverse_noalloc: variances for callers that cannot allocate
device memory (a thread that must stay out of the CUDA allocator, or a
process whose device memory belongs to another allocator).  Its output must
match the ordinary spi_diag_inverse on the same factor, on two calls in a row
(the fixed scratch array keeps the previous call's contents, which the call
must clear).  This file is collected last on purpose."""
import numpy as np
import pytest

from spigen import TINY, generate, random_spd, scaled, SCALE

TOL = 1e-10


@pytest.mark.gpu
def test_noalloc_matches_diag_inverse_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    dev = torch.device("cuda:0")
    for pb in (generate(TINY), generate(scaled(SCALE, 1500, seed=9)), random_spd(200, 0.03, 4)):
        s = P.Solver.for_problem(pb)
        s.factor(pb.values)
        rng = np.random.default_rng(pb.n)
        idx = torch.from_numpy(rng.permutation(pb.n)[: min(300, pb.n)].astype(np.int32)).to(dev)
        ref = s.diag_inverse(idx).cpu().numpy()
        st = torch.cuda.current_stream(dev)
        outs = []
        for _ in range(2):
            out = torch.full((idx.numel(),), -1.0, dtype=torch.float64, device=dev)
            P.spi_diag_inverse_noalloc(s._h, idx, out, stream=st)
            outs.append(out.cpu().numpy())
        for o in outs:
            assert (np.abs(o - ref) / ref).max() <= TOL
        # a second, different index set after the first (stale scratch contents)
        idx2 = torch.arange(pb.n - 1, -1, -1, dtype=torch.int32, device=dev)
        out2 = torch.empty(pb.n, dtype=torch.float64, device=dev)
        P.spi_diag_inverse_noalloc(s._h, idx2, out2, stream=st)
        full = s.diag_inverse()
        assert (np.abs(out2.cpu().numpy() - full[::-1]) / full[::-1]).max() <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_bad_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
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
