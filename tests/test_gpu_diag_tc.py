"""The mixed form's variances on the tensor cores (spi_options.diag_tc_min_pivots):
the supernodes with at least that many pivots, and their ancestors, run as
3 x TF32 products of TMA-staged operand tiles -- the blocked forward
substitution z_i = X_ii z_in_i + sum_{j<i} (-X_ii L_ij) z_j over 128-row tiles
of a supernode's own rows, then z_below += (-L21) z_own (paper Sec. 3.3.1) --
and the rest of every path on the SIMT kernel.  Checked element by element
against the FP64 oracle at the mixed form's variance bound, and against the
SIMT-only form of the same factorization."""
import numpy as np
import pytest

import oracle
from spigen import BAND, SCALE, TINY, generate, generate_bands, random_spd, scaled, sky_scaled

pytestmark = pytest.mark.gpu
MIXED_VAR_TOL = 3e-5  # the mixed form's variance bound (first order in its FP32 factor error)
# between the tensor-core and the SIMT variances of one FP32 factor: both are FP32
# forward substitutions of the same panels, differing in rounding only
TC_VS_SIMT_TOL = 2e-5


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def variances(P, pb, min_pivots, **kw):
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32, diag_tc_min_pivots=min_pivots, **kw)
    s.factor(pb.values)
    return s, s.diag_inverse()


CASES = [lambda: generate(TINY), lambda: generate(scaled(SCALE, 1500, seed=9)), lambda: random_spd(300, 0.01, 6),
         lambda: random_spd(700, 0.02, 11), lambda: generate(sky_scaled(1500, 1.2, 40))]


@pytest.mark.parametrize("make", CASES)
@pytest.mark.parametrize("min_pivots", [1, 8, 0])
def test_tensor_core_variances_match_oracle(P, make, min_pivots):
    pb = make()
    v_ref = oracle.OracleFactor.from_problem(pb).inv_diag()
    s, v = variances(P, pb, min_pivots)
    _, v_simt = variances(P, pb, -1)
    info = s.info()
    ev = (np.abs(v - v_ref) / v_ref).max()
    es = (np.abs(v - v_simt) / v_simt).max()
    print(f"n={pb.n} min_pivots={min_pivots} tc_supernodes={info['diag_tc_supernodes']} "
          f"tiles={info['diag_tc_tiles']} flops={info['diag_tc_flops']:.3e} var_err={ev:.2e} vs_simt={es:.2e}")
    if min_pivots == 1:  # every supernode on the tensor cores
        assert info["diag_tc_supernodes"] == info["n_supernodes"] and info["diag_tc_flops"] > 0
    assert ev <= MIXED_VAR_TOL
    assert es <= TC_VS_SIMT_TOL


def test_simt_only_reports_no_tensor_core_work(P):
    pb = generate(scaled(SCALE, 1500, seed=9))
    s, _ = variances(P, pb, -1)
    i = s.info()
    assert i["diag_tc_supernodes"] == 0 and i["diag_tc_flops"] == 0


@pytest.mark.parametrize("rhs_block", [32, 64, 128, 256])
def test_block_sizes_and_index_subsets(P, rhs_block):
    """Blocks of 32..128 right-hand sides take the tensor cores; 256 stays on SIMT.
    A subset of indices (a plan of its own) gives the same values as the full set."""
    pb = generate(scaled(SCALE, 1500, seed=9))
    v_ref = oracle.OracleFactor.from_problem(pb).inv_diag()
    s, v = variances(P, pb, 1, rhs_block=rhs_block)
    assert (np.abs(v - v_ref) / v_ref).max() <= MIXED_VAR_TOL
    assert (s.info()["diag_tc_flops"] > 0) == (rhs_block <= 128)
    sel = np.random.default_rng(rhs_block).permutation(pb.n)[:700].astype(np.int32)
    vs = s.diag_inverse(sel)
    assert (np.abs(vs - v_ref[sel]) / v_ref[sel]).max() <= MIXED_VAR_TOL


def test_repeated_factorizations_repack(P):
    """The operand tiles are rebuilt at every factorization: new values, new variances."""
    pb = generate(scaled(SCALE, 1500, seed=9))
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32, diag_tc_min_pivots=1)
    for scale in (1.0, 3.0, 1.0):
        s.factor(pb.values * scale)
        v = s.diag_inverse()
        v_ref = oracle.OracleFactor.from_problem(pb).inv_diag() / scale
        assert (np.abs(v - v_ref) / v_ref).max() <= MIXED_VAR_TOL


def test_batched_bands(P):
    """Same-pattern bands: one variance launch over all bands (blockIdx.y), each band
    with its own packed operands."""
    bands = generate_bands(scaled(BAND, 400, seed=2), 4)
    s = P.Solver(bands.n, bands.colptr, bands.rowind, batch=bands.nbands, precision=P.SPI_PREC_MIXED_FP32,
                 diag_tc_min_pivots=1)
    s.factor_batch(bands.values)
    v = s.diag_inverse_batch().reshape(bands.nbands, bands.n)
    assert s.info()["diag_tc_flops"] > 0
    for j in range(bands.nbands):
        v_ref = oracle.OracleFactor.from_problem(bands.band(j)).inv_diag()
        assert (np.abs(v[j] - v_ref) / v_ref).max() <= MIXED_VAR_TOL, j


def test_variance_wait_timeout_reported(P):
    """wait_limit < 0: the tensor-core variance kernel's first pipeline wait gives up;
    it drains its own copy and products, frees its tensor memory, and
    spi_diag_inverse returns SPI_ERR_TIMEOUT.  (The factorization here waits
    nowhere: SIMT Schur complements, launches level by level.)"""
    pb = generate(scaled(SCALE, 1500, seed=9))
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32, diag_tc_min_pivots=1, wait_limit=-1,
                             force_schur=1, dag=1)
    s.factor(pb.values)
    with pytest.raises(P.SpiError) as e:
        s.diag_inverse()
    assert e.value.code == 6
    # the device is still usable
    s2, v = variances(P, pb, 1)
    v_ref = oracle.OracleFactor.from_problem(pb).inv_diag()
    assert (np.abs(v - v_ref) / v_ref).max() <= MIXED_VAR_TOL


def test_variances_beside_the_dependency_driven_solve(P):
    """The benchmark's step runs the variances on a second stream while the refined
    solve (one dependency-driven launch whose CTAs wait on each other) runs on the
    first.  Each overlapped step's variances must equal those computed alone on
    the same factor right after (every step refactors, and the mixed factor's
    FP32 atomics make refactorizations differ in their last bits): a Z chunk read
    before the previous tile's epilogue had written it showed up only in this
    setting."""
    import torch
    pb = generate(sky_scaled(3000, 2.0, 60))
    dev = torch.device("cuda:0")
    s = P.Solver.for_problem(pb, precision=P.SPI_PREC_MIXED_FP32, async_=True, dag=2)
    vals = torch.from_numpy(pb.values).to(dev)
    b = torch.from_numpy(pb.b).to(dev)
    idx = torch.from_numpy(pb.sky_columns).to(dev)
    x = torch.empty_like(b)
    var = torch.empty(pb.n_sky, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    st2 = torch.cuda.Stream(dev)
    s.factor(vals, stream=st)
    s.solve(b, x, stream=st)  # the solve's form is chosen here
    s.diag_inverse(idx, out=var, stream=st)
    s.sync(st)
    assert s.info()["solve_dag_tasks"] > 0 and s.info()["diag_tc_supernodes"] > 0
    for _ in range(5):
        s.factor(vals, stream=st)
        done = torch.cuda.Event()
        done.record(st)
        st2.wait_event(done)
        s.diag_inverse(idx, out=var, stream=st2)
        s.solve(b, x, stream=st)
        st.wait_stream(st2)
        ref = s.diag_inverse(idx, stream=st).clone()  # alone, on the same factor
        s.sync(st)
        torch.cuda.synchronize()
        # FP64 sums over the tiles in any order: equal to the last bits
        assert (torch.abs(var - ref) / ref).max().item() <= 1e-12
