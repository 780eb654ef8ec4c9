"""The normal equations on the device (N = H^T W H on the analysed pattern,
b = H^T W y) and their column update, against the oracle's sparse product;
then the factorization of the assembled N against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from spigen import SCALE, TINY, generate, scaled, sky_scaled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def rel(a, ref):
    return np.abs(a - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("cfg", [TINY, scaled(SCALE, 2000, seed=3), sky_scaled(300, 4.0, 20)])
def test_assemble_matches_oracle(P, cfg):
    pb = generate(cfg, sparse_design=True)
    H = pb.H
    s = P.Solver.for_problem(pb).normal_setup(H)
    nv, b = s.normal_assemble(H.data, pb.w, pb.y)
    nref, bref = oracle.normal_equations(H, pb.w, pb.y, pb.colptr, pb.rowind)
    assert rel(nv, nref) <= 1e-13 and rel(b, bref) <= 1e-13
    # every term is positive here, so each entry is accurate on its own scale
    nz = nref != 0
    assert (np.abs(nv[nz] - nref[nz]) / nref[nz]).max() <= 1e-12


def test_assembled_matrix_factors_to_the_oracle(P):
    import torch
    pb = generate(scaled(SCALE, 2000, seed=4), sparse_design=True)
    H = pb.H
    s = P.Solver.for_problem(pb).normal_setup(H)
    dev = torch.device("cuda")
    hv = torch.from_numpy(H.data).to(dev)
    w = torch.from_numpy(pb.w).to(dev)
    y = torch.from_numpy(pb.y).to(dev)
    nv = torch.empty(pb.nnz, dtype=torch.float64, device=dev)
    b = torch.empty(pb.n, dtype=torch.float64, device=dev)
    s.normal_assemble(hv, w, y, nv, b)
    s.factor(nv)
    x = s.solve(b)
    v = s.diag_inverse()
    f = oracle.OracleFactor.from_problem(pb)
    xr, vr = f.solve(pb.b), f.inv_diag()
    assert rel(x.cpu().numpy(), xr) <= 1e-10
    assert (np.abs(v - vr) / vr).max() <= 1e-10


def test_column_update(P):
    pb = generate(scaled(SCALE, 2000, seed=6), sparse_design=True)
    H = pb.H.copy()
    s = P.Solver.for_problem(pb).normal_setup(H)
    nv, b = s.normal_assemble(H.data, pb.w, pb.y)
    rng = np.random.default_rng(2)
    cols = rng.choice(pb.n, 300, replace=False).astype(np.int32)
    H2 = H.copy()
    sel = np.isin(H2.indices, cols)
    H2.data[sel] *= rng.uniform(0.5, 1.5, sel.sum())
    old_nv, old_b = nv.copy(), b.copy()
    s.normal_update(cols, H2.data, pb.w, pb.y, nv, b)
    nref, bref = oracle.normal_equations(H2, pb.w, pb.y, pb.colptr, pb.rowind)
    assert rel(nv, nref) <= 1e-13 and rel(b, bref) <= 1e-13
    # entries in no row or column of the changed unknowns are left as they were
    colj = np.repeat(np.arange(pb.n), np.diff(pb.colptr))
    keep = ~np.isin(colj, cols) & ~np.isin(pb.rowind, cols)
    assert np.array_equal(nv[keep], old_nv[keep])
    assert np.array_equal(b[~np.isin(np.arange(pb.n), cols)], old_b[~np.isin(np.arange(pb.n), cols)])


def test_missing_pattern_entry_is_reported(P):
    pb = generate(TINY, sparse_design=True)
    # drop one off-diagonal entry of N's pattern: its product terms have no place
    low = sp.csc_matrix((pb.values, pb.rowind, pb.colptr), shape=(pb.n, pb.n))
    j = int(np.argmax(np.diff(pb.colptr)))
    k = int(pb.colptr[j]) + 1
    keep = np.ones(pb.nnz, bool)
    keep[k] = False
    rows = pb.rowind[keep]
    cp = np.concatenate([[0], np.cumsum(np.diff(pb.colptr) - np.bincount([j], minlength=pb.n))]).astype(np.int64)
    s = P.Solver(pb.n, cp, rows).normal_setup(pb.H)
    with pytest.raises(P.SpiError) as e:
        s.normal_assemble(pb.H.data, pb.w, pb.y)
    assert e.value.code == 2
    del low
