"""CPU-side checks of the C-ABI library: it loads, exports every symbol the
header declares, and its host analysis (ordering, elimination tree,
postorder, column counts) is right.  No compute call needs a GPU here."""
import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from spigen import SCALE, TINY, generate, random_spd, scaled

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1305_5683_gb300 as P
    P.build.build()
    return P


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "spi.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(spi_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol(P):
    lib = ctypes.CDLL(P.build.OUT)
    syms = header_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(lib, name), name
    assert sorted(P.spi.EXPORTS) == syms


def test_strerror_and_defaults(P):
    o = P.spi_default_options()
    assert o.rhs_block == 0 and o.precision == 0 and o.ordering == 0
    for code in range(8):
        assert P.spi_strerror(code)


def test_pattern_validation(P):
    n = 3
    good_cp = np.array([0, 2, 3, 4], np.int64)
    good_ri = np.array([0, 2, 1, 2], np.int32)
    P.spi_destroy(P.spi_analyse(n, good_cp, good_ri))
    bad = [
        (np.array([0, 2, 3, 4], np.int64), np.array([2, 0, 1, 2], np.int32)),  # no leading diagonal
        (np.array([0, 1, 1, 2], np.int64), np.array([0, 2], np.int32)),        # empty column
        (np.array([0, 3, 4, 5], np.int64), np.array([0, 2, 2, 1, 2], np.int32)),  # duplicate
        (np.array([0, 2, 3, 4], np.int64), np.array([0, 3, 1, 2], np.int32)),  # out of range
    ]
    for cp, ri in bad:
        with pytest.raises(P.SpiError) as e:
            P.spi_analyse(n, cp, ri)
        assert e.value.code == 2
    with pytest.raises(P.SpiError) as e:
        P.spi_analyse(-1, good_cp, good_ri)
    assert e.value.code == 1


def test_empty_matrix(P):
    s = P.Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert s.info()["n"] == 0


def _check_analysis(P, pb, ordering):
    s = P.Solver.for_problem(pb, ordering=ordering)
    n = pb.n
    perm = s.perm()
    assert sorted(perm) == list(range(n))
    parent = s.etree()
    # postorder: parent after child, subtrees contiguous
    assert np.all((parent == -1) | (parent > np.arange(n)))
    size = np.ones(n, np.int64)
    for j in range(n):
        if parent[j] >= 0:
            size[parent[j]] += size[j]
    first = np.arange(n) - size + 1
    for j in range(n):
        if parent[j] >= 0:
            assert first[parent[j]] <= first[j]
    # exact column counts == the oracle's factor of the permuted matrix
    A = pb.full_matrix()
    Ap = A[perm][:, perm]
    low = sp.tril(Ap).tocsc(); low.sort_indices()
    f = oracle.OracleFactor(n, low.indptr.astype(np.int64), low.indices.astype(np.int32), low.data)
    Lp, Li, Lx, D, par = f.factors()
    assert np.array_equal(par, parent)
    info = s.info()
    assert info["nnz_l"] == int(Lp[-1])
    cnt = np.diff(Lp) + 1
    assert info["factor_flops"] == float(np.sum(cnt.astype(float) ** 2 - 1))
    assert info["diag_flops_all"] == pytest.approx(f.inv_diag_flops(), rel=1e-12)
    return info


@pytest.mark.parametrize("ordering", [0, 1])
def test_analysis_matches_oracle_structure(P, ordering):
    _check_analysis(P, generate(TINY), ordering)
    _check_analysis(P, random_spd(150, 0.03, 4), ordering)


def test_nested_dissection_reduces_variance_work(P):
    pb = generate(scaled(SCALE, 4000, seed=2))
    nd = P.Solver.for_problem(pb, ordering=0).info()
    nat = P.Solver.for_problem(pb, ordering=1).info()
    assert nd["diag_flops_all"] < 0.5 * nat["diag_flops_all"]
    assert nd["nnz_l"] < nat["nnz_l"]


def _permuted(pb, seed):
    """The same problem with its columns shuffled (the leaf columns' index
    order then carries no time order, so interval cuts rarely apply)."""
    from spigen import SpiProblem
    q = np.random.default_rng(seed).permutation(pb.n)
    A = pb.full_matrix()[q][:, q]
    low = sp.tril(A).tocsc(); low.sort_indices()
    return SpiProblem(cfg=pb.cfg, n=pb.n, colptr=low.indptr.astype(np.int64), rowind=low.indices.astype(np.int32),
                      values=low.data, b=pb.b[q], x_true=pb.x_true[q], kind=pb.kind[q], n_pointing=pb.n_pointing,
                      n_detcol=pb.n_detcol, n_bins=pb.n_bins)


def test_nested_dissection_on_shuffled_input(P):
    """A valid ordering (exact structure against the oracle) whatever the
    input order; the interval cuts need the leaves in time order, and the
    level-structure separators still beat the natural order without it."""
    pb = _permuted(generate(TINY), 11)
    _check_analysis(P, pb, 0)
    big = generate(scaled(SCALE, 4000, seed=2))
    sh = _permuted(big, 5)
    nd_sh = P.Solver.for_problem(sh, ordering=0).info()
    nd = P.Solver.for_problem(big, ordering=0).info()
    nat = P.Solver.for_problem(big, ordering=1).info()
    assert nd_sh["diag_flops_all"] < nat["diag_flops_all"]
    assert nd["diag_flops_all"] <= nd_sh["diag_flops_all"]


def test_compute_without_gpu_fails_loudly(P):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    pb = random_spd(20, 0.2, 1)
    s = P.Solver.for_problem(pb)
    with pytest.raises(P.SpiError) as e:
        s.factor(pb.values)
    assert e.value.code == 5
    with pytest.raises(P.SpiError) as e:
        s.diag_inverse()
    assert e.value.code == 7
    with pytest.raises(P.SpiError) as e:
        s.inverse_block(np.array([0, 1], np.int32))
    assert e.value.code == 7
    with pytest.raises(P.SpiError) as e:
        s.inverse_entries(np.array([0, 1], np.int32), np.array([1, 1], np.int32))
    assert e.value.code == 7
    with pytest.raises(P.SpiError) as e:
        s.diag_inverse_refined(np.array([0, 1], np.int32))
    assert e.value.code == 7


def test_normal_setup_validates_on_the_host(P):
    """Pattern checks of the design matrix happen before any device work."""
    pb = random_spd(20, 0.2, 1)
    s = P.Solver.for_problem(pb)
    with pytest.raises(P.SpiError) as e:  # columns not ascending within a row
        P.spi_normal_setup(s._h, np.array([0, 2], np.int64), np.array([3, 1], np.int32))
    assert e.value.code == 2
    with pytest.raises(P.SpiError) as e:  # column out of range
        P.spi_normal_setup(s._h, np.array([0, 1], np.int64), np.array([20], np.int32))
    assert e.value.code == 2
    with pytest.raises(P.SpiError) as e:  # assembly before setup
        s.normal_assemble(np.zeros(1), np.zeros(1), np.zeros(1))
    assert e.value.code == 7
    with pytest.raises(P.SpiError) as e:  # the empty-field loop before setup
        s.background_fit(1, np.zeros(1, np.int32), np.ones(1), np.zeros(1), np.ones(1), np.ones(1), np.ones(1))
    assert e.value.code == 7


def test_struct_layouts_match_header(P, tmp_path):
    """The binding's ctypes structures have the C header's sizes and field
    offsets (compiled here with gcc against include/spi.h)."""
    import ctypes as ct
    import subprocess
    fields = {"spi_options": [f for f, _ in P.spi.spi_options._fields_],
              "spi_stats": [f for f, _ in P.spi.spi_stats._fields_]}
    cname = {"async_": "async"}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "spi.h"', "int main(void) {"]
    for st, fl in fields.items():
        src.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fl:
            src.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {cname.get(f, f)}));')
    src.append("  return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, cls in (("spi_options", P.spi.spi_options), ("spi_stats", P.spi.spi_stats)):
        assert int(got[st]) == ct.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


@pytest.mark.parametrize("field,value", [("rhs_block", -1), ("rhs_block", 513), ("precision", 2),
                                         ("ordering", 2), ("relax", -1), ("refine_max", -1),
                                         ("nd_leaf", -1), ("diag_ctas_per_sm", -1), ("diag_unpruned", 2),
                                         ("autotune", -2), ("autotune", 2), ("force_panel", 3),
                                         ("force_schur", -1), ("dag", 3), ("pivoting", 2)])
def test_options_are_validated(P, field, value):
    """spi_analyse rejects out-of-range options before any work."""
    pb = random_spd(20, 0.2, 1)
    with pytest.raises(P.SpiError) as e:
        P.Solver.for_problem(pb, **{field: value})
    assert e.value.code == 1
