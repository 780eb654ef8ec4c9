"""Pins for the oracle's symmetric indefinite LDL^T with 1x1 and 2x2 pivots
(Bunch-Kaufman partial pivoting) and its inverse diagonal: reconstruction
of the permuted matrix, a library inverse, Sylvester's law of inertia, the
SPD case against the plain LDL^T oracle, and small matrices whose pivot
sequence is fixed by the pivoting rule.  The last test plants mistakes in
copies of the oracle's Python source and checks that the pins catch each."""
import os
import types

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from spigen import random_spd


def _sym(n, seed):
    B = np.random.default_rng(seed).standard_normal((n, n))
    return B + B.T


def pivot_pins(orc):
    fails = []
    # reconstruction and the inverse diagonal on random symmetric indefinite matrices
    for n, seed in ((7, 1), (40, 2), (90, 3)):
        A = _sym(n, seed)
        try:
            p, L, D, blocks = orc.ldlt_pivoted(A)
            if np.abs(A[np.ix_(p, p)] - L @ D @ L.T).max() > 1e-12 * np.abs(A).max():
                fails.append(f"reconstruction n={n}")
            if not np.allclose(np.triu(L, 1), 0.0) or not np.allclose(np.diag(L), 1.0):
                fails.append(f"L unit lower n={n}")
            v = orc.inv_diag_pivoted(A)
            ref = np.diag(np.linalg.inv(A))
            if np.abs(v - ref).max() > 1e-10 * np.abs(ref).max():
                fails.append(f"inverse diagonal n={n}")
            # Sylvester: D has the inertia of A
            ev = np.concatenate([np.linalg.eigvalsh(D[k:k + s, k:k + s]) for k, s in blocks])
            ea = np.linalg.eigvalsh(A)
            if (ev > 0).sum() != (ea > 0).sum() or (ev < 0).sum() != (ea < 0).sum():
                fails.append(f"inertia n={n}")
        except Exception as e:  # a mistake may break the factorization outright
            fails.append(f"n={n}: {type(e).__name__}")
    # zero diagonal: only a 2x2 pivot works
    try:
        p, L, D, blocks = orc.ldlt_pivoted(np.array([[0.0, 1.0], [1.0, 0.0]]))
        if blocks != [(0, 2)] or np.abs(orc.inv_diag_pivoted(np.array([[0.0, 1.0], [1.0, 0.0]]))).max() != 0.0:
            fails.append("2x2 exchange matrix")
    except Exception as e:
        fails.append(f"2x2 exchange matrix: {type(e).__name__}")
    # the rule picks the 2x2 pivot of rows 0 and 2 (rows k and r, r brought to k + 1)
    try:
        A3 = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [1.0, 0.0, 0.0]])
        p, L, D, blocks = orc.ldlt_pivoted(A3)
        if list(p) != [0, 2, 1] or blocks != [(0, 2), (2, 1)]:
            fails.append("3x3 pivot sequence")
    except Exception as e:
        fails.append(f"3x3 pivot sequence: {type(e).__name__}")
    # SPD input: positive 1x1 pivots only, and the plain LDL^T oracle's variances
    pb = random_spd(60, 0.1, 5)
    low = sp.csc_matrix((pb.values, pb.rowind, pb.colptr), shape=(pb.n, pb.n))
    A = (low + sp.tril(low, -1).T).toarray()
    try:
        p, L, D, blocks = orc.ldlt_pivoted(A)
        if any(s != 1 for _, s in blocks) or np.any(np.diag(D) <= 0):
            fails.append("SPD pivots")
        ref = oracle.OracleFactor.from_problem(pb).inv_diag()
        if np.abs(orc.inv_diag_pivoted(A) - ref).max() > 1e-12 * ref.max():
            fails.append("SPD variances")
    except Exception as e:
        fails.append(f"SPD: {type(e).__name__}")
    return fails


def test_pivot_pins_hold_for_the_oracle():
    assert pivot_pins(oracle) == []


PIVOT_MUTATIONS = {
    "2x2 update sign": ("A[k + size:, k + size:] -= C @ Einv @ C.T\n", "A[k + size:, k + size:] += C @ Einv @ C.T\n"),
    "2x2 partner not moved to k + 1": ("                swap(k + 1, r)\n", "                swap(k, r)\n"),
    "alpha test reversed": ("elif abs(A[k, k]) >= BK_ALPHA * lam:\n", "elif abs(A[k, k]) <= BK_ALPHA * lam:\n"),
    "inverse with D, not D^-1": ("s += float(zb @ np.linalg.solve(D[k:k + size, k:k + size], zb))\n",
                                 "s += float(zb @ D[k:k + size, k:k + size] @ zb)\n"),
    "multipliers without E^-1": ("L[k + size:, k:k + size] = C @ Einv\n", "L[k + size:, k:k + size] = C\n"),
}


@pytest.mark.parametrize("name", sorted(PIVOT_MUTATIONS))
def test_pivot_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "__init__.py")).read()
    old, new = PIVOT_MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oracle.__file__
    exec(compile(src.replace(old, new), "oracle_mutant", "exec"), mod.__dict__)
    assert pivot_pins(mod) != [], f"planted mistake '{name}' was not caught"
