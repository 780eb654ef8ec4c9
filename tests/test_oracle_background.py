"""Pins for the oracle's Algorithm 1 (the appendix on the "empty-field"
pattern: solve, re-estimate the pattern U, update H, repeat).  Each check ties
the oracle to something other than itself: a dense least-squares routine per
pattern value, a numerical one-dimensional maximiser of the Poisson
likelihood, the noise-free problem whose fixed point is the generator's own
(U, x), and convergence to the true pattern (up to the model's scale) on a
problem without the detector-pattern columns.  The last test plants mistakes
in copies of the oracle's Python source and checks that the pins catch each."""
import os
import types

import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from spigen import TINY, generate

ND = 19


def _perturbed(u, seed=1):
    rng = np.random.default_rng(seed)
    return u * (1 + 0.2 * rng.uniform(-1, 1, len(u)))


def _lsq(Hc, y, w):
    N = (Hc.T @ sp.diags(w) @ Hc).tocsc()
    return spla.spsolve(N, Hc.T @ (w * y))


def background_pins(orc):
    """Returns the list of failed pins for an oracle module `orc`."""
    fails = []
    pb = generate(TINY, sparse_design=True)
    P = pb.n_pointing
    M = pb.H.shape[0]
    pat, t = pb.bg_pat, pb.bg_t
    cpt = np.arange(M) // ND  # the pointing column of each row
    U0 = _perturbed(pb.bg_u)

    # set_background: the pointing entries become U[d] t_dp, the rest is H's
    Hc = orc.set_background(pb.H, P, pat, t, U0)
    Hd, H0 = Hc.toarray(), pb.H.toarray()
    if not np.allclose(Hd[np.arange(M), cpt], U0[pat] * t, rtol=1e-15, atol=0):
        fails.append("set_background: background entries")
    Hd2, H02 = Hd.copy(), H0.copy()
    Hd2[np.arange(M), cpt] = 0.0
    H02[np.arange(M), cpt] = 0.0
    if not np.array_equal(Hd2, H02):
        fails.append("set_background: other entries")

    # least-squares pattern step: U_k minimises sum_{rows of k} w (y - y^S - U a)^2,
    # a one-parameter weighted least-squares problem per detector (dense lstsq)
    x = _lsq(Hc, pb.y, pb.w)
    U1 = orc.background_pattern(Hc, x, pb.y, pb.w, P, pat, t, U0, "lsq")
    yS = Hd2 @ x
    a = t * x[cpt]
    for k in range(ND):
        r = pat == k
        sw = np.sqrt(pb.w[r])
        ref = np.linalg.lstsq((sw * a[r])[:, None], sw * (pb.y[r] - yS[r]), rcond=None)[0][0]
        if abs(U1[k] - ref) > 1e-10 * abs(ref):
            fails.append(f"lsq pattern step, detector {k}")
            break

    # likelihood pattern step with y^S = 0 (only the pointing columns in x): the
    # paper's formula is the exact maximiser of the detector's Poisson likelihood
    x0 = np.zeros(pb.n)
    x0[:P] = pb.x_true[:P]
    Um = orc.background_pattern(Hc, x0, pb.y, pb.w, P, pat, t, U0, "mle")
    a0 = t * x0[cpt]
    for k in range(ND):
        r = pat == k

        def negl(u, r=r):
            e = u * a0[r]
            return float(np.sum(e - pb.y[r] * np.log(e)))
        ref = so.minimize_scalar(negl, bounds=(1.0, 1000.0), method="bounded",
                                 options={"xatol": 1e-10}).x
        if abs(Um[k] - ref) > 1e-6 * abs(ref):
            fails.append(f"mle pattern step, detector {k}")
            break
    # and with sources present it matches the detector's total counts
    Um = orc.background_pattern(Hc, x, pb.y, pb.w, P, pat, t, U0, "mle")
    e = Hd2 @ x + Um[pat] * a
    tot_e = np.bincount(pat, weights=e, minlength=ND)
    tot_y = np.bincount(pat, weights=pb.y, minlength=ND)
    if np.abs(tot_e - tot_y).max() > 1e-9 * tot_y.max():
        fails.append("mle pattern step: counts per detector")

    # the loop: max_iter = 1 keeps U0 and returns the least-squares solution
    xf, Uf, st, var = orc.background_fit(pb.H, pb.y, pb.w, P, pat, t, U0, max_iter=1)
    if len(st) != 1 or not np.array_equal(Uf, U0) or np.abs(xf - x).max() > 1e-9 * np.abs(x).max():
        fails.append("max_iter = 1")
    Nd = (Hc.T @ sp.diags(pb.w) @ Hc).toarray()
    if var is None or np.any(var <= 0) or np.any(var * np.diag(Nd) < 1 - 1e-12):
        fails.append("variances: positive and at least 1 / N_ii")
    # a tolerance of 1 stops after the second solve and returns its (U, x)
    xf, Uf, st, _ = orc.background_fit(pb.H, pb.y, pb.w, P, pat, t, U0, tol=1.0, variances=False)
    x2 = _lsq(orc.set_background(pb.H, P, pat, t, U1), pb.y, pb.w)
    if len(st) != 2 or np.abs(Uf - U1).max() > 1e-12 * U1.max() or np.abs(xf - x2).max() > 1e-9 * np.abs(x2).max():
        fails.append("stop rule with tol = 1")

    # noise-free counts and the true pattern: a fixed point at the generator's (U, x)
    pf = generate(TINY, sparse_design=True, noise=False)
    for mode in ("lsq", "mle"):
        xf, Uf, st, _ = orc.background_fit(pf.H, pf.y, pf.w, P, pf.bg_pat, pf.bg_t, pf.bg_u, mode=mode,
                                           max_iter=3, variances=False)
        if (np.abs(xf - pf.x_true).max() > 1e-8 * np.abs(pf.x_true).max()
                or np.abs(Uf - pf.bg_u).max() > 1e-8 * pf.bg_u.max()):
            fails.append(f"noise-free fixed point ({mode})")

    # without the detector-pattern columns the least-squares loop walks to the
    # true pattern (up to the scale shared by U and the pointing normalisations):
    # chi^2 falls at every solve, by 1e3 in 12 solves, and U / U_true flattens
    keep = np.r_[0:P, P + pf.n_detcol:pf.n]
    Hr = sp.csr_matrix(pf.H)[:, keep]
    yr = Hr @ pf.x_true[keep]
    wr = 1.0 / np.maximum(np.round(yr), 1.0)
    _, Uf, st, _ = orc.background_fit(Hr, yr, wr, P, pf.bg_pat, pf.bg_t, _perturbed(pf.bg_u), max_iter=12,
                                      tol=0.0, variances=False)
    ratio = Uf / pf.bg_u
    if not (len(st) == 12 and np.all(np.diff(st) < 0) and st[-1] < 1e-3 * st[0]
            and (ratio.max() - ratio.min()) < 0.05 * ratio.mean()):
        fails.append("convergence to the true pattern")
    return fails


def test_background_pins_hold_for_the_oracle():
    assert background_pins(oracle) == []


BG_MUTATIONS = {
    "lsq step drops w in the numerator": ("num[k] += r[i] * a[i] * w[i]\n", "num[k] += r[i] * a[i]\n"),
    "a_i without the pointing's x": ("a[i] = t[i] * x[j]\n", "a[i] = t[i]\n"),
    "mle step ignores y^S": ("num[k] += r[i]\n", "num[k] += y[i]\n"),
    "set_background drops t": ("Hs.data[bg[0]] = U[upat[i]] * t[i]\n", "Hs.data[bg[0]] = U[upat[i]]\n"),
    "no pattern update": ("U = background_pattern(Hc, x, yy, ww, k0, upat, t, U, mode)\n", "pass\n"),
}


@pytest.mark.parametrize("name", sorted(BG_MUTATIONS))
def test_background_pins_catch_planted_mistake(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "__init__.py")).read()
    old, new = BG_MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oracle.__file__
    exec(compile(src.replace(old, new), "oracle_mutant", "exec"), mod.__dict__)
    assert background_pins(mod) != [], f"planted mistake '{name}' was not caught"
