"""Seeded synthetic INTEGRAL/SPI-like least-squares problems.

This module is the input generator shared by the tests, the benchmark and the
oracle's callers.  It builds the design matrix H of the SPI sky-plus-background
model and hands out the normal matrix N = H^T W H and right-hand side
b = H^T W y as plain arrays.  It holds none of the arithmetic of the method
under test (no factorization, no triangular solve, no inverse entry).

Model (paper Sec. 2.2.3):
  * rows are (pointing p, detector d) pairs, M = n_p * n_d (Eq. 1, Eq. 4);
  * background, Eq. 2: one normalisation column per pointing and a set of
    detector-pattern columns per block of pointings;
  * each point source J is split into K_J contiguous time-bins (Box I), one
    column per bin, so N = sum_J K_J unknowns;
  * counts are Poisson, sigma_i^2 = y_i (Sec. 2.4.1), W = 1 / max(y, 1);
  * normal equations (H^T Sigma^-2 H) x = H^T Sigma^-2 y (Eq. 7).

Readings where the paper is silent (stated once here, fixed for all configs):
  * pointings cycle a 5x5 dither raster (step 2 deg) about the field centre
    (0, 0); a source is visible from a pointing when their great-circle
    distance is below 15 deg;
  * response R(d, source, dither position) ~ U(0.1, 1), drawn from a
    counter-based SplitMix64 hash so that no table has to be stored;
  * pointing-column entries u_d * g_dp and detector-column entries h_dp with
    g, h ~ U(0.8, 1.2) drawn independently per (d, p): entries u_d * t_dp and
    t_dp for both would make N exactly singular (sum over d of u_d times the
    detector columns equals the sum of the block's pointing columns);
  * time-bin lengths are log-uniform integers in [lo, hi]; the last bin is
    cut at n_p and a remainder shorter than lo is merged into the previous
    bin; bins in which the source is never visible are dropped (a zero column
    would make N singular);
  * detector-pattern blocks hold det_block consecutive pointings; a trailing
    block shorter than half a block is merged into the previous one;
  * true intensities: pointing normalisations U(0.9, 1.1), detector-pattern
    amplitudes U(0, 5), source fluxes U(0, 20) per bin; per-detector
    background means u_d ~ U(50, 200).
  * with `targets` > 0 the pointings visit a targets x targets grid of
    field positions `target_step` apart, each as a 25-pointing block of the
    dither raster, cycling through the grid; a pointing's position is then
    (target, dither offset), and responses are drawn per position;
  * with `sky_pix_deg` > 0 a diffuse sky of square pixels of that size
    covering `sky_field_deg` on a side adds one column per pixel, visible
    from a pointing within fov_deg like a point source, with one bin
    spanning the whole observation; pixels never visible are dropped.
Column order: [pointings; detector-pattern columns (block-major);
time-bins sorted by (start, source); sky pixels (row-major)].
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

N_DET = 19
_DITHER = 5  # 5x5 raster


@dataclasses.dataclass(frozen=True)
class SpiConfig:
    name: str
    n_pointings: int
    n_sources: int
    bin_lo: int
    bin_hi: int
    det_block: int          # pointings per detector-pattern block
    field_deg: float = 40.0  # sources uniform in [-field/2, field/2]^2
    fov_deg: float = 15.0
    dither_step: float = 2.0
    seed: int = 0
    targets: int = 0         # pointing targets per side of the target grid (0 = field centre only)
    target_step: float = 10.0
    sky_pix_deg: float = 0.0  # diffuse-sky pixel size (0 = no sky columns)
    sky_field_deg: float = 70.0


# The workloads: a tiny one the oracle finishes in seconds (P = 300), and the
# P = 20,000 observation (380,000 rows, 500 sources) the benchmark times.
TINY = SpiConfig("spi-tiny-P300", n_pointings=300, n_sources=40, bin_lo=10,
                 bin_hi=300, det_block=100)
SCALE = SpiConfig("spi-P20000", n_pointings=20000, n_sources=500, bin_lo=20,
                  bin_hi=2000, det_block=500)
# Same-pattern energy-band member (one band); bands rescale values only.
BAND = SpiConfig("spi-band-P5000", n_pointings=5000, n_sources=200, bin_lo=10,
                 bin_hi=200, det_block=500)


# Diffuse-sky family (pointing targets on a 7 x 7 grid 10 deg apart, 25-pointing
# dither blocks, point sources plus a pixel grid over 70 deg).  SKY_FULL is
# the large configuration (P = 80,000, 2,000 sources, 0.5 deg pixels); SKY is
# the member of the family the benchmark and the full-size tests run.
SKY_FULL = SpiConfig("spi-sky-P80000", n_pointings=80000, n_sources=2000, bin_lo=20,
                     bin_hi=2000, det_block=500, field_deg=70.0, targets=7,
                     sky_pix_deg=0.5)
SKY = SpiConfig("spi-sky-P8000", n_pointings=8000, n_sources=200, bin_lo=20,
                bin_hi=2000, det_block=500, field_deg=70.0, targets=7,
                sky_pix_deg=1.0)


# The large configuration's diffuse sky at its full size -- 0.5 deg pixels over
# 70 deg, 19,600 sky columns -- with 2,000 pointings and 50 sources, so that the
# FP64 oracle can factor it (its largest front has about 13,500 rows).
SKY_PIX05 = SpiConfig("spi-sky-P2000-pix0.5", n_pointings=2000, n_sources=50, bin_lo=20,
                      bin_hi=2000, det_block=500, field_deg=70.0, targets=7, sky_pix_deg=0.5)


def sky_scaled(n_pointings: int, pix_deg: float, n_sources: int, seed: int = 0) -> SpiConfig:
    """A member of the diffuse-sky family with P pointings and pixels of pix_deg."""
    return dataclasses.replace(SKY, name=f"spi-sky-P{n_pointings}-pix{pix_deg:g}",
                               n_pointings=n_pointings, n_sources=n_sources,
                               bin_lo=max(5, n_pointings // 400), bin_hi=max(10, n_pointings // 4),
                               det_block=max(25, min(500, n_pointings // 8)),
                               sky_pix_deg=pix_deg, seed=seed)


def uneven_config(index: int) -> SpiConfig:
    """Member `index` of the uneven independent batch: P log-uniform in
    [50, 2000], n_s = max(5, round(P/10)), seed = index."""
    rng = np.random.default_rng(1_000_003 + index)
    P = int(round(math.exp(rng.uniform(math.log(50), math.log(2000)))))
    ns = max(5, int(round(P / 10)))
    lo = max(5, P // 40)
    return SpiConfig(f"spi-uneven-{index}", n_pointings=P, n_sources=ns,
                     bin_lo=lo, bin_hi=max(lo + 1, P // 2),
                     det_block=max(25, P // 4), seed=index)


def scaled(cfg: SpiConfig, n_pointings: int, n_sources: int | None = None,
           seed: int | None = None) -> SpiConfig:
    """A smaller member of the same family (for parity tests)."""
    r = n_pointings / cfg.n_pointings
    ns = n_sources if n_sources is not None else max(5, int(round(cfg.n_sources * r)))
    return dataclasses.replace(
        cfg, name=f"{cfg.name}-P{n_pointings}", n_pointings=n_pointings,
        n_sources=ns, bin_lo=max(5, int(round(cfg.bin_lo * r))),
        bin_hi=max(10, int(round(cfg.bin_hi * r))),
        det_block=max(25, int(round(cfg.det_block * r))),
        seed=cfg.seed if seed is None else seed)


# --------------------------------------------------------------------------
# counter-based uniform numbers (SplitMix64 finaliser), vectorised
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix_u01(key: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = key.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _response(seed: int, src: np.ndarray, q: np.ndarray, d: np.ndarray) -> np.ndarray:
    """R(d, source, dither position) ~ U(0.1, 1)."""
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) * np.uint64(0x100000001B3)
               + src.astype(np.uint64) * np.uint64(1 << 20)
               + q.astype(np.uint64) * np.uint64(64) + d.astype(np.uint64))
    return 0.1 + 0.9 * _splitmix_u01(key)


def _angdist_deg(lon1, lat1, lon2, lat2):
    l1, b1, l2, b2 = (np.radians(v) for v in (lon1, lat1, lon2, lat2))
    s = (np.sin((b2 - b1) / 2) ** 2
         + np.cos(b1) * np.cos(b2) * np.sin((l2 - l1) / 2) ** 2)
    return np.degrees(2 * np.arcsin(np.sqrt(np.clip(s, 0.0, 1.0))))


@dataclasses.dataclass
class SpiProblem:
    """One least-squares problem.  N is given as its lower triangle in CSC
    (0-based, rows sorted, diagonal present), the layout the solver takes."""
    cfg: SpiConfig
    n: int
    colptr: np.ndarray   # int64 [n+1]
    rowind: np.ndarray   # int32 [nnz]
    values: np.ndarray   # float64 [nnz]
    b: np.ndarray        # float64 [n]
    x_true: np.ndarray   # float64 [n]
    kind: np.ndarray     # int8 [n]: 0 pointing, 1 detector pattern, 2 time-bin, 3 sky pixel
    n_pointing: int
    n_detcol: int
    n_bins: int
    n_sky: int = 0

    @property
    def sky_columns(self) -> np.ndarray:
        """Indices of the sky-pixel columns (the last n_sky)."""
        return np.arange(self.n - self.n_sky, self.n, dtype=np.int32)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def full_matrix(self) -> sp.csc_matrix:
        """Symmetric N as a scipy matrix (for tests)."""
        low = sp.csc_matrix((self.values, self.rowind, self.colptr), shape=(self.n, self.n))
        return (low + sp.tril(low, -1).T).tocsc()


def _bins_for_sources(rng, cfg: SpiConfig):
    P = cfg.n_pointings
    lo, hi = cfg.bin_lo, cfg.bin_hi
    starts, ends, srcs = [], [], []
    for s in range(cfg.n_sources):
        edges = [0]
        while edges[-1] < P:
            L = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
            edges.append(min(P, edges[-1] + max(1, L)))
        if len(edges) > 2 and edges[-1] - edges[-2] < lo:
            edges.pop(-2)
        for a, b in zip(edges[:-1], edges[1:]):
            starts.append(a); ends.append(b); srcs.append(s)
    return np.array(starts), np.array(ends), np.array(srcs)


def generate(cfg: SpiConfig, *, window: int = 64, noise: bool = True,
             band_scale: np.ndarray | None = None, counts_seed: int | None = None,
             dense_design: bool = False, sparse_design: bool = False) -> SpiProblem:
    """Build the problem for `cfg`.

    noise=False replaces the Poisson draw by y = H x_true exactly (the
    noise-free case whose least-squares solution is x_true).  band_scale, if
    given (one factor per source), rescales every response value of that
    source (energy-band members share one pattern); counts_seed reseeds only
    the Poisson draw.  dense_design=True (small problems only) also returns
    the dense design matrix H and the weights as attributes `H` and `w` of
    the problem, assembled row block by row block, for checking N = H^T W H.
    sparse_design=True returns H as a scipy CSR matrix instead (rows =
    (pointing, detector) in order, columns ascending within a row), with
    the weights w and counts y, for assembling N = H^T W H elsewhere.
    Either also returns the background model's parts: bg_t (g_dp per row),
    bg_pat (the row's detector) and bg_u (u_d), so that the pointing
    column's entry of row p * 19 + d is bg_u[bg_pat] * bg_t.
    """
    rng = np.random.default_rng(cfg.seed)
    P, nd = cfg.n_pointings, N_DET
    half = cfg.field_deg / 2
    src_lon = rng.uniform(-half, half, cfg.n_sources)
    src_lat = rng.uniform(-half, half, cfg.n_sources)
    u_d = rng.uniform(50.0, 200.0, nd)
    g = rng.uniform(0.8, 1.2, (P, nd))
    h = rng.uniform(0.8, 1.2, (P, nd))
    starts, ends, srcs = _bins_for_sources(rng, cfg)
    # pointing positions: the dither raster about the field centre, or about
    # each target of the target grid (position id = target * 25 + dither offset)
    nq = _DITHER * _DITHER
    qpos = np.arange(nq)
    dlon = ((qpos % _DITHER) - _DITHER // 2) * cfg.dither_step
    dlat = ((qpos // _DITHER) - _DITHER // 2) * cfg.dither_step
    if cfg.targets > 0:
        T = cfg.targets
        ti = np.arange(T * T)
        tlon = ((ti % T) - (T - 1) / 2) * cfg.target_step
        tlat = ((ti // T) - (T - 1) / 2) * cfg.target_step
        plon = (tlon[:, None] + dlon[None, :]).ravel()
        plat = (tlat[:, None] + dlat[None, :]).ravel()
        qofp = ((np.arange(P) // nq) % (T * T)) * nq + np.arange(P) % nq
    else:
        plon, plat = dlon, dlat
        qofp = np.arange(P) % nq
    npos = len(plon)
    vis = _angdist_deg(src_lon[:, None], src_lat[:, None], plon[None, :], plat[None, :]) < cfg.fov_deg
    # keep bins with at least one visible pointing
    keep = np.zeros(len(starts), bool)
    for i, (a, b_, s) in enumerate(zip(starts, ends, srcs)):
        qs = np.unique(qofp[a:b_]) if b_ - a < npos else np.arange(npos)
        keep[i] = bool(vis[s, qs].any())
    starts, ends, srcs = starts[keep], ends[keep], srcs[keep]
    order = np.lexsort((srcs, starts))
    starts, ends, srcs = starts[order], ends[order], srcs[order]
    nbins = len(starts)
    # detector-pattern blocks of det_block pointings; a trailing block shorter
    # than half a block joins the previous one (a block of one pointing would
    # make that pointing's column a combination of the block's 19 columns)
    nblk = max(1, P // cfg.det_block + (1 if P % cfg.det_block >= (cfg.det_block + 1) // 2 else 0))

    def blk(p):
        return np.minimum(np.asarray(p) // cfg.det_block, nblk - 1)
    ndet = nblk * nd
    # diffuse-sky pixels seen from at least one pointing made
    if cfg.sky_pix_deg > 0:
        npx = int(round(cfg.sky_field_deg / cfg.sky_pix_deg))
        cgrid = (np.arange(npx) + 0.5) * cfg.sky_pix_deg - cfg.sky_field_deg / 2
        pix_lon, pix_lat = np.tile(cgrid, npx), np.repeat(cgrid, npx)
        pvis = _angdist_deg(pix_lon[:, None], pix_lat[:, None], plon[None, :], plat[None, :]) < cfg.fov_deg
        seen = pvis[:, np.unique(qofp)].any(axis=1)
        pvis = pvis[seen]
    else:
        pvis = np.zeros((0, npos), bool)
    nsky = pvis.shape[0]
    n = P + ndet + nbins + nsky
    col_bin0 = P + ndet
    col_sky0 = col_bin0 + nbins
    x_true = np.concatenate([rng.uniform(0.9, 1.1, P), rng.uniform(0.0, 5.0, ndet),
                             rng.uniform(0.0, 20.0, nbins)])
    if nsky:
        x_true = np.concatenate([x_true, rng.uniform(0.0, 5.0, nsky)])
    kind = np.concatenate([np.zeros(P, np.int8), np.ones(ndet, np.int8), np.full(nbins, 2, np.int8),
                           np.full(nsky, 3, np.int8)])
    scale = np.ones(cfg.n_sources) if band_scale is None else np.asarray(band_scale, float)
    dd = np.arange(nd)

    def sky_response(pix: np.ndarray, pos) -> np.ndarray:
        """R(d, pixel, position) ~ U(0.1, 1); pixels are numbered after the sources."""
        return _response(cfg.seed, cfg.n_sources + np.asarray(pix), np.asarray(pos), dd)

    def window_block(p0: int, p1: int):
        """Dense H restricted to rows of pointings [p0, p1) and the columns
        active there; returns (global column ids, H_w, number of sky columns,
        which come last)."""
        np_ = p1 - p0
        kb0, kb1 = int(blk(p0)), int(blk(p1 - 1)) + 1
        act = np.nonzero((starts < p1) & (ends > p0))[0]
        apix = np.nonzero(pvis[:, np.unique(qofp[p0:p1])].any(axis=1))[0] if nsky else np.zeros(0, np.int64)
        cols = np.concatenate([np.arange(p0, p1),
                               P + np.arange(kb0 * nd, kb1 * nd),
                               col_bin0 + act, col_sky0 + apix])
        Hw = np.zeros((np_ * nd, len(cols)))
        if len(apix):
            c0 = np_ + (kb1 - kb0) * nd + len(act)
            for p in range(p0, p1):
                sel = np.nonzero(pvis[apix, qofp[p]])[0]
                R = sky_response(apix[sel][:, None], qofp[p])
                Hw[(p - p0) * nd + dd[None, :], (c0 + sel)[:, None]] = R
        pp = np.arange(p0, p1)
        rows = (pp - p0)[:, None] * nd + np.arange(nd)[None, :]
        Hw[rows, (pp - p0)[:, None]] = u_d[None, :] * g[p0:p1]
        detc = np_ + (blk(pp) - kb0)[:, None] * nd + np.arange(nd)[None, :]
        Hw[rows, detc] = h[p0:p1]
        if len(act):
            a = np.maximum(starts[act], p0); b_ = np.minimum(ends[act], p1)
            cnt = b_ - a
            bi = np.repeat(np.arange(len(act)), cnt)
            off = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
            p = np.repeat(a, cnt) + off
            s = srcs[act][bi]
            q = qofp[p]
            ok = vis[s, q]
            p, s, q, bi = p[ok], s[ok], q[ok], bi[ok]
            R = _response(cfg.seed, s[:, None], q[:, None], dd[None, :]) * scale[s][:, None]
            r = (p - p0)[:, None] * nd + dd[None, :]
            Hw[r, (np_ + (kb1 - kb0) * nd + bi)[:, None]] = R
        return cols, Hw, len(apix)

    # pass 1: expected counts, Poisson draw (one global draw, window independent)
    e = np.empty(P * nd)
    for p0 in range(0, P, window):
        p1 = min(P, p0 + window)
        cols, Hw, _ = window_block(p0, p1)
        e[p0 * nd:p1 * nd] = Hw @ x_true[cols]
    Hd = None
    if dense_design:
        Hd = np.zeros((P * nd, n))
        for p0 in range(0, P, window):
            p1 = min(P, p0 + window)
            cols, Hw, _ = window_block(p0, p1)
            Hd[p0 * nd:p1 * nd][:, cols] = Hw
    if sparse_design:
        parts = []
        for p0 in range(0, P, window):
            p1 = min(P, p0 + window)
            cols, Hw, _ = window_block(p0, p1)
            o = np.argsort(cols)
            hw = sp.csr_matrix(Hw[:, o])
            hw.indices = cols[o][hw.indices].astype(np.int32)
            parts.append(sp.csr_matrix((hw.data, hw.indices, hw.indptr), shape=(Hw.shape[0], n)))
        Hd = sp.vstack(parts, format="csr")
        Hd.sort_indices()
    if noise:
        crng = rng if counts_seed is None else np.random.default_rng(counts_seed)
        y = crng.poisson(e).astype(np.float64)
        w = 1.0 / np.maximum(y, 1.0)
    else:
        y = e.copy()
        w = 1.0 / np.maximum(np.round(e), 1.0)
    # pass 2: N = H^T W H (lower triangle) and b = H^T W y
    rr, cc, vv = [], [], []
    bvec = np.zeros(n)
    for p0 in range(0, P, window):
        p1 = min(P, p0 + window)
        cols, Hw, ns = window_block(p0, p1)
        ww = w[p0 * nd:p1 * nd]
        if ns == 0:
            G = Hw.T @ (Hw * ww[:, None])
            bvec[cols] += Hw.T @ (ww * y[p0 * nd:p1 * nd])
            gi, gj = np.nonzero(np.tril(np.ones_like(G, dtype=bool)) & (G != 0.0))
        else:
            # rows: the window's non-sky columns; sky x sky is summed per position below
            nw = len(cols) - ns
            G = Hw[:, :nw].T @ (Hw * ww[:, None])
            bvec[cols[:nw]] += Hw[:, :nw].T @ (ww * y[p0 * nd:p1 * nd])
            low = np.ones_like(G, dtype=bool)
            low[:, :nw] = np.tril(low[:, :nw])
            gi, gj = np.nonzero(low & (G != 0.0))
        ri, cj = cols[gi], cols[gj]
        sw = ri < cj
        ri2 = np.where(sw, cj, ri); cj2 = np.where(sw, ri, cj)
        rr.append(ri2); cc.append(cj2); vv.append(G[gi, gj])
    if nsky:
        # sky x sky: pointings at one position see the same pixels with the same
        # responses, so sum their weights per (position, detector) first
        Wt = np.zeros((npos, nd)); Yt = np.zeros((npos, nd))
        np.add.at(Wt, qofp, w.reshape(P, nd))
        np.add.at(Yt, qofp, (w * y).reshape(P, nd))
        # the positions of one target (its 25 dither offsets) see nearly the same
        # pixels: one dense product per target over the union of their pixels
        acc = np.zeros((nsky, nsky))
        groups = ([np.arange(t * nq, (t + 1) * nq) for t in range(npos // nq)] if cfg.targets > 0
                  else [np.arange(npos)])
        for grp in groups:
            qs = [int(q) for q in grp if Wt[q].any() and pvis[:, q].any()]
            if not qs:
                continue
            U = np.nonzero(pvis[:, qs].any(axis=1))[0]
            Rs = np.zeros((len(qs) * nd, len(U)))
            for i, q in enumerate(qs):
                sel = np.nonzero(pvis[U, q])[0]
                R = _response(cfg.seed, cfg.n_sources + U[sel][None, :], np.full((1, 1), q), dd[:, None])  # [nd, |V|]
                Rs[i * nd:(i + 1) * nd, sel] = R
                bvec[col_sky0 + U[sel]] += R.T @ Yt[q]
            acc[np.ix_(U, U)] += Rs.T @ (Rs * Wt[qs].ravel()[:, None])
        # lower triangle, a block of columns at a time
        for j0 in range(0, nsky, 2048):
            j1 = min(nsky, j0 + 2048)
            gi, gj = np.nonzero(acc[j0:, j0:j1])
            low = gi >= gj
            gi, gj = gi[low] + j0, gj[low] + j0
            rr.append(col_sky0 + gi); cc.append(col_sky0 + gj); vv.append(acc[gi, gj])
    rr = np.concatenate(rr); cc = np.concatenate(cc); vv = np.concatenate(vv)
    low = sp.coo_matrix((vv, (rr, cc)), shape=(n, n)).tocsc()
    low.sum_duplicates()
    low.sort_indices()
    pb = SpiProblem(cfg=cfg, n=n, colptr=low.indptr.astype(np.int64),
                    rowind=low.indices.astype(np.int32), values=low.data.astype(np.float64),
                    b=bvec, x_true=x_true, kind=kind, n_pointing=P, n_detcol=ndet, n_bins=nbins,
                    n_sky=nsky)
    if dense_design or sparse_design:
        pb.H, pb.w, pb.y = Hd, w, y
        # the background model's parts (Eq. A4: B_dp = U^d I_p^bg t_dp): the
        # pointing columns (the first P) hold u_d * g_dp in row p * nd + d
        pb.bg_t = g.ravel().copy()                              # t_dp per row
        pb.bg_pat = np.tile(np.arange(nd, dtype=np.int32), P)   # detector per row
        pb.bg_u = u_d.copy()                                    # U^d
    return pb


def random_spd(n: int, density: float, seed: int, *, dominance: float = 1.0) -> SpiProblem:
    """A random sparse SPD matrix (B^T B + shift) of order n, lower CSC, for
    small generic tests; not SPI shaped."""
    rng = np.random.default_rng(seed)
    m = max(n, int(1.5 * n))
    B = sp.random(m, n, density=density, random_state=rng, format="csc")
    B.data = rng.uniform(0.5, 1.5, B.nnz)
    A = (B.T @ B).tocsc() + dominance * sp.identity(n, format="csc")
    low = sp.tril(A).tocsc()
    low.sum_duplicates(); low.sort_indices()
    b = rng.standard_normal(n)
    cfg = SpiConfig(f"random-spd-{n}-{seed}", 0, 0, 1, 1, 1, seed=seed)
    return SpiProblem(cfg=cfg, n=n, colptr=low.indptr.astype(np.int64),
                      rowind=low.indices.astype(np.int32), values=low.data.astype(np.float64),
                      b=b, x_true=np.zeros(n), kind=np.full(n, 2, np.int8),
                      n_pointing=0, n_detcol=0, n_bins=n)


@dataclasses.dataclass
class BandBatch:
    """Same-pattern energy bands: one pattern, `nbands` value sets and
    right-hand sides stacked band after band."""
    cfg: SpiConfig
    n: int
    colptr: np.ndarray
    rowind: np.ndarray
    values: np.ndarray   # float64 [nbands * nnz]
    b: np.ndarray        # float64 [nbands * n]
    energies_kev: np.ndarray
    nbands: int

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def band(self, k: int) -> SpiProblem:
        nnz = self.nnz
        return SpiProblem(cfg=self.cfg, n=self.n, colptr=self.colptr, rowind=self.rowind,
                          values=self.values[k * nnz:(k + 1) * nnz], b=self.b[k * self.n:(k + 1) * self.n],
                          x_true=np.zeros(self.n), kind=np.zeros(self.n, np.int8), n_pointing=0, n_detcol=0,
                          n_bins=0)


def generate_bands(cfg: SpiConfig, nbands: int, *, e_lo: float = 20.0, e_hi: float = 1000.0) -> BandBatch:
    """Energy bands of one observation: band k has energy E_k (log-spaced in
    [e_lo, e_hi] keV); every source's responses are scaled by
    (E_k / e_lo)^-alpha_s with spectral index alpha_s ~ U(1.5, 3) per source,
    and the counts are redrawn per band.  The pattern does not depend on the
    band (every structural entry of N is a sum of positive terms)."""
    rng = np.random.default_rng(10_000 + cfg.seed)
    alpha = rng.uniform(1.5, 3.0, cfg.n_sources)
    energies = np.exp(np.linspace(np.log(e_lo), np.log(e_hi), nbands)) if nbands > 1 else np.array([e_lo])
    vals, bs = [], []
    pattern = None
    for k, e in enumerate(energies):
        pb = generate(cfg, band_scale=(e / e_lo) ** (-alpha), counts_seed=cfg.seed * 100_003 + k)
        if pattern is None:
            pattern = (pb.n, pb.colptr, pb.rowind)
        elif not (pb.n == pattern[0] and np.array_equal(pb.colptr, pattern[1])
                  and np.array_equal(pb.rowind, pattern[2])):
            raise RuntimeError("band pattern differs from band 0")
        vals.append(pb.values)
        bs.append(pb.b)
    return BandBatch(cfg=cfg, n=pattern[0], colptr=pattern[1], rowind=pattern[2],
                     values=np.concatenate(vals), b=np.concatenate(bs), energies_kev=energies, nbands=nbands)


def generate_uneven(count: int, start: int = 0) -> list:
    """`count` independent problems of uneven size (members start..start+count-1)."""
    return [generate(uneven_config(i)) for i in range(start, start + count)]
