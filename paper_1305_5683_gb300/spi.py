"""Thin ctypes binding of include/spi.h (argument marshalling only).

Every function here forwards to the compiled CUDA library libspi_gb300.so;
there is no Python or CPU implementation of any numeric step.  If the
library is missing or cannot be loaded, `load()` raises -- there is no
fallback path.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); `on_device` is derived from the argument type.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SPI_OK, SPI_ERR_ARG, SPI_ERR_PATTERN, SPI_ERR_NOT_SPD, SPI_ERR_OOM, SPI_ERR_CUDA, SPI_ERR_TIMEOUT, \
    SPI_ERR_STATE, SPI_ERR_SCRATCH = range(9)
SPI_PREC_FP64, SPI_PREC_MIXED_FP32 = 0, 1
SPI_ORDER_ND, SPI_ORDER_NATURAL = 0, 1

EXPORTS = ["spi_default_options", "spi_analyse", "spi_analyse_multi", "spi_factor", "spi_factor_batch",
           "spi_solve", "spi_solve_batch", "spi_diag_inverse", "spi_diag_inverse_batch", "spi_info", "spi_sync",
           "spi_get_perm", "spi_get_etree", "spi_strerror", "spi_destroy", "spi_diag_inverse_noalloc",
           "spi_inverse_block", "spi_normal_setup", "spi_normal_assemble", "spi_normal_update", "spi_mle_newton",
           "spi_background_fit", "spi_inverse_entries", "spi_diag_inverse_refined", "spi_measure_peak"]
SPI_INVERSE_BLOCK_MAX = 512
SPI_PATTERN_MAX = 2048
SPI_FIT_LSQ, SPI_FIT_MLE = 0, 1


class spi_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("ordering", ctypes.c_int), ("rhs_block", ctypes.c_int),
                ("relax", ctypes.c_int), ("refine_max", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("async_", ctypes.c_int), ("nd_leaf", ctypes.c_int), ("batch", ctypes.c_int),
                ("wait_limit", ctypes.c_int), ("diag_ctas_per_sm", ctypes.c_int), ("diag_unpruned", ctypes.c_int),
                ("autotune", ctypes.c_int), ("force_panel", ctypes.c_int), ("force_schur", ctypes.c_int),
                ("dag", ctypes.c_int), ("tune_cache", ctypes.c_char_p), ("pivoting", ctypes.c_int),
                ("diag_tc_min_pivots", ctypes.c_int)]


class spi_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_a", ctypes.c_int64), ("nnz_l", ctypes.c_int64),
                ("nnz_l_stored", ctypes.c_int64), ("n_supernodes", ctypes.c_int64),
                ("n_levels", ctypes.c_int64), ("max_front", ctypes.c_int64), ("bad_pivot", ctypes.c_int64),
                ("bad_band", ctypes.c_int64),
                ("factor_flops", ctypes.c_double), ("diag_flops", ctypes.c_double),
                ("solve_flops", ctypes.c_double), ("diag_flops_all", ctypes.c_double),
                ("diag_work_flops", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("launches_factor", ctypes.c_int64),
                ("launches_solve", ctypes.c_int64), ("launches_diag", ctypes.c_int64),
                ("refine_steps", ctypes.c_int64), ("solve_relres", ctypes.c_double),
                ("rhs_block", ctypes.c_int64),
                ("analyse_seconds", ctypes.c_double), ("mle_steps", ctypes.c_int64),
                ("mle_cash", ctypes.c_double), ("bg_iters", ctypes.c_int64), ("bg_stat", ctypes.c_double),
                ("launches_factor_fused", ctypes.c_int64), ("launches_factor_tc", ctypes.c_int64),
                ("tiles_factor_tc", ctypes.c_int64), ("tune_source", ctypes.c_int64),
                ("tune_seconds", ctypes.c_double), ("tune_panel_buckets", ctypes.c_int64),
                ("tune_panel_fused", ctypes.c_int64), ("tune_schur_buckets", ctypes.c_int64),
                ("tune_schur_tc", ctypes.c_int64), ("factor_tc_flops", ctypes.c_double),
                ("factor_work_flops", ctypes.c_double), ("factor_dag_tasks", ctypes.c_int64),
                ("factor_dag_levels", ctypes.c_int64), ("tune_ms_launches", ctypes.c_double),
                ("tune_ms_dag", ctypes.c_double), ("solve_dag_tasks", ctypes.c_int64),
                ("tune_solve_ms_launches", ctypes.c_double), ("tune_solve_ms_dag", ctypes.c_double),
                ("pivots_2x2", ctypes.c_int64), ("pivot_delays", ctypes.c_int64), ("pivot_restarts", ctypes.c_int64),
                ("diag_tc_supernodes", ctypes.c_int64), ("diag_tc_tiles", ctypes.c_int64),
                ("diag_tc_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SpiError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {lib().spi_strerror(code).decode()} (status {code})")
        self.code = code


_LIB = None


def load(path: str | None = None, build_if_missing: bool = False) -> ctypes.CDLL:
    """Open libspi_gb300.so and declare the C signatures of include/spi.h."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or _build.OUT
    if not os.path.exists(p):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libspi_gb300.so not built ({p}); run paper_1305_5683_gb300.build.build()")
    L = ctypes.CDLL(p)
    V, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.spi_default_options.argtypes = [ctypes.POINTER(spi_options)]; L.spi_default_options.restype = None
    L.spi_analyse.argtypes = [I64, V, V, ctypes.POINTER(spi_options), ctypes.POINTER(V)]
    L.spi_analyse.restype = I
    L.spi_analyse_multi.argtypes = [ctypes.c_int32, V, V, V, ctypes.POINTER(spi_options), ctypes.POINTER(V)]
    L.spi_analyse_multi.restype = I
    L.spi_factor.argtypes = [V, V, I, V]; L.spi_factor.restype = I
    L.spi_factor_batch.argtypes = [V, ctypes.c_int32, V, I, V]; L.spi_factor_batch.restype = I
    L.spi_solve_batch.argtypes = [V, ctypes.c_int32, V, V, I, V]; L.spi_solve_batch.restype = I
    L.spi_diag_inverse_batch.argtypes = [V, ctypes.c_int32, V, I64, V, I, V]
    L.spi_diag_inverse_batch.restype = I
    L.spi_solve.argtypes = [V, V, V, I, V]; L.spi_solve.restype = I
    L.spi_diag_inverse.argtypes = [V, V, I64, V, I, V]; L.spi_diag_inverse.restype = I
    L.spi_diag_inverse_noalloc.argtypes = [V, V, I64, V, V]; L.spi_diag_inverse_noalloc.restype = I
    L.spi_inverse_block.argtypes = [V, V, I64, V, I, V]; L.spi_inverse_block.restype = I
    L.spi_inverse_entries.argtypes = [V, V, V, I64, V, I, V]; L.spi_inverse_entries.restype = I
    L.spi_diag_inverse_refined.argtypes = [V, V, I64, V, I, V]; L.spi_diag_inverse_refined.restype = I
    L.spi_normal_setup.argtypes = [V, I64, V, V]; L.spi_normal_setup.restype = I
    L.spi_normal_assemble.argtypes = [V, V, V, V, V, V, I, V]; L.spi_normal_assemble.restype = I
    L.spi_normal_update.argtypes = [V, I64, V, V, V, V, V, V, I, V]; L.spi_normal_update.restype = I
    L.spi_mle_newton.argtypes = [V, V, V, V, I, ctypes.c_double, V, I, V]; L.spi_mle_newton.restype = I
    L.spi_background_fit.argtypes = [V, I64, V, V, I, V, V, V, V, V, I, I, ctypes.c_double, V, V, I, V]
    L.spi_background_fit.restype = I
    L.spi_measure_peak.argtypes = [I, I, ctypes.POINTER(ctypes.c_double)]; L.spi_measure_peak.restype = I
    L.spi_info.argtypes = [V, ctypes.POINTER(spi_stats)]; L.spi_info.restype = I
    L.spi_sync.argtypes = [V, V]; L.spi_sync.restype = I
    L.spi_get_perm.argtypes = [V, V]; L.spi_get_perm.restype = I
    L.spi_get_etree.argtypes = [V, V]; L.spi_get_etree.restype = I
    L.spi_strerror.argtypes = [I]; L.spi_strerror.restype = ctypes.c_char_p
    L.spi_destroy.argtypes = [V]; L.spi_destroy.restype = None
    if path is None:
        _LIB = L
    return L


def lib() -> ctypes.CDLL:
    return load()


# ---------------------------------------------------------------- marshalling helpers
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _buf(a, dtype):
    """(pointer, on_device, keepalive) of a numpy array or CUDA tensor."""
    if a is None:
        return None, 0, None
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc: int, where: str):
    if rc != SPI_OK:
        raise SpiError(rc, where)


# ---------------------------------------------------------------- the C entry points
def spi_default_options() -> spi_options:
    o = spi_options()
    lib().spi_default_options(ctypes.byref(o))
    return o


def spi_analyse(n, colptr, rowind, opt: spi_options | None = None) -> ctypes.c_void_p:
    cp, _, k1 = _buf(colptr, np.int64)
    ri, _, k2 = _buf(rowind, np.int32)
    h = ctypes.c_void_p()
    rc = lib().spi_analyse(int(n), cp, ri, ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(rc, "spi_analyse")
    del k1, k2
    return h


def spi_analyse_multi(ns, colptrs, rowinds, opt: spi_options | None = None) -> ctypes.c_void_p:
    """Block-diagonal batch of independent problems (concatenated numbering)."""
    k = len(ns)
    n_arr = np.ascontiguousarray(ns, dtype=np.int64)
    keep = [np.ascontiguousarray(c, dtype=np.int64) for c in colptrs]
    keep2 = [np.ascontiguousarray(r, dtype=np.int32) for r in rowinds]
    cp_ptrs = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in keep])
    ri_ptrs = (ctypes.c_void_p * max(k, 1))(*[a.ctypes.data for a in keep2])
    h = ctypes.c_void_p()
    rc = lib().spi_analyse_multi(k, n_arr.ctypes.data_as(ctypes.c_void_p), ctypes.cast(cp_ptrs, ctypes.c_void_p),
                                 ctypes.cast(ri_ptrs, ctypes.c_void_p),
                                 ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(rc, "spi_analyse_multi")
    del keep, keep2
    return h


def spi_factor_batch(ctx, nbatch, values, stream=None) -> None:
    v, dev, keep = _buf(values, np.float64)
    _check(lib().spi_factor_batch(ctx, int(nbatch), v, dev, _stream(stream)), "spi_factor_batch")
    del keep


def spi_solve_batch(ctx, nbatch, b, x, stream=None) -> None:
    bp, dev, k1 = _buf(b, np.float64)
    xp, dev2, k2 = _buf(x, np.float64)
    if dev != dev2 or (not _is_torch(x) and xp.value != x.ctypes.data):
        raise TypeError("x must be a contiguous float64 buffer on the same side as b")
    _check(lib().spi_solve_batch(ctx, int(nbatch), bp, xp, dev, _stream(stream)), "spi_solve_batch")
    del k1, k2


def spi_diag_inverse_batch(ctx, nbatch, idx, out, stream=None) -> None:
    op, dev, k1 = _buf(out, np.float64)
    if not _is_torch(out) and op.value != out.ctypes.data:
        raise TypeError("out must be a contiguous float64 buffer")
    if idx is None:
        ip, nidx, k2 = None, 0, None
    else:
        ip, dev_i, k2 = _buf(idx, np.int32)
        if dev_i != dev:
            raise TypeError("idx and out must both be host or both be device buffers")
        nidx = int(idx.numel() if _is_torch(idx) else len(k2))
    _check(lib().spi_diag_inverse_batch(ctx, int(nbatch), ip, nidx, op, dev, _stream(stream)),
           "spi_diag_inverse_batch")
    del k1, k2


def spi_factor(ctx, values, stream=None) -> None:
    v, dev, keep = _buf(values, np.float64)
    _check(lib().spi_factor(ctx, v, dev, _stream(stream)), "spi_factor")
    del keep


def spi_solve(ctx, b, x, stream=None) -> None:
    bp, dev, k1 = _buf(b, np.float64)
    if not _is_torch(x) and not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise TypeError("x must be a contiguous float64 numpy array or CUDA tensor")
    xp, dev2, k2 = _buf(x, np.float64)
    if dev != dev2:
        raise TypeError("b and x must both be host or both be device buffers")
    _check(lib().spi_solve(ctx, bp, xp, dev, _stream(stream)), "spi_solve")
    del k1, k2


def spi_diag_inverse(ctx, idx, out, stream=None) -> None:
    """out[t] = (N^-1)[idx[t], idx[t]]; idx None means every index."""
    if not _is_torch(out) and not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise TypeError("out must be a contiguous float64 numpy array or CUDA tensor")
    op, dev, k1 = _buf(out, np.float64)
    if idx is None:
        ip, nidx, k2 = None, 0, None
    else:
        ip, dev_i, k2 = _buf(idx, np.int32)
        if dev_i != dev:
            raise TypeError("idx and out must both be host or both be device buffers")
        nidx = int(idx.numel() if _is_torch(idx) else len(k2))
    _check(lib().spi_diag_inverse(ctx, ip, nidx, op, dev, _stream(stream)), "spi_diag_inverse")
    del k1, k2


def spi_inverse_block(ctx, idx, out, stream=None) -> None:
    """out[s * m + t] = (N^-1)[idx[s], idx[t]] for m = len(idx) <= SPI_INVERSE_BLOCK_MAX."""
    if not _is_torch(out) and not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise TypeError("out must be a contiguous float64 numpy array or CUDA tensor")
    op, dev, k1 = _buf(out, np.float64)
    ip, dev_i, k2 = _buf(idx, np.int32)
    if dev_i != dev:
        raise TypeError("idx and out must both be host or both be device buffers")
    nidx = int(idx.numel() if _is_torch(idx) else len(k2))
    _check(lib().spi_inverse_block(ctx, ip, nidx, op, dev, _stream(stream)), "spi_inverse_block")
    del k1, k2


def spi_diag_inverse_refined(ctx, idx, out, stream=None) -> None:
    """Variances of a mixed-precision factor with the first-order error removed."""
    if not _is_torch(out) and not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise TypeError("out must be a contiguous float64 numpy array or CUDA tensor")
    op, dev, k1 = _buf(out, np.float64)
    ip, dev_i, k2 = _buf(idx, np.int32)
    if dev_i != dev:
        raise TypeError("idx and out must both be host or both be device buffers")
    nidx = int(idx.numel() if _is_torch(idx) else len(k2))
    _check(lib().spi_diag_inverse_refined(ctx, ip, nidx, op, dev, _stream(stream)), "spi_diag_inverse_refined")
    del k1, k2


def spi_inverse_entries(ctx, rows, cols, out, stream=None) -> None:
    """out[t] = (N^-1)[rows[t], cols[t]] for any list of index pairs."""
    if not _is_torch(out) and not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise TypeError("out must be a contiguous float64 numpy array or CUDA tensor")
    op, dev, k1 = _buf(out, np.float64)
    rp, dev_r, k2 = _buf(rows, np.int32)
    cp, dev_c, k3 = _buf(cols, np.int32)
    if not (dev_r == dev_c == dev):
        raise TypeError("rows, cols and out must all be host or all be device buffers")
    nent = int(rows.numel() if _is_torch(rows) else len(k2))
    ncol = int(cols.numel() if _is_torch(cols) else len(k3))
    if ncol != nent:
        raise ValueError("rows and cols must have the same length")
    _check(lib().spi_inverse_entries(ctx, rp, cp, nent, op, dev, _stream(stream)), "spi_inverse_entries")
    del k1, k2, k3


def spi_normal_setup(ctx, rowptr, colind) -> None:
    """Record the pattern of the design matrix H (CSR, host arrays)."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    _check(lib().spi_normal_setup(ctx, len(rp) - 1, rp.ctypes.data_as(ctypes.c_void_p),
                                  ci.ctypes.data_as(ctypes.c_void_p)), "spi_normal_setup")


def _normal_bufs(hvals, w, y, nvals, b):
    bufs = [_buf(a, np.float64) for a in (hvals, w, y, nvals, b)]
    devs = {d for _, d, _ in bufs}
    if len(devs) != 1:
        raise TypeError("hvals, w, y, nvals and b must all be host or all be device buffers")
    for a in (nvals, b):
        if not _is_torch(a) and not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError("nvals and b must be contiguous float64 numpy arrays or CUDA tensors")
    return bufs, devs.pop()


def spi_normal_assemble(ctx, hvals, w, y, nvals, b, stream=None) -> None:
    """nvals = N = H^T W H on the analysed pattern, b = H^T W y."""
    bufs, dev = _normal_bufs(hvals, w, y, nvals, b)
    _check(lib().spi_normal_assemble(ctx, *[p for p, _, _ in bufs], dev, _stream(stream)), "spi_normal_assemble")
    del bufs


def spi_normal_update(ctx, cols, hvals, w, y, nvals, b, stream=None) -> None:
    """Recompute the entries of N and b touched by the columns `cols` of H."""
    cc = np.ascontiguousarray(cols, dtype=np.int32)
    bufs, dev = _normal_bufs(hvals, w, y, nvals, b)
    _check(lib().spi_normal_update(ctx, len(cc), cc.ctypes.data_as(ctypes.c_void_p), *[p for p, _, _ in bufs],
                                   dev, _stream(stream)), "spi_normal_update")
    del bufs


def spi_mle_newton(ctx, hvals, y, x, max_iter=30, tol=1e-12, var=None, stream=None) -> None:
    """Poisson maximum-likelihood fit: x (in: start, out: fit), var = diag(Hess^-1) or None."""
    bufs = [_buf(a, np.float64) for a in (hvals, y, x)]
    devs = {d for _, d, _ in bufs}
    vb = _buf(var, np.float64) if var is not None else (None, None, None)
    if vb[1] is not None:
        devs.add(vb[1])
    if len(devs) != 1:
        raise TypeError("hvals, y, x and var must all be host or all be device buffers")
    for a in (x, var):
        if a is not None and not _is_torch(a) and not (isinstance(a, np.ndarray) and a.dtype == np.float64
                                                       and a.flags.c_contiguous):
            raise TypeError("x and var must be contiguous float64 numpy arrays or CUDA tensors")
    _check(lib().spi_mle_newton(ctx, bufs[0][0], bufs[1][0], bufs[2][0], int(max_iter), float(tol), vb[0],
                                devs.pop(), _stream(stream)), "spi_mle_newton")
    del bufs, vb


def spi_background_fit(ctx, k0, upat, t, hvals, w, y, U, x, mode=SPI_FIT_LSQ, max_iter=20, tol=1e-9,
                       stat=None, var=None, stream=None) -> None:
    """Algorithm 1 (the empty-field pattern): hvals and U in/out, x and var out,
    stat (host float64[max_iter]) receives the statistic of each solve."""
    bufs = [_buf(a, np.float64) for a in (t, hvals, w, y, U, x)]
    pb = _buf(upat, np.int32)
    vb = _buf(var, np.float64) if var is not None else (None, None, None)
    devs = {d for _, d, _ in bufs} | {pb[1]}
    if vb[1] is not None:
        devs.add(vb[1])
    if len(devs) != 1:
        raise TypeError("upat, t, hvals, w, y, U, x and var must all be host or all be device buffers")
    for a in (hvals, U, x, var):
        if a is not None and not _is_torch(a) and not (isinstance(a, np.ndarray) and a.dtype == np.float64
                                                       and a.flags.c_contiguous):
            raise TypeError("hvals, U, x and var must be contiguous float64 numpy arrays or CUDA tensors")
    sp_ = None
    if stat is not None:
        if not (isinstance(stat, np.ndarray) and stat.dtype == np.float64 and stat.flags.c_contiguous
                and stat.size >= max_iter):
            raise TypeError("stat must be a contiguous float64 numpy array of max_iter entries")
        sp_ = stat.ctypes.data_as(ctypes.c_void_p)
    U_len = U.numel() if _is_torch(U) else len(U)
    _check(lib().spi_background_fit(ctx, int(k0), pb[0], bufs[0][0], int(U_len), bufs[1][0], bufs[2][0],
                                    bufs[3][0], bufs[4][0], bufs[5][0], int(mode), int(max_iter), float(tol), sp_,
                                    vb[0], devs.pop(), _stream(stream)), "spi_background_fit")
    del bufs, pb, vb


def spi_diag_inverse_noalloc(ctx, idx, out, stream=None) -> None:
    """Variances for device idx into device out without any device allocation
    by the library (fixed scratch array; see include/spi.h)."""
    if not (_is_torch(idx) and _is_torch(out) and idx.is_cuda and out.is_cuda):
        raise TypeError("idx and out must be CUDA tensors")
    ip, _, k1 = _buf(idx, np.int32)
    op, _, k2 = _buf(out, np.float64)
    _check(lib().spi_diag_inverse_noalloc(ctx, ip, int(idx.numel()), op, _stream(stream)),
           "spi_diag_inverse_noalloc")
    del k1, k2


PEAK_UNITS = {"fp64_fma": 0, "fp64_dmma": 1, "fp32_fma": 2, "tf32_tcgen05": 3, "bf16_tcgen05": 4}


def spi_measure_peak(unit: str, reps: int = 3) -> float:
    """Measured TFLOP/s of one arithmetic unit (see PEAK_UNITS) on the current device."""
    t = ctypes.c_double(0.0)
    _check(lib().spi_measure_peak(PEAK_UNITS[unit], reps, ctypes.byref(t)), f"spi_measure_peak({unit})")
    return t.value


def spi_info(ctx) -> dict:
    st = spi_stats()
    _check(lib().spi_info(ctx, ctypes.byref(st)), "spi_info")
    return st.as_dict()


def spi_sync(ctx, stream=None) -> None:
    _check(lib().spi_sync(ctx, _stream(stream)), "spi_sync")


def spi_get_perm(ctx, n: int) -> np.ndarray:
    p = np.empty(n, np.int32)
    _check(lib().spi_get_perm(ctx, p.ctypes.data_as(ctypes.c_void_p)), "spi_get_perm")
    return p


def spi_get_etree(ctx, n: int) -> np.ndarray:
    p = np.empty(n, np.int32)
    _check(lib().spi_get_etree(ctx, p.ctypes.data_as(ctypes.c_void_p)), "spi_get_etree")
    return p


def spi_strerror(code: int) -> str:
    return lib().spi_strerror(code).decode()


def spi_destroy(ctx) -> None:
    lib().spi_destroy(ctx)


# ---------------------------------------------------------------- convenience wrapper
class Solver:
    """analyse -> factor -> solve -> diag_inverse on one pattern (owns the context)."""

    def __init__(self, n, colptr, rowind, *, precision=SPI_PREC_FP64, ordering=SPI_ORDER_ND,
                 rhs_block=0, relax=1, refine_max=10, refine_tol=1e-13, nd_leaf=0, async_=False, batch=1,
                 wait_limit=0, diag_ctas_per_sm=0, diag_unpruned=False, autotune=0, force_panel=0, force_schur=0,
                 dag=0, tune_cache=None, pivoting=False, diag_tc_min_pivots=0, _multi=None):
        o = spi_default_options()
        o.precision, o.ordering, o.rhs_block, o.relax = precision, ordering, rhs_block, relax
        o.refine_max, o.refine_tol, o.nd_leaf, o.async_ = refine_max, refine_tol, nd_leaf, int(async_)
        o.batch = batch
        o.wait_limit = wait_limit
        o.diag_ctas_per_sm = diag_ctas_per_sm
        o.diag_unpruned = int(diag_unpruned)
        o.autotune, o.force_panel, o.force_schur, o.dag = autotune, force_panel, force_schur, dag
        o.tune_cache = None if tune_cache is None else os.fsencode(tune_cache)
        o.pivoting = int(pivoting)
        o.diag_tc_min_pivots = diag_tc_min_pivots
        self.n = int(n)
        self.batch = batch
        if _multi is not None:
            self._h = spi_analyse_multi(*_multi, o)
        else:
            self._h = spi_analyse(n, colptr, rowind, o)

    @classmethod
    def for_problems(cls, problems, **kw):
        """One context over independent problems (block-diagonal batch)."""
        ns = [p.n for p in problems]
        return cls(sum(ns), None, None, _multi=(ns, [p.colptr for p in problems], [p.rowind for p in problems]),
                   **kw)

    def factor_batch(self, values, nbatch=None, stream=None):
        nb = nbatch if nbatch is not None else self.batch
        spi_factor_batch(self._h, nb, values, stream)
        return self

    def solve_batch(self, b, x=None, nbatch=None, stream=None):
        nb = nbatch if nbatch is not None else self.batch
        if x is None:
            x = b.new_empty(b.shape) if _is_torch(b) else np.empty(nb * self.n, np.float64)
        spi_solve_batch(self._h, nb, b, x, stream)
        return x

    def diag_inverse_batch(self, idx=None, out=None, nbatch=None, stream=None, device=None):
        nb = nbatch if nbatch is not None else self.batch
        m = self.n if idx is None else (idx.numel() if _is_torch(idx) else len(idx))
        if out is None:
            if device is not None:
                import torch
                out = torch.empty(nb * m, dtype=torch.float64, device=device)
            else:
                out = np.empty(nb * m, np.float64)
        spi_diag_inverse_batch(self._h, nb, idx, out, stream)
        return out

    @classmethod
    def for_problem(cls, pb, **kw):
        return cls(pb.n, pb.colptr, pb.rowind, **kw)

    def factor(self, values, stream=None):
        spi_factor(self._h, values, stream)
        return self

    def solve(self, b, x=None, stream=None):
        if x is None:
            x = b.new_empty(b.shape) if _is_torch(b) else np.empty(self.n, np.float64)
        spi_solve(self._h, b, x, stream)
        return x

    def diag_inverse(self, idx=None, out=None, stream=None, device=None):
        m = self.n if idx is None else (idx.numel() if _is_torch(idx) else len(idx))
        if out is None:
            if device is not None or (idx is not None and _is_torch(idx)):
                import torch
                out = torch.empty(m, dtype=torch.float64, device=device or idx.device)
            else:
                out = np.empty(m, np.float64)
        spi_diag_inverse(self._h, idx, out, stream)
        return out

    def inverse_block(self, idx, out=None, stream=None):
        """The dense block (N^-1)[idx, idx] as an (m, m) array (or `out`)."""
        m = idx.numel() if _is_torch(idx) else len(idx)
        if out is None:
            if _is_torch(idx) and idx.is_cuda:
                import torch
                out = torch.empty((m, m), dtype=torch.float64, device=idx.device)
            else:
                out = np.empty((m, m), np.float64)
        spi_inverse_block(self._h, idx, out, stream)
        return out

    def diag_inverse_refined(self, idx, out=None, stream=None):
        """Variances of selected unknowns with the factor's first-order error removed."""
        m = idx.numel() if _is_torch(idx) else len(idx)
        if out is None:
            if _is_torch(idx) and idx.is_cuda:
                import torch
                out = torch.empty(m, dtype=torch.float64, device=idx.device)
            else:
                out = np.empty(m, np.float64)
        spi_diag_inverse_refined(self._h, idx, out, stream)
        return out

    def inverse_entries(self, rows, cols, out=None, stream=None):
        """(N^-1)[rows[t], cols[t]] for every t, as a vector (or into `out`)."""
        m = rows.numel() if _is_torch(rows) else len(rows)
        if out is None:
            if _is_torch(rows) and rows.is_cuda:
                import torch
                out = torch.empty(m, dtype=torch.float64, device=rows.device)
            else:
                out = np.empty(m, np.float64)
        spi_inverse_entries(self._h, rows, cols, out, stream)
        return out

    def normal_setup(self, H):
        """Record the pattern of the design matrix H (scipy sparse, rows = observations)."""
        import scipy.sparse as sp
        Hr = sp.csr_matrix(H)
        Hr.sort_indices()
        spi_normal_setup(self._h, Hr.indptr, Hr.indices)
        self._hnnz = Hr.nnz
        return self

    def normal_assemble(self, hvals, w, y, nvals=None, b=None, stream=None):
        """(N values on the analysed pattern, b) from H's values in CSR order."""
        if nvals is None:
            nvals = np.empty(self.info()["nnz_a"], np.float64)
        if b is None:
            b = np.empty(self.n, np.float64)
        spi_normal_assemble(self._h, hvals, w, y, nvals, b, stream)
        return nvals, b

    def normal_update(self, cols, hvals, w, y, nvals, b, stream=None):
        """Update (nvals, b) in place after H's columns `cols` changed."""
        spi_normal_update(self._h, cols, hvals, w, y, nvals, b, stream)
        return nvals, b

    def mle_newton(self, hvals, y, x0, max_iter=30, tol=1e-12, variances=True, stream=None):
        """Poisson maximum-likelihood fit from x0: (x, diag(Hess^-1) or None)."""
        if _is_torch(x0):
            x = x0.clone()
            var = x0.new_empty(x0.shape) if variances else None
        else:
            x = np.array(x0, dtype=np.float64)
            var = np.empty(self.n, np.float64) if variances else None
        spi_mle_newton(self._h, hvals, y, x, max_iter, tol, var, stream)
        return x, var

    def background_fit(self, k0, upat, t, hvals, w, y, U0, mode="lsq", max_iter=20, tol=1e-9,
                       variances=True, stream=None):
        """Algorithm 1: fit the empty-field pattern U with the solution.  hvals
        (float64 numpy array or CUDA tensor, CSR order of normal_setup) is
        rewritten in place with the returned pattern.  Returns
        (x, U, statistic per solve, diag(Hess^-1) or None)."""
        m = SPI_FIT_LSQ if mode == "lsq" else SPI_FIT_MLE
        if _is_torch(hvals):
            import torch
            U = torch.as_tensor(U0, dtype=torch.float64, device=hvals.device).clone()
            x = torch.empty(self.n, dtype=torch.float64, device=hvals.device)
            var = torch.empty_like(x) if variances else None
        else:
            U = np.array(U0, dtype=np.float64)
            x = np.empty(self.n, np.float64)
            var = np.empty(self.n, np.float64) if variances else None
        stat = np.zeros(max_iter, np.float64)
        spi_background_fit(self._h, k0, upat, t, hvals, w, y, U, x, m, max_iter, tol, stat, var, stream)
        iters = int(self.info()["bg_iters"])
        return x, U, stat[:iters].copy(), var

    def info(self) -> dict:
        return spi_info(self._h)

    def perm(self) -> np.ndarray:
        return spi_get_perm(self._h, self.n)

    def etree(self) -> np.ndarray:
        return spi_get_etree(self._h, self.n)

    def sync(self, stream=None):
        spi_sync(self._h, stream)

    def close(self):
        if getattr(self, "_h", None) is not None:
            spi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
