"""GB300-native Asp-Clean2016 minor cycle (Zhang, Bhatnagar, Rau & Zhang 2016).

Thin Python binding of ``libasp.so`` (C-ABI in ``include/asp.h``).  The
functions carry the C names (``asp_init``, ``asp_find_peak``,
``asp_fit_active_set``, ``asp_subtract``, ``asp_minor_cycle``, ...) and only
marshal arguments; PyTorch provides device memory and streams.  There is no
CPU path: without the built library, importing the binding's calls raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    ASP_INIT_AUTO, ASP_INIT_SIMPLE, ASP_INIT_SMOOTH, ASP_KMAX, ASP_LM_CAP, ASP_LM_CONVERGED, ASP_LM_STALLED,
    ASP_PEAK_SIMPLE, ASP_PEAK_SMOOTH, ASP_SUB_AUTO, ASP_SUB_DIRECT, ASP_SUB_FFT, ASP_SUB_FFT_MIN_PIXELS,
    ASP_STOP_CAPACITY, ASP_STOP_ITER, ASP_STOP_NOISE, ASP_STOP_NONE,
    asp_component, asp_cycle_stats, asp_fit_info, asp_gauss, asp_iter_record, asp_params, asp_peak,
    asp_gauss_ell, asp_component_ell, ASP_ELL_KMAX,
)

__all__ = [
    "AspError", "lib", "default_params", "asp_init", "asp_init_host", "asp_destroy", "asp_get_beam",
    "asp_find_peak", "asp_fit_active_set", "asp_fit_lm", "asp_fit_2004", "asp_fit_elliptical",
    "asp_fit_beam_elliptical", "asp_deconvolve_elliptical", "asp_batch_fit_joint", "asp_measure_alu_peaks", "asp_subtract_beam", "asp_eval_normal_equations", "asp_subtract", "asp_minor_cycle",
    "asp_smooth", "asp_num_scales", "asp_copy_residual", "asp_set_residual", "asp_get_components",
    "asp_get_history", "asp_get_stats", "asp_get_state", "asp_set_state", "asp_save_state", "asp_load_state",
    "asp_get_last_fit", "asp_batch_create", "asp_batch_destroy", "asp_batch_reset", "asp_batch_minor_cycle",
    "asp_batch_autotune", "asp_batch_run_queue", "asp_batch_image", "asp_batch_launch_count",
    "Context", "Batch", "MLP", "mlp_pack", "mlp_unpack",
]

_LIB: Optional[C.CDLL] = None


def lib() -> C.CDLL:
    """The loaded libasp.so (raises ImportError if it is not built)."""
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


class AspError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        name = _lib.STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {name}" + (f" ({message})" if message else ""))


def _check(status: int, where: str, handle=None):
    if status != 0:
        msg = ""
        if handle:
            raw = lib().asp_last_error(handle)
            msg = raw.decode() if raw else ""
        raise AspError(status, where, msg)


def default_params(**overrides) -> asp_params:
    """asp_params with the library defaults, then ``overrides`` applied."""
    p = asp_params()
    lib().asp_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _cuda_f32(t, shape, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


def _host_f32(a, shape, name):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.shape != tuple(shape):
        raise ValueError(f"{name} has shape {a.shape}, expected {tuple(shape)}")
    return a


# ----------------------------------------------------------------- C-named calls

def asp_init(params: asp_params, dirty, psf, stream=None):
    """asp_init: dirty (H x W) and psf (2H x 2W) as float32 CUDA tensors."""
    H, W = int(dirty.shape[0]), int(dirty.shape[1])
    dp = _cuda_f32(dirty, (H, W), "dirty")
    pp = _cuda_f32(psf, (2 * H, 2 * W), "psf")
    h = C.c_void_p()
    _check(lib().asp_init(C.byref(params), H, W, dp, pp, _stream_handle(stream), C.byref(h)), "asp_init")
    return h


def asp_init_host(params: asp_params, dirty, psf, stream=None):
    """asp_init_host: dirty and psf as host arrays (copied inside the call)."""
    d = _host_f32(dirty, np.shape(dirty), "dirty")
    H, W = d.shape
    p = _host_f32(psf, (2 * H, 2 * W), "psf")
    h = C.c_void_p()
    _check(lib().asp_init_host(C.byref(params), H, W, d.ctypes.data, p.ctypes.data, _stream_handle(stream),
                               C.byref(h)), "asp_init_host")
    return h


def asp_destroy(h):
    _check(lib().asp_destroy(h), "asp_destroy")


def asp_get_beam(h):
    v = [C.c_double() for _ in range(4)]
    _check(lib().asp_get_beam(h, *[C.byref(x) for x in v]), "asp_get_beam", h)
    return tuple(x.value for x in v)


def asp_find_peak(h, mode: int = ASP_PEAK_SIMPLE) -> dict:
    out = asp_peak()
    _check(lib().asp_find_peak(h, int(mode), C.byref(out)), "asp_find_peak", h)
    return {f: getattr(out, f) for f, _ in asp_peak._fields_}


def _gauss_array(rows):
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 4)
    arr = (asp_gauss * len(rows))()
    for i, (a, x, y, w) in enumerate(rows):
        arr[i] = asp_gauss(a, x, y, w)
    return arr, len(rows)


def asp_fit_active_set(h, init, n_old: int = 0):
    """Joint LM fit; ``init`` rows (a, x, y, w).  Returns (fitted rows, info)."""
    arr, n = _gauss_array(init)
    out = (asp_gauss * n)()
    info = asp_fit_info()
    _check(lib().asp_fit_active_set(h, arr, n, int(n_old), out, C.byref(info)), "asp_fit_active_set", h)
    res = np.array([[g.amp, g.x, g.y, g.width] for g in out])
    return res, {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_}


def asp_fit_lm(h, init, n_old: int, lambda0: float, max_iter: int, start=None):
    """The fit defined by ``init`` / ``n_old``, LM started at ``start``
    (default ``init``) with damping ``lambda0``, at most ``max_iter`` damped
    solves.  Returns (kept rows, info dict, last trial rows, chi^2 of the
    last pass)."""
    arr, n = _gauss_array(init)
    sarr = None
    if start is not None:
        sarr, ns = _gauss_array(start)
        if ns != n:
            raise ValueError("start must have as many rows as init")
    out = (asp_gauss * n)()
    trial = (asp_gauss * n)()
    info = asp_fit_info()
    c2 = C.c_double()
    _check(lib().asp_fit_lm(h, arr, n, int(n_old), sarr, float(lambda0), int(max_iter), out, C.byref(info), trial,
                            C.byref(c2)), "asp_fit_lm", h)
    rows = lambda a: np.array([[g.amp, g.x, g.y, g.width] for g in a])   # noqa: E731
    return rows(out), {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_}, rows(trial), c2.value


def asp_measure_alu_peaks() -> dict:
    """Measured FP32 FMA and MUFU ex2 issue rates of the current device."""
    out = _lib.asp_alu_peaks()
    _check(lib().asp_measure_alu_peaks(C.byref(out)), "asp_measure_alu_peaks")
    return {f: getattr(out, f) for f, _ in _lib.asp_alu_peaks._fields_ if f != "reserved"}


def asp_fit_2004(h, init, n_old: int = 0, omega_min: float = 0.1):
    """LM on Asp-Clean2004's Eq. 3 objective (unconvolved components through
    the full PSF by FFT).  Returns (fitted rows, info dict)."""
    arr, n = _gauss_array(init)
    out = (asp_gauss * n)()
    info = asp_fit_info()
    _check(lib().asp_fit_2004(h, arr, n, int(n_old), float(omega_min), out, C.byref(info)), "asp_fit_2004", h)
    return (np.array([[g.amp, g.x, g.y, g.width] for g in out]),
            {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_})


def _ell_array(rows):
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 6)
    arr = (asp_gauss_ell * len(rows))()
    for i, r in enumerate(rows):
        arr[i] = asp_gauss_ell(*[float(v) for v in r])
    return arr, len(rows)


def _ell_rows(arr):
    return np.array([[g.amp, g.x, g.y, g.pxx, g.pxy, g.pyy] for g in arr])


def asp_fit_elliptical(h, init, n_old: int = 0):
    """Eq. 6 with elliptical members: rows (amp, x, y, A, B, C), the
    precision matrix [[A, B], [B, C]].  Returns (fitted rows, info dict)."""
    arr, n = _ell_array(init)
    out = (asp_gauss_ell * n)()
    info = asp_fit_info()
    _check(lib().asp_fit_elliptical(h, arr, n, int(n_old), out, C.byref(info)), "asp_fit_elliptical", h)
    return _ell_rows(out), {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_}


def asp_fit_beam_elliptical(h):
    """The elliptical beam (alpha_b, x_b, y_b, A_b, B_b, C_b) on the PSF grid."""
    out = asp_gauss_ell()
    _check(lib().asp_fit_beam_elliptical(h, C.byref(out)), "asp_fit_beam_elliptical", h)
    return _ell_rows([out])[0]


def asp_deconvolve_elliptical(h, rows, beam):
    """Eqs. 7-8 for ellipses on the device: rows (flux, amp, x, y, sxx, sxy,
    syy, is_point)."""
    arr, n = _ell_array(rows)
    b, _ = _ell_array(beam)
    out = (asp_component_ell * max(n, 1))()
    _check(lib().asp_deconvolve_elliptical(h, arr, n, b, out), "asp_deconvolve_elliptical", h)
    return np.array([[c.flux, c.amp, c.x, c.y, c.sxx, c.sxy, c.syy, c.is_point] for c in out[:n]])


def asp_batch_fit_joint(h, init, n_old: int, n_chan: int):
    rows = np.ascontiguousarray(np.asarray(init, dtype=np.float64).reshape(-1, 3 + n_chan))
    n = rows.shape[0]
    out = np.empty_like(rows)
    flux = np.empty((n, n_chan))
    pt = np.empty(n, dtype=np.int32)
    info = asp_fit_info()
    _check(lib().asp_batch_fit_joint(h, rows.ctypes.data, n, int(n_old), out.ctypes.data, flux.ctypes.data,
                                     pt.ctypes.data, C.byref(info)), "asp_batch_fit_joint")
    return out, flux, pt.astype(bool), {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_}


def asp_eval_normal_equations(h, theta, n_old: int, window):
    arr, n = _gauss_array(theta)
    P = 4 * n
    A = np.zeros((P, P))
    g = np.zeros(P)
    chi2 = np.zeros(1)
    x0, x1, y0, y1 = (int(v) for v in window)
    _check(lib().asp_eval_normal_equations(h, arr, n, int(n_old), x0, x1, y0, y1, A.ctypes.data, g.ctypes.data,
                                           chi2.ctypes.data), "asp_eval_normal_equations", h)
    return A, g, float(chi2[0])


def _component_array(rows):
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 6)
    arr = (asp_component * len(rows))()
    for i, (F, a, x, y, w, pt) in enumerate(rows):
        arr[i] = asp_component(F, a, x, y, w, int(pt), 0)
    return arr, len(rows)


def asp_subtract(h, comps, gain: float = 1.0):
    """R -= B * (gain * sum of components); rows (flux, amp, x, y, width, is_point)."""
    arr, n = _component_array(comps)
    _check(lib().asp_subtract(h, arr, n, float(gain)), "asp_subtract", h)


def asp_subtract_beam(h, comps, gain: float = 1.0):
    """R -= gain * sum of the components' single-Gaussian-beam images."""
    arr, n = _component_array(comps)
    _check(lib().asp_subtract_beam(h, arr, n, float(gain)), "asp_subtract_beam", h)


def _stats_dict(s: asp_cycle_stats) -> dict:
    return {f: getattr(s, f) for f, _ in asp_cycle_stats._fields_ if f != "reserved"}


def asp_minor_cycle(h, n_iter: int) -> dict:
    s = asp_cycle_stats()
    _check(lib().asp_minor_cycle(h, int(n_iter), C.byref(s)), "asp_minor_cycle", h)
    return _stats_dict(s)


def asp_get_stats(h) -> dict:
    s = asp_cycle_stats()
    _check(lib().asp_get_stats(h, C.byref(s)), "asp_get_stats", h)
    return _stats_dict(s)


def asp_num_scales(h):
    n = C.c_int()
    _check(lib().asp_num_scales(h, C.byref(n), None), "asp_num_scales", h)
    sc = np.zeros(max(n.value, 1))
    _check(lib().asp_num_scales(h, C.byref(n), sc.ctypes.data), "asp_num_scales", h)
    return sc[: n.value]


def asp_smooth(h, scale_index: int, out):
    """Smoothed residual of one scale into ``out`` (float32 CUDA tensor H x W)."""
    _check(lib().asp_smooth(h, int(scale_index), out.data_ptr()), "asp_smooth", h)
    return out


def asp_copy_residual(h, out):
    """Residual into ``out``: a float32 CUDA tensor or a numpy float32 array."""
    if isinstance(out, np.ndarray):
        assert out.dtype == np.float32 and out.flags.c_contiguous
        _check(lib().asp_copy_residual(h, out.ctypes.data, 1), "asp_copy_residual", h)
    else:
        _check(lib().asp_copy_residual(h, out.data_ptr(), 0), "asp_copy_residual", h)
    return out


def asp_set_residual(h, src):
    if isinstance(src, np.ndarray):
        a = np.ascontiguousarray(src, dtype=np.float32)
        _check(lib().asp_set_residual(h, a.ctypes.data, 1), "asp_set_residual", h)
    else:
        _check(lib().asp_set_residual(h, src.data_ptr(), 0), "asp_set_residual", h)


def _comp_rows(arr, n):
    return np.array([[c.flux, c.amp, c.x, c.y, c.width, c.is_point] for c in arr[:n]]).reshape(-1, 6)


def asp_get_components(h) -> np.ndarray:
    """Component list as rows (flux, amp, x, y, width, is_point)."""
    n = C.c_int()
    _check(lib().asp_get_components(h, None, 0, C.byref(n)), "asp_get_components", h)
    arr = (asp_component * max(n.value, 1))()
    _check(lib().asp_get_components(h, arr, n.value, C.byref(n)), "asp_get_components", h)
    return _comp_rows(arr, n.value)


def asp_get_history(h) -> list:
    n = C.c_int()
    _check(lib().asp_get_history(h, None, 0, C.byref(n)), "asp_get_history", h)
    arr = (asp_iter_record * max(n.value, 1))()
    _check(lib().asp_get_history(h, arr, n.value, C.byref(n)), "asp_get_history", h)
    return [{f: getattr(r, f) for f, _ in asp_iter_record._fields_} for r in arr[: n.value]]


def asp_get_state(h) -> dict:
    nc, nr = C.c_int(), C.c_int()
    t = C.c_int64()
    wi, w0 = C.c_double(), C.c_double()
    _check(lib().asp_get_state(h, None, 0, C.byref(nc), None, 0, C.byref(nr), C.byref(t), C.byref(wi),
                               C.byref(w0)), "asp_get_state", h)
    comps = (asp_component * max(nc.value, 1))()
    ret = (C.c_int * max(nr.value, 1))()
    _check(lib().asp_get_state(h, comps, nc.value, C.byref(nc), ret, nr.value, C.byref(nr), C.byref(t),
                               C.byref(wi), C.byref(w0)), "asp_get_state", h)
    return dict(comps=_comp_rows(comps, nc.value), retained=[ret[i] for i in range(nr.value)], t=t.value,
                last_wi=wi.value, last_w0=w0.value)


def asp_set_state(h, comps, retained: Sequence[int], t: int, last_wi: float, last_w0: float):
    arr, n = _component_array(comps if len(comps) else np.zeros((0, 6)))
    ret = (C.c_int * max(len(retained), 1))(*retained)
    _check(lib().asp_set_state(h, arr, n, ret, len(retained), int(t), float(last_wi), float(last_w0)),
           "asp_set_state", h)


def asp_get_last_fit(h):
    """The most recent fit: (rows (a, x, y, w) in member order, info dict)."""
    n = C.c_int()
    arr = (asp_gauss * ASP_KMAX)()
    info = asp_fit_info()
    _check(lib().asp_get_last_fit(h, arr, ASP_KMAX, C.byref(n), C.byref(info)), "asp_get_last_fit", h)
    return (np.array([[g.amp, g.x, g.y, g.width] for g in arr[: n.value]]),
            {f.rstrip("_"): getattr(info, f) for f, _ in asp_fit_info._fields_})


def asp_save_state(h, path: str):
    _check(lib().asp_save_state(h, os.fsencode(path)), "asp_save_state", h)


def asp_load_state(h, path: str):
    _check(lib().asp_load_state(h, os.fsencode(path)), "asp_load_state", h)


# ----------------------------------------------------------------- batches

def asp_batch_create(params: asp_params, dirty: Sequence, psf: Sequence, stream=None):
    """asp_batch_create: lists of per-image dirty (H x W) and psf (2H x 2W)
    arrays, all numpy (host) or all float32 CUDA tensors (device)."""
    n = len(dirty)
    if n != len(psf) or n == 0:
        raise ValueError("dirty and psf must be non-empty lists of equal length")
    on_host = isinstance(dirty[0], np.ndarray)
    H = (C.c_int * n)()
    W = (C.c_int * n)()
    dp = (C.c_void_p * n)()
    pp = (C.c_void_p * n)()
    keep = []
    for i in range(n):
        h_, w_ = (int(dirty[i].shape[0]), int(dirty[i].shape[1]))
        H[i], W[i] = h_, w_
        if on_host:
            d = _host_f32(dirty[i], (h_, w_), "dirty")
            q = _host_f32(psf[i], (2 * h_, 2 * w_), "psf")
            keep += [d, q]
            dp[i], pp[i] = d.ctypes.data, q.ctypes.data
        else:
            dp[i] = _cuda_f32(dirty[i], (h_, w_), "dirty")
            pp[i] = _cuda_f32(psf[i], (2 * h_, 2 * w_), "psf")
    h = C.c_void_p()
    _check(lib().asp_batch_create(C.byref(params), n, H, W, dp, pp, 1 if on_host else 0, _stream_handle(stream),
                                  C.byref(h)), "asp_batch_create")
    return h.value


def asp_batch_destroy(b):
    _check(lib().asp_batch_destroy(b), "asp_batch_destroy")


def asp_batch_reset(b):
    _check(lib().asp_batch_reset(b), "asp_batch_reset")


def asp_batch_minor_cycle(b, n_iter: int, n_images: int) -> list:
    stats = (asp_cycle_stats * n_images)()
    _check(lib().asp_batch_minor_cycle(b, n_iter, stats), "asp_batch_minor_cycle")
    return [_stats_dict(stats[i]) for i in range(n_images)]


def asp_batch_run_queue(b, n_iter: int, n_lanes: int, px_per_cta: int, n_images: int) -> list:
    stats = (asp_cycle_stats * n_images)()
    _check(lib().asp_batch_run_queue(b, n_iter, n_lanes, px_per_cta, stats), "asp_batch_run_queue")
    return [_stats_dict(stats[i]) for i in range(n_images)]


def asp_batch_autotune(b, n_trial_iter: int) -> dict:
    t = _lib.asp_batch_tuning()
    _check(lib().asp_batch_autotune(b, n_trial_iter, C.byref(t)), "asp_batch_autotune")
    return {f: getattr(t, f) for f, _ in t._fields_}


def asp_batch_image(b, i: int):
    h = C.c_void_p()
    _check(lib().asp_batch_image(b, i, C.byref(h)), "asp_batch_image")
    return h.value


def asp_batch_launch_count(b) -> int:
    n = C.c_int64()
    _check(lib().asp_batch_launch_count(b, C.byref(n)), "asp_batch_launch_count")
    return n.value


# ----------------------------------------------------------------- convenience

class Context:
    """Owns one libasp context.  ``dirty``/``psf``: float32 CUDA tensors
    (device inputs) or numpy arrays (host inputs, copied in the call)."""

    def __init__(self, dirty, psf, params: Optional[asp_params] = None, stream=None, **overrides):
        self.params = params if params is not None else default_params(**overrides)
        if isinstance(dirty, np.ndarray):
            self.h = asp_init_host(self.params, dirty, psf, stream)
            self.H, self.W = np.shape(dirty)
        else:
            self.h = asp_init(self.params, dirty, psf, stream)
            self.H, self.W = int(dirty.shape[0]), int(dirty.shape[1])

    @classmethod
    def borrow(cls, h, H: int, W: int, params: asp_params) -> "Context":
        """A view of a context owned elsewhere (a batch image): same queries,
        close() leaves it alone."""
        c = cls.__new__(cls)
        c.h, c.H, c.W, c.params, c._borrowed = h, H, W, params, True
        return c

    def close(self):
        if self.h and not getattr(self, "_borrowed", False):
            asp_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def beam(self):
        return asp_get_beam(self.h)

    def find_peak(self, mode=ASP_PEAK_SIMPLE):
        return asp_find_peak(self.h, mode)

    def fit(self, init, n_old=0):
        return asp_fit_active_set(self.h, init, n_old)

    def fit_2004(self, init, n_old=0, omega_min=0.1):
        return asp_fit_2004(self.h, init, n_old, omega_min)

    def fit_elliptical(self, init, n_old=0):
        return asp_fit_elliptical(self.h, init, n_old)

    def beam_elliptical(self):
        return asp_fit_beam_elliptical(self.h)

    def deconvolve_elliptical(self, rows, beam):
        return asp_deconvolve_elliptical(self.h, rows, beam)

    def fit_lm(self, init, n_old, lambda0, max_iter, start=None):
        return asp_fit_lm(self.h, init, n_old, lambda0, max_iter, start)

    def normal_equations(self, theta, n_old, window):
        return asp_eval_normal_equations(self.h, theta, n_old, window)

    def subtract(self, comps, gain=1.0):
        asp_subtract(self.h, comps, gain)

    def subtract_beam(self, comps, gain=1.0):
        asp_subtract_beam(self.h, comps, gain)

    def minor_cycle(self, n_iter):
        return asp_minor_cycle(self.h, n_iter)

    def stats(self):
        return asp_get_stats(self.h)

    def set_profiling(self, on: bool):
        """CUDA events around every launch (direct launches, no graph)."""
        _check(lib().asp_set_profiling(self.h, 1 if on else 0), "asp_set_profiling", self.h)

    def kernel_times(self):
        """Per kernel class since profiling was switched on: name, launches,
        total milliseconds."""
        kt = (_lib.asp_kernel_time * 32)()
        nk = C.c_int()
        _check(lib().asp_get_kernel_times(self.h, kt, 32, C.byref(nk)), "asp_get_kernel_times", self.h)
        return [{"name": k.name.decode(), "launches": int(k.launches), "total_ms": float(k.total_ms)}
                for k in kt[: nk.value]]

    def residual(self) -> np.ndarray:
        out = np.empty((self.H, self.W), dtype=np.float32)
        return asp_copy_residual(self.h, out)

    def residual_device(self):
        import torch
        out = torch.empty((self.H, self.W), dtype=torch.float32, device="cuda")
        return asp_copy_residual(self.h, out)

    def set_residual(self, src):
        asp_set_residual(self.h, src)

    def components(self):
        return asp_get_components(self.h)

    def history(self):
        return asp_get_history(self.h)

    def state(self):
        return asp_get_state(self.h)

    def last_fit(self):
        return asp_get_last_fit(self.h)

    def set_state(self, comps, retained, t, last_wi, last_w0):
        asp_set_state(self.h, comps, retained, t, last_wi, last_w0)

    def smooth(self, j):
        import torch
        out = torch.empty((self.H, self.W), dtype=torch.float32, device="cuda")
        return asp_smooth(self.h, j, out)

    def scales(self):
        return asp_num_scales(self.h)

    def set_mlp(self, weights: Optional[dict], enable: bool = True):
        """Learned initial values from the network ``weights`` (dict of
        W1 b1 W2 b2 W3 b3); ``enable=False`` (or None) switches them off."""
        if weights is None or not enable:
            _check(lib().asp_set_mlp(self.h, None, 0), "asp_set_mlp")
            return
        v = np.ascontiguousarray(mlp_pack(weights), dtype=np.float32)
        _check(lib().asp_set_mlp(self.h, v.ctypes.data, 1), "asp_set_mlp")

    def set_harvest(self, patches=None, targets=None):
        """Record (patch, converged-fit target) pairs into CUDA tensors
        patches (cap x 1024) and targets (cap x 8); None switches it off."""
        if patches is None:
            _check(lib().asp_set_harvest(self.h, None, None, 0), "asp_set_harvest")
            return
        cap = int(patches.shape[0])
        if tuple(patches.shape) != (cap, 1024) or tuple(targets.shape) != (cap, 8):
            raise ValueError("patches must be cap x 1024 and targets cap x 8")
        _check(lib().asp_set_harvest(self.h, _cuda_f32(patches, (cap, 1024), "patches"),
                                     _cuda_f32(targets, (cap, 8), "targets"), cap), "asp_set_harvest")


class Batch:
    """Owns one libasp batch: independent images advanced together, the LM
    fits of all images in one cooperative launch per iteration."""

    def __init__(self, dirty: Sequence, psf: Sequence, params: Optional[asp_params] = None, stream=None,
                 **overrides):
        self.params = params if params is not None else default_params(**overrides)
        self.shapes = [(int(d.shape[0]), int(d.shape[1])) for d in dirty]
        self.h = asp_batch_create(self.params, dirty, psf, stream)

    @property
    def n(self) -> int:
        return len(self.shapes)

    def close(self):
        if self.h:
            asp_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        asp_batch_reset(self.h)

    def minor_cycle(self, n_iter: int) -> list:
        return asp_batch_minor_cycle(self.h, n_iter, self.n)

    def autotune(self, n_trial_iter: int = 16) -> dict:
        return asp_batch_autotune(self.h, n_trial_iter)

    def run_queue(self, n_iter: int, n_lanes: int = 8, px_per_cta: int = 0) -> list:
        """Work queue: every image runs its own minor cycle, the images spread
        over n_lanes CUDA streams (asp_batch_run_queue)."""
        return asp_batch_run_queue(self.h, n_iter, n_lanes, px_per_cta, self.n)

    def fit_joint(self, init, n_old: int = 0):
        """Joint wide-band fit over the batch's images as channels: rows
        (x, y, s, a_1 .. a_C).  Returns (fitted rows, flux [n, C] by Eq. 8
        per channel, is_point [n], info dict)."""
        return asp_batch_fit_joint(self.h, init, n_old, self.n)

    def image(self, i: int) -> Context:
        H, W = self.shapes[i]
        return Context.borrow(asp_batch_image(self.h, i), H, W, self.params)

    def launches(self) -> int:
        return asp_batch_launch_count(self.h)

    def set_mlp(self, weights: Optional[dict], enable: bool = True):
        """Learned initial values for every image (see Context.set_mlp)."""
        if weights is None or not enable:
            _check(lib().asp_batch_set_mlp(self.h, None, 0), "asp_batch_set_mlp")
            return
        v = np.ascontiguousarray(mlp_pack(weights), dtype=np.float32)
        _check(lib().asp_batch_set_mlp(self.h, v.ctypes.data, 1), "asp_batch_set_mlp")


# ----------------------------------------------------------------- learned initial values

MLP_SHAPES = (("W1", (256, 1024)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (4, 256)), ("b3", (4,)))


def mlp_pack(weights: dict) -> np.ndarray:
    """Parameter dict (W1, b1, W2, b2, W3, b3) -> the library's FP32 vector."""
    return np.concatenate([np.asarray(weights[n], dtype=np.float32).reshape(-1) for n, _ in MLP_SHAPES])


def mlp_unpack(vec) -> dict:
    out, o = {}, 0
    for n, shp in MLP_SHAPES:
        k = int(np.prod(shp))
        out[n] = np.asarray(vec[o:o + k]).reshape(shp)
        o += k
    return out


class MLP:
    """Owns one trainer of the learned-initial-value network (asp_mlp_*)."""

    def __init__(self, weights: dict, max_batch: int = 1024, stream=None):
        n = C.c_longlong()
        _check(lib().asp_mlp_num_params(C.byref(n)), "asp_mlp_num_params")
        self.n_params = n.value
        v = np.ascontiguousarray(mlp_pack(weights), dtype=np.float32)
        if v.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {v.size}")
        h = C.c_void_p()
        _check(lib().asp_mlp_create(v.ctypes.data, int(max_batch), _stream_handle(stream), C.byref(h)), "asp_mlp_create")
        self.h = h.value
        self.max_batch = int(max_batch)

    def close(self):
        if self.h:
            lib().asp_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        if X.ndim != 2 or X.shape[1] != 1024 or T.shape != (X.shape[0], 4):
            raise ValueError("X must be n x 1024 and T n x 4")
        _check(lib().asp_mlp_set_data(self.h, X.ctypes.data, T.ctypes.data, X.shape[0]), "asp_mlp_set_data")

    def step(self, idx, lr: float = 1e-3, update: bool = True, grads: bool = False):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        loss = C.c_float()
        g = np.empty(self.n_params, dtype=np.float32) if grads else None
        _check(lib().asp_mlp_step(self.h, idx.ctypes.data_as(C.POINTER(C.c_int)), idx.size, float(lr), int(update),
                                  C.byref(loss), g.ctypes.data if grads else None), "asp_mlp_step")
        return (loss.value, mlp_unpack(g)) if grads else loss.value

    def predict(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.empty((X.shape[0], 4), dtype=np.float32)
        _check(lib().asp_mlp_predict(self.h, X.ctypes.data, X.shape[0], Y.ctypes.data), "asp_mlp_predict")
        return Y

    def params(self) -> dict:
        v = np.empty(self.n_params, dtype=np.float32)
        _check(lib().asp_mlp_get_params(self.h, v.ctypes.data), "asp_mlp_get_params")
        return mlp_unpack(v)
