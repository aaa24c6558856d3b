"""ctypes binding of libgce.so (include/gce.h), with the C ABI's names.

Argument marshalling only: tensors are checked for dtype, device and layout
and passed as raw pointers together with torch's current CUDA stream; every
step of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgce.so")

GCE_OK, GCE_ERR_INVALID, GCE_ERR_CUDA, GCE_ERR_NOMEM, GCE_ERR_UNSUPPORTED = range(5)
GCE_PHASE_FP64, GCE_PHASE_SPLIT32, GCE_PHASE_FIXED32 = 0, 1, 2
GCE_FLAG_NO_GRAPH = 1
GCE_FLAG_TIME_KERNEL = 2
GCE_FLAG_OVERLAP = 4
GCE_MAX_PHASE_BINS, GCE_MAX_MAG_BINS, GCE_MAX_CURVE_POINTS, GCE_MAX_TOPK = 256, 255, 65535, 64
GCE_MAX_BANDS = 8
MODES = {"fp64": GCE_PHASE_FP64, "split32": GCE_PHASE_SPLIT32, "fixed32": GCE_PHASE_FIXED32}


class GceError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class gce_config(ctypes.Structure):
    _fields_ = [("n_phase_bins", ctypes.c_int32), ("n_mag_bins", ctypes.c_int32),
                ("phase_mode", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("t0", ctypes.c_double)]


class gce_tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("tpt", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("slot_range", ctypes.c_int32)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_CFG = ctypes.POINTER(gce_config)
_TUN = ctypes.POINTER(gce_tuning)
_HOFF = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); every symbol declared in include/gce.h
SIGNATURES = {
    "gce_create": (_I32, [ctypes.POINTER(_P), _I32]),
    "gce_destroy": (_I32, [_P]),
    "gce_status_string": (ctypes.c_char_p, [_I32]),
    "gce_last_error": (ctypes.c_char_p, [_P]),
    "gce_check_job": (_I32, [_HOFF, _I32, _I32, _I32, _CFG, _I32]),
    "gce_ce_grid": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _P, _P]),
    "gce_ce_topk": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _I32, _P, _P, _P]),
    "gce_ce_detect": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _I32, _P, _P, _P,
                             _P, _P, _P]),
    "gce_ce_grid_bands": (_I32, [_P, _P, _P, _P, _I32, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _P,
                                 _P]),
    "gce_ce_detect_bands": (_I32, [_P, _P, _P, _P, _I32, _HOFF, _I32, _P, _I32, _P, _I32, _CFG,
                                   _I32, _P, _P, _P, _P, _P, _P]),
    "gce_ce_topk_host": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _I32, _P, _P,
                                _P]),
    "gce_ce_topk_static": (_I32, [_P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _I32, _P, _P,
                                  _P]),
    "gce_ce_grid_single": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _P, _P]),
    "gce_ce_counts": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG, _I64, _P, _P, _P,
                             _P]),
    "gce_stream_status": (_I32, [_P, _P]),
    "gce_kernel_time": (_I32, [_P, ctypes.POINTER(ctypes.c_float)]),
    "gce_last_launches": (_I32, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "gce_autotune": (_I32, [_P, _CFG, _I32, _I64]),
    "gce_autotune_job": (_I32, [_P, _P, _P, _HOFF, _I32, _P, _I32, _P, _I32, _CFG]),
    "gce_get_tuning": (_I32, [_P, _CFG, _I32, _I32, _TUN]),
    "gce_set_tuning": (_I32, [_P, _CFG, _I32, _TUN]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                               "(python -m paper_2006_06866_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


@dataclass
class Config:
    n_phase_bins: int = 15
    n_mag_bins: int = 10
    phase_mode: int = GCE_PHASE_FIXED32
    t0: float = 0.0
    use_graph: bool = True
    time_kernel: bool = False
    overlap: bool = False

    def c(self):
        mode = MODES[self.phase_mode] if isinstance(self.phase_mode, str) else self.phase_mode
        flags = (0 if self.use_graph else GCE_FLAG_NO_GRAPH) | \
            (GCE_FLAG_TIME_KERNEL if self.time_kernel else 0) | \
            (GCE_FLAG_OVERLAP if self.overlap else 0)
        return gce_config(int(self.n_phase_bins), int(self.n_mag_bins), int(mode), flags,
                          float(self.t0))


def _check(status, handle=None):
    if status != GCE_OK:
        L = lib()
        msg = L.gce_last_error(handle) or L.gce_status_string(status)
        raise GceError(status, msg.decode() if isinstance(msg, bytes) else str(msg))


def _host_offsets(offsets):
    if hasattr(offsets, "detach"):
        offsets = offsets.detach().cpu().numpy()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return off, off.ctypes.data_as(_HOFF)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Handle:
    """Owns one gce_handle (device workspace, autotune cache, CUDA graphs)."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().gce_create(ctypes.byref(self._h), int(device)))
        self.device = device

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            lib().gce_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gce_check_job(offsets, n_periods, n_pdots, cfg: Config, k=0):
    off, poff = _host_offsets(offsets)
    c = cfg.c()
    return lib().gce_check_job(poff, off.shape[0] - 1, int(n_periods), int(n_pdots),
                               ctypes.byref(c), int(k))


def one_device(named, device=None):
    """The CUDA device index shared by every tensor of (name, tensor) pairs
    (None entries skipped); raises ValueError if they lie on different devices or
    not on `device` (a handle's device) when that is given."""
    idx = None
    for name, t in named:
        if t is None:
            continue
        d = t.device.index
        if idx is None:
            idx = d
        elif d != idx:
            raise ValueError(f"{name} is on cuda:{d}, the other arrays on cuda:{idx}")
    if device is not None and idx is not None and idx != device:
        raise ValueError(f"the arrays are on cuda:{idx}, the handle on cuda:{device}")
    return idx


def _common(times, mags, offsets, periods, pdots, handle=None):
    import torch
    off, poff = _host_offsets(offsets)
    out = (off, poff, _dev(times, torch.float64, "times"), _dev(mags, torch.float64, "mags"),
           _dev(periods, torch.float64, "periods"), _dev(pdots, torch.float64, "pdots"))
    one_device([("times", times), ("mags", mags), ("periods", periods), ("pdots", pdots)],
               None if handle is None else handle.device)
    return out


def gce_ce_grid(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config, out=None,
                stream=None):
    """H[n_curves, n_pdots, n_periods] (float32 CUDA tensor)."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    if out is None:
        out = torch.empty((nc, pdots.numel(), periods.numel()), dtype=torch.float32,
                          device=times.device)
    c = cfg.c()
    _check(lib().gce_ce_grid(handle.ptr, pt, pm, poff, nc, pp, periods.numel(), pd, pdots.numel(),
                             ctypes.byref(c), _dev(out, torch.float32, "out"), _stream(stream)),
           handle.ptr)
    return out


def gce_ce_grid_single(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config,
                       out=None, stream=None):
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    if out is None:
        out = torch.empty((nc, pdots.numel(), periods.numel()), dtype=torch.float32,
                          device=times.device)
    c = cfg.c()
    _check(lib().gce_ce_grid_single(handle.ptr, pt, pm, poff, nc, pp, periods.numel(), pd,
                                    pdots.numel(), ctypes.byref(c),
                                    _dev(out, torch.float32, "out"), _stream(stream)),
           handle.ptr)
    return out


def gce_ce_topk(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config, k: int,
                out_H=None, out_idx=None, stream=None):
    """(topk_H float32[n_curves, k], topk_idx int64[n_curves, k]) CUDA tensors."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    if out_H is None:
        out_H = torch.empty((nc, k), dtype=torch.float32, device=times.device)
    if out_idx is None:
        out_idx = torch.empty((nc, k), dtype=torch.int64, device=times.device)
    c = cfg.c()
    _check(lib().gce_ce_topk(handle.ptr, pt, pm, poff, nc, pp, periods.numel(), pd,
                             pdots.numel(), ctypes.byref(c), int(k),
                             _dev(out_H, torch.float32, "topk_H"),
                             _dev(out_idx, torch.int64, "topk_idx"), _stream(stream)),
           handle.ptr)
    return out_H, out_idx


def gce_ce_detect(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config, k: int,
                  stream=None):
    """(topk_H, topk_idx, mean, std, rho) CUDA tensors: the k smallest cells and the
    significance rho = (mean - H_min) / std of each curve (Eq. 5)."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    dev = times.device
    tH = torch.empty((nc, k), dtype=torch.float32, device=dev)
    tI = torch.empty((nc, k), dtype=torch.int64, device=dev)
    mean = torch.empty(nc, dtype=torch.float64, device=dev)
    std = torch.empty(nc, dtype=torch.float64, device=dev)
    rho = torch.empty(nc, dtype=torch.float32, device=dev)
    c = cfg.c()
    _check(lib().gce_ce_detect(handle.ptr, pt, pm, poff, nc, pp, periods.numel(), pd,
                               pdots.numel(), ctypes.byref(c), int(k),
                               _dev(tH, torch.float32, "topk_H"), _dev(tI, torch.int64, "topk_idx"),
                               _dev(mean, torch.float64, "mean"), _dev(std, torch.float64, "std"),
                               _dev(rho, torch.float32, "rho"), _stream(stream)), handle.ptr)
    return tH, tI, mean, std, rho


def gce_ce_grid_bands(handle: Handle, times, mags, bands, n_bands: int, offsets, periods, pdots,
                      cfg: Config, out=None, stream=None):
    """gce_ce_grid on multi-filter input: bands is a uint8 CUDA tensor (the filter
    of each point, < n_bands); each (curve, filter) is median/std normalised."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    if out is None:
        out = torch.empty((nc, pdots.numel(), periods.numel()), dtype=torch.float32,
                          device=times.device)
    c = cfg.c()
    _check(lib().gce_ce_grid_bands(handle.ptr, pt, pm, _dev(bands, torch.uint8, "bands"),
                                   int(n_bands), poff, nc, pp, periods.numel(), pd, pdots.numel(),
                                   ctypes.byref(c), _dev(out, torch.float32, "out"),
                                   _stream(stream)), handle.ptr)
    return out


def gce_ce_detect_bands(handle: Handle, times, mags, bands, n_bands: int, offsets, periods, pdots,
                        cfg: Config, k: int, significance=True, stream=None):
    """gce_ce_detect on multi-filter input; (topk_H, topk_idx, mean, std, rho), the
    last three None when significance is False."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    dev = times.device
    tH = torch.empty((nc, k), dtype=torch.float32, device=dev)
    tI = torch.empty((nc, k), dtype=torch.int64, device=dev)
    mean = std = rho = None
    pm_, ps_, pr_ = None, None, None
    if significance:
        mean = torch.empty(nc, dtype=torch.float64, device=dev)
        std = torch.empty(nc, dtype=torch.float64, device=dev)
        rho = torch.empty(nc, dtype=torch.float32, device=dev)
        pm_ = _dev(mean, torch.float64, "mean")
        ps_ = _dev(std, torch.float64, "std")
        pr_ = _dev(rho, torch.float32, "rho")
    c = cfg.c()
    _check(lib().gce_ce_detect_bands(handle.ptr, pt, pm, _dev(bands, torch.uint8, "bands"),
                                     int(n_bands), poff, nc, pp, periods.numel(), pd,
                                     pdots.numel(), ctypes.byref(c), int(k),
                                     _dev(tH, torch.float32, "topk_H"),
                                     _dev(tI, torch.int64, "topk_idx"), pm_, ps_, pr_,
                                     _stream(stream)), handle.ptr)
    return tH, tI, mean, std, rho


def gce_ce_topk_host(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config, k: int,
                     out_H=None, out_idx=None, stream=None):
    """Host arrays in, host arrays out (numpy or CPU tensors; pinned CPU tensors
    make the copies asynchronous).  Synchronous; returns (topk_H, topk_idx)."""
    import torch

    def host(a, dt, name):
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != dt or not a.is_contiguous():
                raise TypeError(f"{name} must be a contiguous CPU {dt} tensor")
            return a, ctypes.c_void_p(a.data_ptr())
        arr = np.ascontiguousarray(a, dtype=np.float64 if dt == torch.float64 else None)
        return arr, ctypes.c_void_p(arr.ctypes.data)

    off, poff = _host_offsets(offsets)
    nc = off.shape[0] - 1
    t, pt = host(times, torch.float64, "times")
    m, pm = host(mags, torch.float64, "mags")
    p, pp = host(periods, torch.float64, "periods")
    d, pd = host(pdots, torch.float64, "pdots")
    n_p = int(p.numel() if isinstance(p, torch.Tensor) else p.size)
    n_q = int(d.numel() if isinstance(d, torch.Tensor) else d.size)
    if out_H is None:
        out_H = torch.empty((nc, k), dtype=torch.float32)
    if out_idx is None:
        out_idx = torch.empty((nc, k), dtype=torch.int64)
    c = cfg.c()
    _check(lib().gce_ce_topk_host(handle.ptr, pt, pm, poff, nc, pp, n_p, pd, n_q,
                                  ctypes.byref(c), int(k), ctypes.c_void_p(out_H.data_ptr()),
                                  ctypes.c_void_p(out_idx.data_ptr()), _stream(stream)),
           handle.ptr)
    return out_H, out_idx


def gce_ce_topk_static(times, mags, offsets, periods, pdots, cfg: Config, k: int, out_H=None,
                       out_idx=None, stream=None):
    """gce_ce_topk without a handle and without any device allocation by the
    library (its workspace is a built-in 32 MiB array).  Synchronous; raises
    GceError on a non-OK status (GCE_ERR_NOMEM: the job is too large for it)."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots)
    nc = off.shape[0] - 1
    if out_H is None:
        out_H = torch.empty((nc, k), dtype=torch.float32, device=times.device)
    if out_idx is None:
        out_idx = torch.empty((nc, k), dtype=torch.int64, device=times.device)
    one_device([("times", times), ("topk_H", out_H), ("topk_idx", out_idx)])
    c = cfg.c()
    # the call runs on the current device: make it the arrays' device
    with torch.cuda.device(times.device):
        st = lib().gce_ce_topk_static(pt, pm, poff, nc, pp, periods.numel(), pd, pdots.numel(),
                                      ctypes.byref(c), int(k),
                                      _dev(out_H, torch.float32, "topk_H"),
                                      _dev(out_idx, torch.int64, "topk_idx"), _stream(stream))
    if st != GCE_OK:
        raise GceError(st, lib().gce_status_string(st).decode())
    return out_H, out_idx


def gce_ce_counts(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config, cell_curve,
                  cell_trial, stream=None):
    """uint32 counts[n_cells, n_mag_bins, n_phase_bins] as an int32 CUDA tensor view."""
    import torch
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    nc = off.shape[0] - 1
    n_cells = cell_curve.numel()
    counts = torch.empty((n_cells, cfg.n_mag_bins, cfg.n_phase_bins), dtype=torch.int32,
                         device=times.device)
    c = cfg.c()
    _check(lib().gce_ce_counts(handle.ptr, pt, pm, poff, nc, pp, periods.numel(), pd,
                               pdots.numel(), ctypes.byref(c), n_cells,
                               _dev(cell_curve, torch.int64, "cell_curve"),
                               _dev(cell_trial, torch.int64, "cell_trial"),
                               _dev(counts, torch.int32, "counts"), _stream(stream)),
           handle.ptr)
    return counts


def gce_stream_status(handle: Handle, stream=None) -> int:
    """Waits for the stream; returns the status of the device-side input checks."""
    return lib().gce_stream_status(handle.ptr, _stream(stream))


def gce_kernel_time(handle: Handle) -> float:
    """Milliseconds of the CE kernel of the last call made with time_kernel=True."""
    ms = ctypes.c_float()
    _check(lib().gce_kernel_time(handle.ptr, ctypes.byref(ms)), handle.ptr)
    return float(ms.value)


def gce_last_launches(handle: Handle) -> int:
    """Kernels the last search call on this handle launched (directly or in its graph)."""
    n = ctypes.c_int32()
    _check(lib().gce_last_launches(handle.ptr, ctypes.byref(n)), handle.ptr)
    return int(n.value)


def gce_autotune(handle: Handle, cfg: Config, n_obs_hint: int, n_trials_hint: int):
    c = cfg.c()
    _check(lib().gce_autotune(handle.ptr, ctypes.byref(c), int(n_obs_hint), int(n_trials_hint)),
           handle.ptr)


def gce_autotune_job(handle: Handle, times, mags, offsets, periods, pdots, cfg: Config):
    """Tune the launch shape on a bounded slice of this job (see gce.h)."""
    off, poff, pt, pm, pp, pd = _common(times, mags, offsets, periods, pdots, handle)
    c = cfg.c()
    _check(lib().gce_autotune_job(handle.ptr, pt, pm, poff, off.shape[0] - 1, pp, periods.numel(),
                                  pd, pdots.numel(), ctypes.byref(c)), handle.ptr)


def gce_get_tuning(handle: Handle, cfg: Config, n_obs_hint: int, n_pdots: int = 1):
    c = cfg.c()
    t = gce_tuning()
    _check(lib().gce_get_tuning(handle.ptr, ctypes.byref(c), int(n_obs_hint), int(n_pdots),
                                ctypes.byref(t)), handle.ptr)
    return {"block": t.block, "tpt": t.tpt, "ctas_per_sm": t.ctas_per_sm, "chunk": t.chunk,
            "slot_range": t.slot_range}


def gce_set_tuning(handle: Handle, cfg: Config, n_obs_hint: int, block=256, tpt=2,
                   ctas_per_sm=0, chunk=2048, slot_range=0):
    c = cfg.c()
    t = gce_tuning(int(block), int(tpt), int(ctas_per_sm), int(chunk), int(slot_range))
    _check(lib().gce_set_tuning(handle.ptr, ctypes.byref(c), int(n_obs_hint), ctypes.byref(t)),
           handle.ptr)
