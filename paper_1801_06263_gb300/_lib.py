"""Thin ctypes binding of the C-ABI in include/osscir.h (argument marshalling only).

Every function here forwards to the CUDA library libosscir.so with the same
name; torch tensors are passed as raw device pointers and streams as raw
cudaStream_t handles.  There is no CPU fallback: if the library is missing or
a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

OSSCIR_OK = 0
OSSCIR_E_INVALID = -1
OSSCIR_E_NOMEM = -2
OSSCIR_E_CUDA = -3
OSSCIR_E_TIMEOUT = -4
OSSCIR_E_DIVERGED = -5
OSSCIR_E_BUSY = -6
OSSCIR_E_NOTFOUND = -7

# Every symbol include/osscir.h declares.
EXPORTS = (
    "osscir_status_string", "osscir_create", "osscir_destroy", "osscir_info", "osscir_forward",
    "osscir_backproject", "osscir_simulate", "osscir_set_counts", "osscir_mocca_step", "osscir_get_maps",
    "osscir_get_state", "osscir_set_state", "osscir_dtpl", "osscir_footprint_rays",
    "osscir_footprint_pixels", "osscir_reconstruct", "osscir_last_kernel_ms", "osscir_dtpl_counts_static",
    "osscir_server_create", "osscir_server_destroy", "osscir_submit", "osscir_poll", "osscir_server_info",
    "osscir_batch_create", "osscir_batch_destroy", "osscir_batch_step", "osscir_batch_get_config",
    "osscir_batch_set_config", "osscir_batch_last_kernel_ms", "osscir_poisson_noise", "osscir_mocca_partial",
    "osscir_mocca_apply", "osscir_memory",
)


class OsscirError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} failed: {status} ({_status_string(status)})")


class Geometry(ct.Structure):
    _fields_ = [("n", ct.c_int), ("pixel_mm", ct.c_double), ("n_views", ct.c_int),
                ("arc_deg", ct.c_double), ("start_deg", ct.c_double), ("n_bins", ct.c_int),
                ("bin_mm", ct.c_double), ("sid_mm", ct.c_double), ("sdd_mm", ct.c_double)]


class Spectra(ct.Structure):
    _fields_ = [("n_energies", ct.c_int), ("s", ct.POINTER(ct.c_float)), ("N", ct.POINTER(ct.c_float)),
                ("n_windows", ct.c_int)]


class Params(ct.Structure):
    _fields_ = [("lambda_", ct.c_double), ("model", ct.c_int), ("use_box", ct.c_int),
                ("lo", ct.c_float * 3), ("hi", ct.c_float * 3), ("spc", ct.c_int), ("counts_model", ct.c_int),
                ("inner", ct.c_int)]


class Request(ct.Structure):
    _fields_ = [("geom", Geometry), ("spectra", Spectra), ("mu", ct.POINTER(ct.c_float)), ("params", Params),
                ("counts", ct.POINTER(ct.c_float)), ("n_iters", ct.c_int)]


class BatchConfig(ct.Structure):
    _fields_ = [("proj_views", ct.c_int), ("proj_grid", ct.c_int), ("proj_order", ct.c_int),
                ("ray_grid", ct.c_int), ("ray_order", ct.c_int), ("bp_tile_x", ct.c_int),
                ("bp_grid", ct.c_int), ("bp_order", ct.c_int), ("branches", ct.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Stats(ct.Structure):
    _fields_ = [("status", ct.c_int), ("iterations", ct.c_int), ("dtpl", ct.c_double),
                ("latency_ms", ct.c_double), ("queue_ms", ct.c_double), ("gpu_ms", ct.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libosscir.so (building it first if allowed); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {_build.LIB}")
        _build.build()
    L = ct.CDLL(_build.LIB)
    vp, ip, fp, dp = ct.c_void_p, ct.POINTER(ct.c_int), ct.c_void_p, ct.POINTER(ct.c_double)
    sig = {
        "osscir_status_string": ([ct.c_int], ct.c_char_p),
        "osscir_create": ([ct.POINTER(Geometry), ct.POINTER(Spectra), ct.POINTER(ct.c_float),
                           ct.POINTER(Params), ct.POINTER(ct.c_void_p)], ct.c_int),
        "osscir_destroy": ([vp], ct.c_int),
        "osscir_info": ([vp, ip, ip, ip], ct.c_int),
        "osscir_forward": ([vp, fp, fp, vp], ct.c_int),
        "osscir_backproject": ([vp, fp, fp, vp], ct.c_int),
        "osscir_simulate": ([vp, fp, fp, vp], ct.c_int),
        "osscir_set_counts": ([vp, fp, vp], ct.c_int),
        "osscir_mocca_step": ([vp, ct.c_int, vp], ct.c_int),
        "osscir_get_maps": ([vp, fp, vp], ct.c_int),
        "osscir_get_state": ([vp, fp, fp, fp, ip, vp], ct.c_int),
        "osscir_set_state": ([vp, fp, fp, fp, ct.c_int, vp], ct.c_int),
        "osscir_dtpl": ([vp, ct.c_int, dp, vp], ct.c_int),
        "osscir_footprint_rays": ([vp, ct.c_int, ct.c_int, ct.c_int, vp, vp, vp, vp], ct.c_int),
        "osscir_footprint_pixels": ([vp, ct.c_int, ct.c_int, ct.c_int, vp, vp, vp, vp], ct.c_int),
        "osscir_reconstruct": ([vp, vp, ct.c_int, vp, vp], ct.c_int),
        "osscir_last_kernel_ms": ([vp, ct.POINTER(ct.c_float), vp], ct.c_int),
        "osscir_dtpl_counts_static": ([vp, vp, ct.c_int, vp, vp], ct.c_int),
        "osscir_server_create": ([ct.c_size_t, ct.c_int, ct.POINTER(ct.c_void_p)], ct.c_int),
        "osscir_server_destroy": ([vp], ct.c_int),
        "osscir_submit": ([vp, ct.POINTER(Request), ct.POINTER(ct.c_uint64)], ct.c_int),
        "osscir_poll": ([vp, ct.c_uint64, ct.c_int, vp, ct.POINTER(Stats)], ct.c_int),
        "osscir_server_info": ([vp, ip, ip, ct.POINTER(ct.c_size_t)], ct.c_int),
        "osscir_batch_create": ([ct.POINTER(ct.c_void_p), ct.c_int, ct.c_int, ct.POINTER(ct.c_void_p)], ct.c_int),
        "osscir_batch_destroy": ([vp], ct.c_int),
        "osscir_batch_step": ([vp, ct.c_int, vp], ct.c_int),
        "osscir_batch_get_config": ([vp, ct.POINTER(BatchConfig)], ct.c_int),
        "osscir_batch_set_config": ([vp, ct.POINTER(BatchConfig)], ct.c_int),
        "osscir_batch_last_kernel_ms": ([vp, ct.POINTER(ct.c_float), vp], ct.c_int),
        "osscir_poisson_noise": ([vp, ct.c_int, ct.c_uint64, vp, vp], ct.c_int),
        "osscir_mocca_partial": ([vp, ct.c_int, ct.c_int, vp, vp], ct.c_int),
        "osscir_mocca_apply": ([vp, vp, vp], ct.c_int),
        "osscir_memory": ([vp, ct.POINTER(ct.c_size_t), ct.POINTER(ct.c_size_t)], ct.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _status_string(s: int) -> str:
    try:
        return load().osscir_status_string(int(s)).decode()
    except Exception:  # pragma: no cover - only used for messages
        return "?"


def _check(fn, st):
    if st != OSSCIR_OK:
        raise OsscirError(fn, st)


def _ptr(t):
    """Device pointer of a contiguous torch tensor (or None)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ct.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------------------- C-ABI mirrors

def _geometry(geom):
    return Geometry(int(geom.n), float(geom.pixel_mm), int(geom.n_views), float(geom.arc_deg),
                    float(geom.start_deg), int(geom.n_bins), float(geom.bin_mm), float(geom.sid_mm),
                    float(geom.sdd_mm))


def _params(lam, model=0, box=None, spc=0, counts_model=0, inner=1):
    lo, hi = (box if box is not None else ((0.0,) * 3, (0.0,) * 3))
    return Params(float(lam), int(model), int(box is not None), (ct.c_float * 3)(*lo), (ct.c_float * 3)(*hi),
                  int(spc), int(counts_model), int(inner))


def window_stride(n_windows: int) -> int:
    """Floats per ray of the per-ray window arrays (counts, dual): 4 for four windows, 8 for five."""
    return 4 * ((int(n_windows) + 3) // 4)


def osscir_create(geom, s, N, mu, lam, model=0, box=None, spc=0, counts_model=0, inner=1):
    """geom: object with the osscir_geometry fields; s [n_bins, nE, W], N [n_bins, W]
    (W = 4 or 5 windows), mu [3, nE] host arrays (copied).  Returns the handle (int)."""
    L = load()
    s32 = np.ascontiguousarray(s, dtype=np.float32)
    N32 = np.ascontiguousarray(N, dtype=np.float32)
    mu32 = np.ascontiguousarray(mu, dtype=np.float32)
    if s32.ndim != 3 or N32.shape != (s32.shape[0], s32.shape[2]):
        raise ValueError("s must be [n_bins, nE, W] and N [n_bins, W]")
    g = _geometry(geom)
    sp = Spectra(int(s32.shape[1]), s32.ctypes.data_as(ct.POINTER(ct.c_float)),
                 N32.ctypes.data_as(ct.POINTER(ct.c_float)), int(s32.shape[2]))
    p = _params(lam, model, box, spc, counts_model, inner)
    h = ct.c_void_p()
    _check("osscir_create", L.osscir_create(ct.byref(g), ct.byref(sp),
                                            mu32.ctypes.data_as(ct.POINTER(ct.c_float)), ct.byref(p),
                                            ct.byref(h)))
    return h.value


def osscir_destroy(h):
    _check("osscir_destroy", load().osscir_destroy(ct.c_void_p(h)))


def osscir_info(h):
    P, Lr, E = ct.c_int(), ct.c_int(), ct.c_int()
    _check("osscir_info", load().osscir_info(ct.c_void_p(h), ct.byref(P), ct.byref(Lr), ct.byref(E)))
    return P.value, Lr.value, E.value


def osscir_memory(h):
    """(device bytes of the context, bytes of its footprint tables)."""
    d, t = ct.c_size_t(), ct.c_size_t()
    _check("osscir_memory", load().osscir_memory(ct.c_void_p(h), ct.byref(d), ct.byref(t)))
    return d.value, t.value


def osscir_forward(h, x, g, stream=None):
    _check("osscir_forward", load().osscir_forward(ct.c_void_p(h), _ptr(x), _ptr(g), _stream(stream)))


def osscir_backproject(h, rf, img, stream=None):
    _check("osscir_backproject", load().osscir_backproject(ct.c_void_p(h), _ptr(rf), _ptr(img),
                                                           _stream(stream)))


def osscir_simulate(h, f, chat, stream=None):
    _check("osscir_simulate", load().osscir_simulate(ct.c_void_p(h), _ptr(f), _ptr(chat), _stream(stream)))


def osscir_set_counts(h, c, stream=None):
    _check("osscir_set_counts", load().osscir_set_counts(ct.c_void_p(h), _ptr(c), _stream(stream)))


def osscir_mocca_step(h, n_iters, stream=None):
    _check("osscir_mocca_step", load().osscir_mocca_step(ct.c_void_p(h), int(n_iters), _stream(stream)))


def osscir_get_maps(h, x_out, stream=None):
    _check("osscir_get_maps", load().osscir_get_maps(ct.c_void_p(h), _ptr(x_out), _stream(stream)))


def osscir_get_state(h, x, xbar, y, stream=None):
    it = ct.c_int()
    _check("osscir_get_state", load().osscir_get_state(ct.c_void_p(h), _ptr(x), _ptr(xbar), _ptr(y),
                                                       ct.byref(it), _stream(stream)))
    return it.value


def osscir_set_state(h, x, xbar, y, iteration, stream=None):
    _check("osscir_set_state", load().osscir_set_state(ct.c_void_p(h), _ptr(x), _ptr(xbar), _ptr(y),
                                                       int(iteration), _stream(stream)))


def osscir_dtpl(h, which=0, stream=None):
    out = ct.c_double()
    _check("osscir_dtpl", load().osscir_dtpl(ct.c_void_p(h), int(which), ct.byref(out), _stream(stream)))
    return out.value


def osscir_footprint_rays(h, l0, n, cap, cnt, idx, wt, stream=None):
    _check("osscir_footprint_rays", load().osscir_footprint_rays(
        ct.c_void_p(h), int(l0), int(n), int(cap), _ptr(cnt), _ptr(idx), _ptr(wt), _stream(stream)))


def osscir_footprint_pixels(h, k0, n, cap, cnt, idx, wt, stream=None):
    _check("osscir_footprint_pixels", load().osscir_footprint_pixels(
        ct.c_void_p(h), int(k0), int(n), int(cap), _ptr(cnt), _ptr(idx), _ptr(wt), _stream(stream)))


def osscir_mocca_partial(h, v0, v1, chan, stream=None):
    """Ray side of one iteration for the views [v0, v1); chan: contiguous float32 CUDA tensor [9, P]."""
    _check("osscir_mocca_partial", load().osscir_mocca_partial(ct.c_void_p(h), int(v0), int(v1), _ptr(chan),
                                                               _stream(stream)))


def osscir_mocca_apply(h, chan, stream=None):
    """Primal step of every pixel from the channels summed over all view ranges (chan [9, P])."""
    _check("osscir_mocca_apply", load().osscir_mocca_apply(ct.c_void_p(h), _ptr(chan), _stream(stream)))


def osscir_reconstruct(h, c_host, n_iters, maps_out_host, stream=None):
    """c_host [L, WS] and maps_out_host [P, 4]: contiguous float32 CPU tensors (pinned for DMA)."""
    if c_host.is_cuda or maps_out_host.is_cuda:
        raise ValueError("osscir_reconstruct takes host buffers")
    _check("osscir_reconstruct", load().osscir_reconstruct(ct.c_void_p(h), _ptr(c_host), int(n_iters),
                                                           _ptr(maps_out_host), _stream(stream)))


def osscir_last_kernel_ms(h, stream=None):
    """(projection, per-ray, back-projection) device ms of the last iteration."""
    ms = (ct.c_float * 3)()
    _check("osscir_last_kernel_ms", load().osscir_last_kernel_ms(ct.c_void_p(h), ms, _stream(stream)))
    return tuple(ms)


def osscir_dtpl_counts_static(chat, c, out, stream=None):
    """D_TPL of expected counts chat and measured counts c (device float32 [L, 4])
    into out (device float64 [1]) without allocating memory; see include/osscir.h."""
    import torch
    for name, t in (("chat", chat), ("c", c)):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 2 and t.shape[1] == 4):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape [L, 4]")
    if c.shape != chat.shape or c.device != chat.device:
        raise ValueError("chat and c must have the same shape and device")
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1 and out.device == chat.device):
        raise ValueError("out must be a float64 CUDA tensor with at least one element on the device of chat")
    _check("osscir_dtpl_counts_static", load().osscir_dtpl_counts_static(
        _ptr(chat), _ptr(c), int(chat.shape[0]), _ptr(out), _stream(stream)))


# --------------------------------------------------------------------------- served form

def osscir_server_create(hbm_budget_bytes, max_slots):
    h = ct.c_void_p()
    _check("osscir_server_create", load().osscir_server_create(int(hbm_budget_bytes), int(max_slots), ct.byref(h)))
    return h.value


def osscir_server_destroy(server):
    _check("osscir_server_destroy", load().osscir_server_destroy(ct.c_void_p(server)))


def osscir_submit(server, geom, s, N, mu, lam, counts, n_iters, model=0, box=None, spc=0, counts_model=0,
                  inner=1):
    """Host numpy arrays (copied by the call): s [n_bins, nE, 4], N [n_bins, 4], mu [3, nE],
    counts [L, 4].  Returns the ticket."""
    s32 = np.ascontiguousarray(s, dtype=np.float32)
    N32 = np.ascontiguousarray(N, dtype=np.float32)
    mu32 = np.ascontiguousarray(mu, dtype=np.float32)
    c32 = np.ascontiguousarray(counts, dtype=np.float32)
    fptr = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_float))
    req = Request(_geometry(geom), Spectra(int(s32.shape[1]), fptr(s32), fptr(N32), int(s32.shape[2])), fptr(mu32),
                  _params(lam, model, box, spc, counts_model, inner), fptr(c32), int(n_iters))
    t = ct.c_uint64()
    _check("osscir_submit", load().osscir_submit(ct.c_void_p(server), ct.byref(req), ct.byref(t)))
    return t.value


def osscir_poll(server, ticket, timeout_ms, maps_out=None):
    """maps_out: contiguous float32 numpy array [P, 4] or None.  Returns (status, Stats)."""
    st = Stats()
    ptr = None if maps_out is None else maps_out.ctypes.data_as(ct.c_void_p)
    rc = load().osscir_poll(ct.c_void_p(server), ct.c_uint64(ticket), int(timeout_ms), ptr, ct.byref(st))
    return rc, st


def osscir_server_info(server):
    r, q, b = ct.c_int(), ct.c_int(), ct.c_size_t()
    _check("osscir_server_info", load().osscir_server_info(ct.c_void_p(server), ct.byref(r), ct.byref(q),
                                                           ct.byref(b)))
    return r.value, q.value, b.value


# --------------------------------------------------------------------------- batched form

def osscir_batch_create(handles, autotune=False):
    """handles: context handles (ints) of the current device.  Returns the batch handle."""
    arr = (ct.c_void_p * len(handles))(*handles)
    b = ct.c_void_p()
    _check("osscir_batch_create", load().osscir_batch_create(arr, len(handles), int(bool(autotune)), ct.byref(b)))
    return b.value


def osscir_batch_destroy(batch):
    _check("osscir_batch_destroy", load().osscir_batch_destroy(ct.c_void_p(batch)))


def osscir_batch_step(batch, n_iters, stream=None):
    _check("osscir_batch_step", load().osscir_batch_step(ct.c_void_p(batch), int(n_iters), _stream(stream)))


def osscir_batch_get_config(batch):
    c = BatchConfig()
    _check("osscir_batch_get_config", load().osscir_batch_get_config(ct.c_void_p(batch), ct.byref(c)))
    return c.as_dict()


def osscir_batch_set_config(batch, cfg):
    """cfg: dict with the osscir_batch_config fields."""
    c = BatchConfig(**{k: int(v) for k, v in cfg.items()})
    _check("osscir_batch_set_config", load().osscir_batch_set_config(ct.c_void_p(batch), ct.byref(c)))


def osscir_batch_last_kernel_ms(batch, stream=None):
    ms = (ct.c_float * 3)()
    _check("osscir_batch_last_kernel_ms", load().osscir_batch_last_kernel_ms(ct.c_void_p(batch), ms,
                                                                             _stream(stream)))
    return tuple(ms)


def osscir_poisson_noise(chat, seed, out=None, stream=None):
    """Seeded Poisson draws of the expected counts chat (contiguous float32 CUDA tensor)
    into out (same shape, allocated if None); returns out."""
    import torch
    out = torch.empty_like(chat) if out is None else out
    if out.shape != chat.shape:
        raise ValueError("out must have the shape of chat")
    _check("osscir_poisson_noise", load().osscir_poisson_noise(_ptr(chat), int(chat.numel()), ct.c_uint64(int(seed)),
                                                               _ptr(out), _stream(stream)))
    return out
