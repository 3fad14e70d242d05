"""One-step three-material spectral CT reconstruction (MOCCA with m-block-diagonal
step-preconditioning, arXiv:1801.06263) on a GB300 GPU.

The compute path is the CUDA library libosscir.so (C-ABI in include/osscir.h);
``_lib`` mirrors its entry points one to one and ``Reconstructor`` holds one
context with its device tensors.  There is no CPU fallback.
"""
from __future__ import annotations

from . import inputs
from ._lib import (OsscirError, load, osscir_backproject, osscir_create, osscir_destroy, osscir_dtpl,
                   osscir_footprint_pixels, osscir_footprint_rays, osscir_forward, osscir_get_maps,
                   osscir_get_state, osscir_info, osscir_mocca_step, osscir_set_counts, osscir_set_state,
                   osscir_simulate, window_stride)

__all__ = ["inputs", "Reconstructor", "Batch", "OsscirError", "load"]


class Reconstructor:
    """One reconstruction context on the current CUDA device.

    Device arrays are torch float32 tensors: maps [P, 4] (PMMA, Al, Gd, unused),
    projections [L, 4] (four channels), per-ray window arrays (counts, dual)
    [L, WS] with WS = 4 for four windows and 8 for five (windows first, zero padding).
    """

    def __init__(self, geom, spectra, lam: float, *, model: int = 0, box=None, mu=None, spc: int = 0,
                 counts_model: int = 0, inner: int = 1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.geom = geom
        self.handle = osscir_create(geom, spectra.s, spectra.N, spectra.mu if mu is None else mu, lam,
                                    model=model, box=box, spc=spc, counts_model=counts_model,
                                    inner=inner)
        self.n_pixels, self.n_rays, self.n_fp64_pairs = osscir_info(self.handle)
        self.n_windows = int(spectra.s.shape[2])
        self.window_stride = window_stride(self.n_windows)

    # -- tensors
    def _new(self, rows):
        import torch
        return torch.zeros((rows, 4), dtype=torch.float32, device="cuda")

    def image(self):
        return self._new(self.n_pixels)

    def rays(self):
        return self._new(self.n_rays)

    def window_rays(self):
        import torch
        return torch.zeros((self.n_rays, self.window_stride), dtype=torch.float32, device="cuda")

    def _windows(self, c):
        """Counts [L, W] or [L, WS] as the library's [L, WS] layout (zero padding added)."""
        import torch
        if c.dim() == 2 and c.shape[1] == self.n_windows and self.n_windows != self.window_stride:
            out = torch.zeros((c.shape[0], self.window_stride), dtype=c.dtype, device=c.device)
            out[:, :self.n_windows] = c
            return out
        return c

    # -- operators
    def forward(self, x, out=None, stream=None):
        out = self.rays() if out is None else out
        osscir_forward(self.handle, x, out, stream)
        return out

    def backproject(self, rf, out=None, stream=None):
        out = self.image() if out is None else out
        osscir_backproject(self.handle, rf, out, stream)
        return out

    def simulate(self, f, out=None, stream=None):
        out = self.window_rays() if out is None else out
        osscir_simulate(self.handle, f, out, stream)
        return out

    # -- solver
    def set_counts(self, c, stream=None):
        c = self._windows(c)
        osscir_set_counts(self.handle, c, stream)
        self._counts = c   # the copy runs on the stream: keep a padded temporary alive until it has

    def step(self, n_iters: int, stream=None):
        osscir_mocca_step(self.handle, n_iters, stream)

    def maps(self, out=None, stream=None):
        out = self.image() if out is None else out
        osscir_get_maps(self.handle, out, stream)
        return out

    def dtpl(self, which: int = 0, stream=None) -> float:
        return osscir_dtpl(self.handle, which, stream)

    def get_state(self, stream=None):
        x, xbar, y = self.image(), self.image(), self.window_rays()
        it = osscir_get_state(self.handle, x, xbar, y, stream)
        return x, xbar, y, it

    def set_state(self, x, xbar, y, iteration, stream=None):
        osscir_set_state(self.handle, x, xbar, y, iteration, stream)

    def close(self):
        if getattr(self, "handle", None):
            osscir_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Reconstructors advanced together by the batched kernels (one launch
    per kernel per iteration for all of them).  The Reconstructors must stay open
    and must not be stepped on their own while the batch exists."""

    def __init__(self, recons, autotune: bool = False):
        from . import _lib
        self._lib = _lib
        self.recons = list(recons)
        self.handle = _lib.osscir_batch_create([r.handle for r in self.recons], autotune)

    def step(self, n_iters: int, stream=None):
        self._lib.osscir_batch_step(self.handle, n_iters, stream)

    @property
    def config(self):
        return self._lib.osscir_batch_get_config(self.handle)

    @config.setter
    def config(self, cfg):
        self._lib.osscir_batch_set_config(self.handle, cfg)

    def last_kernel_ms(self, stream=None):
        return self._lib.osscir_batch_last_kernel_ms(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            self._lib.osscir_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
