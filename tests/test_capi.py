"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a,
loads, exports every entry point include/osscir.h declares, and rejects invalid
arguments before touching the device."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_1801_06263_gb300 import _lib, inputs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "osscir.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(osscir_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.EXPORTS)


def test_status_strings(lib):
    assert _lib.load().osscir_status_string(0) == b"ok"
    assert _lib.load().osscir_status_string(-1) == b"invalid argument"


def _args():
    g = inputs.make_geometry(8, 0.5, 4, 6)
    sp = inputs.make_spectra(g.n_bins, 1e4)
    return g, sp


@pytest.mark.parametrize("mutate", [
    lambda g, sp: (g.__class__(**{**g.__dict__, "n": 0}), sp),
    lambda g, sp: (g.__class__(**{**g.__dict__, "sid_mm": 1.0}), sp),
    lambda g, sp: (g.__class__(**{**g.__dict__, "sdd_mm": 400.0}), sp),
    lambda g, sp: (g.__class__(**{**g.__dict__, "bin_mm": float("nan")}), sp),
    lambda g, sp: (g, inputs.Spectra(sp.energies, sp.s * 1.01, sp.N, sp.mu)),
    lambda g, sp: (g, inputs.Spectra(sp.energies, sp.s, -sp.N, sp.mu)),
    lambda g, sp: (g, inputs.Spectra(sp.energies, sp.s, sp.N, sp.mu * np.nan)),
])
def test_create_rejects_invalid_inputs(lib, mutate):
    g, sp = mutate(*_args())
    with pytest.raises(_lib.OsscirError) as e:
        _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6)
    assert e.value.status == _lib.OSSCIR_E_INVALID


@pytest.mark.parametrize("lam", [0.0, -1.0, float("inf"), float("nan")])
def test_create_rejects_bad_lambda(lib, lam):
    g, sp = _args()
    with pytest.raises(_lib.OsscirError) as e:
        _lib.osscir_create(g, sp.s, sp.N, sp.mu, lam)
    assert e.value.status == _lib.OSSCIR_E_INVALID


def test_create_rejects_bad_box_and_model(lib):
    g, sp = _args()
    with pytest.raises(_lib.OsscirError):
        _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6, counts_model=2)
    with pytest.raises(_lib.OsscirError):
        _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6, box=((0, 0, 1), (1, 1, 0)))
    inf, nan = float("inf"), float("nan")
    for box in (((0, 0, inf), (1, 1, inf)), ((0, 0, 0), (1, -inf, 1)), ((0, nan, 0), (1, 1, 1))):
        with pytest.raises(_lib.OsscirError):
            _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6, box=box)
    with pytest.raises(_lib.OsscirError):
        _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6, model=7)
    for inner in (-1, 1000001):   # iterations per kept local model of nested MOCCA
        with pytest.raises(_lib.OsscirError):
            _lib.osscir_create(g, sp.s, sp.N, sp.mu, 1e-6, inner=inner)


def test_create_rejects_unsupported_window_counts(lib):
    """Four or five windows; five are refused for nested solves (their kept models hold four)."""
    g, _ = _args()
    for nw in (3, 6):
        sp = inputs.make_spectra(g.n_bins, 1e4, n_windows=5)
        s = np.concatenate([sp.s] * 2, axis=2)[:, :, :nw] if nw > 5 else sp.s[:, :, :nw]
        N = np.concatenate([sp.N] * 2, axis=1)[:, :nw] if nw > 5 else sp.N[:, :nw]
        with pytest.raises(_lib.OsscirError) as e:
            _lib.osscir_create(g, s, N, sp.mu, 1e-6)
        assert e.value.status == _lib.OSSCIR_E_INVALID
    sp5 = inputs.make_spectra(g.n_bins, 1e4, n_windows=5)
    with pytest.raises(_lib.OsscirError) as e:
        _lib.osscir_create(g, sp5.s, sp5.N, sp5.mu, 1e-6, inner=3)
    assert e.value.status == _lib.OSSCIR_E_INVALID
    bad = sp5.s.copy()
    bad[:, :, 4] *= 1.01   # the fifth window's response must be normalised too
    with pytest.raises(_lib.OsscirError) as e:
        _lib.osscir_create(g, bad, sp5.N, sp5.mu, 1e-6)
    assert e.value.status == _lib.OSSCIR_E_INVALID
    with pytest.raises(ValueError):   # N must match s's window count
        _lib.osscir_create(g, sp5.s, sp5.N[:, :4], sp5.mu, 1e-6)


def test_null_handle_calls_are_rejected(lib):
    null = ct.c_void_p(0)
    assert lib.osscir_mocca_step(null, 1, None) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_forward(null, None, None, None) == _lib.OSSCIR_E_INVALID
    out = ct.c_double()
    assert lib.osscir_dtpl(null, 0, ct.byref(out), None) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_destroy(null) == _lib.OSSCIR_OK


def test_batch_calls_reject_invalid_arguments(lib):
    null = ct.c_void_p(0)
    out = ct.c_void_p()
    assert lib.osscir_batch_create(None, 1, 0, ct.byref(out)) == _lib.OSSCIR_E_INVALID
    arr = (ct.c_void_p * 2)(None, None)
    assert lib.osscir_batch_create(arr, 0, 0, ct.byref(out)) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_batch_create(arr, 2, 0, ct.byref(out)) == _lib.OSSCIR_E_INVALID
    # the same context twice: rejected before any device call
    fake = (ct.c_void_p * 2)(0x1000, 0x1000)
    assert lib.osscir_batch_create(fake, 2, 0, ct.byref(out)) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_batch_create(fake, 1, 2, ct.byref(out)) == _lib.OSSCIR_E_INVALID
    assert out.value is None
    assert lib.osscir_batch_step(null, 1, None) == _lib.OSSCIR_E_INVALID
    cfg = _lib.BatchConfig(4, 0, 0, 0, 0, 8, 0, 0, 1)
    assert lib.osscir_batch_get_config(null, ct.byref(cfg)) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_batch_set_config(null, ct.byref(cfg)) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_batch_destroy(null) == _lib.OSSCIR_OK


def test_poisson_noise_rejects_invalid_arguments(lib):
    assert lib.osscir_poisson_noise(None, -1, 0, None, None) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_poisson_noise(None, 4, 0, None, None) == _lib.OSSCIR_E_INVALID
    assert lib.osscir_poisson_noise(None, 0, 0, None, None) == _lib.OSSCIR_OK


# --------------------------------------------------------------------------- boundary checks on a GPU

def _small_context(lam):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = inputs.make_geometry(16, 0.5, 24, 20)
    sp = inputs.make_spectra(g.n_bins, 2e4)
    return torch, g, sp, _lib.osscir_create(g, sp.s, sp.N, sp.mu, lam)


@pytest.mark.gpu
@pytest.mark.parametrize("bad", [-1.0, float("nan"), float("inf")])
def test_reconstruct_rejects_invalid_host_counts(bad):
    torch, g, sp, h = _small_context(1e-6)
    try:
        c = torch.full((g.n_rays, 4), 100.0, dtype=torch.float32)
        c[g.n_rays // 2, 1] = bad
        out = torch.zeros((g.n_pixels, 4), dtype=torch.float32)
        with pytest.raises(_lib.OsscirError) as e:
            _lib.osscir_reconstruct(h, c, 5, out)
        assert e.value.status == _lib.OSSCIR_E_INVALID
        assert torch.all(out == 0)                     # nothing was run or copied back
    finally:
        _lib.osscir_destroy(h)


@pytest.mark.gpu
def test_set_counts_check_is_reported_by_dtpl():
    torch, g, sp, h = _small_context(1e-6)
    try:
        c = torch.full((g.n_rays, 4), 100.0, dtype=torch.float32, device="cuda")
        c[3, 2] = -5.0
        _lib.osscir_set_counts(h, c)
        with pytest.raises(_lib.OsscirError) as e:
            _lib.osscir_dtpl(h, 0)
        assert e.value.status == _lib.OSSCIR_E_INVALID
        c[3, 2] = 5.0                                   # valid counts clear the report
        _lib.osscir_set_counts(h, c)
        assert np.isfinite(_lib.osscir_dtpl(h, 0))
    finally:
        _lib.osscir_destroy(h)


@pytest.mark.gpu
def test_diverged_reconstruction_returns_diverged():
    # a step ratio far above the stable range (the 64 x 64 sweep diverges from 3e-7 on)
    torch, g, sp, h = _small_context(1.0)
    try:
        from paper_1801_06263_gb300 import Reconstructor  # noqa: F401  (loads the library)
        f = np.tile([[1.0, 0.05, 0.005]], (g.n_pixels, 1))
        f4 = torch.zeros((g.n_pixels, 4), dtype=torch.float32, device="cuda")
        f4[:, :3] = torch.tensor(f, dtype=torch.float32, device="cuda")
        chat = torch.zeros((g.n_rays, 4), dtype=torch.float32, device="cuda")
        _lib.osscir_simulate(h, f4, chat)
        c = chat.cpu().contiguous()
        out = torch.zeros((g.n_pixels, 4), dtype=torch.float32)
        with pytest.raises(_lib.OsscirError) as e:
            _lib.osscir_reconstruct(h, c, 200, out)
        assert e.value.status == _lib.OSSCIR_E_DIVERGED
    finally:
        _lib.osscir_destroy(h)


def test_static_dtpl_wrapper_rejects_mismatched_tensors():
    torch = pytest.importorskip("torch")
    a = torch.zeros((8, 4), dtype=torch.float32)
    out = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError):            # host tensors are not device buffers
        _lib.osscir_dtpl_counts_static(a, a, out)
    with pytest.raises(ValueError):            # [L, 3] is not the [L, 4] counts layout
        _lib.osscir_dtpl_counts_static(a[:, :3], a[:, :3], out)


def test_memory_query_rejects_null(lib):
    d, t = ct.c_size_t(), ct.c_size_t()
    assert lib.osscir_memory(ct.c_void_p(0), ct.byref(d), ct.byref(t)) == _lib.OSSCIR_E_INVALID


@pytest.mark.gpu
def test_footprint_tables_are_built_before_the_first_iteration():
    torch, g, sp, h = _small_context(1e-6)
    try:
        dev0, tab0 = _lib.osscir_memory(h)
        assert tab0 == 0 and dev0 > 0
        c = torch.full((g.n_rays, 4), 100.0, dtype=torch.float32, device="cuda")
        _lib.osscir_set_counts(h, c)
        _lib.osscir_mocca_step(h, 1)
        torch.cuda.synchronize()
        dev1, tab1 = _lib.osscir_memory(h)
        # at least the forward pairs: 8 bytes per footprint pair
        cnt = torch.zeros(g.n_rays, dtype=torch.int32, device="cuda")
        _lib.osscir_footprint_rays(h, 0, g.n_rays, 0, cnt, None, None)
        assert tab1 >= 8 * int(cnt.sum().item())
        assert dev1 == dev0 + tab1
    finally:
        _lib.osscir_destroy(h)
