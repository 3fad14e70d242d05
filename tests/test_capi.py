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
