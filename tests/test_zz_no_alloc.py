"""The allocation-free D_TPL entry point against the context-based one.

osscir_dtpl_counts_static serves callers that must not call cudaMalloc after
start-up (a memory arena that owns the device, or a loop that cannot accept the
synchronisation an allocation may cause).  It must give the same D_TPL as
osscir_dtpl evaluated at the same maps and counts, on two calls in a row (its
scratch array is reused between calls).  This file is collected last so that a
failure here stops a `-x` run only after every other test has run.
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_scratch_dtpl_matches_context_dtpl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor, _lib
    w = inputs.workload("small_64")
    R = Reconstructor(w.geom, w.spectra, 1e-7)
    f = torch.zeros((w.geom.n_pixels, 4), dtype=torch.float32, device="cuda")
    f[:, :3] = torch.tensor(w.f_true, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    c = torch.poisson(R.simulate(f), generator=gen).contiguous()
    # maps at which to evaluate: a perturbed truth, as solver state x_n
    x = (f * 0.97).contiguous()
    R.set_counts(c)
    R.set_state(x, x.clone(), torch.zeros_like(c), 0)
    ref = R.dtpl(0)                                   # context-based entry point
    chat = R.simulate(x)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):                                # two calls in a row share the scratch
        out.fill_(float("nan"))
        _lib.osscir_dtpl_counts_static(chat, c, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert np.isfinite(got)
        assert abs(got - ref) <= 1e-5 * abs(ref), (got, ref)
    R.close()


def test_static_scratch_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import _lib
    import ctypes as ct
    lib = _lib.load()
    dummy = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.osscir_dtpl_counts_static(ct.c_void_p(dummy.data_ptr()), ct.c_void_p(dummy.data_ptr()),
                                       4194305, ct.c_void_p(out.data_ptr()), None)
    assert st == _lib.OSSCIR_E_INVALID
