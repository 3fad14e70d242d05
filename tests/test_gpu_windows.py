"""Ideal, non-overlapping photon-counting windows (sharp edges, no overlap: the
response the paper contrasts with its realistic overlapping windows, Sec. 1)
as a spectral variant of the same four-window layout: 200 MOCCA iterations of
small_64 against the FP64 oracle, per material within 1e-4 relative L2."""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sp32(sp):
    return inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                          sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))


def test_mocca_with_ideal_windows_matches_oracle(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor
    w = inputs.workload("small_64")
    sp = inputs.make_spectra(w.geom.n_bins, 1e5, ideal_windows=True)
    s32 = _sp32(sp)
    c = inputs.poisson_counts(orc.counts(w.geom, s32, w.f_true), w.noise_seed)
    n_it, lam = 200, 1e-7
    R = Reconstructor(w.geom, sp, lam)
    R.set_counts(torch.tensor(c, dtype=torch.float32, device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    d = R.dtpl(1)
    R.close()
    st, hist = orc.mocca(w.geom, s32, c.astype(np.float32).astype(np.float64), n_it, lam)
    rel = np.linalg.norm(x - st.x, axis=0) / np.linalg.norm(st.x, axis=0)
    print(f"\nideal windows: rel L2 after {n_it} iterations PMMA {rel[0]:.2e} Al {rel[1]:.2e} Gd {rel[2]:.2e}")
    assert np.all(rel < 1e-4), rel
    assert abs(d - hist[-1]) <= 1e-5 * hist[-1]
