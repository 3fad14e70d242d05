"""The seeded synthetic workloads follow the stated recipe of each configuration.

Sizes, view and bin counts, doses, energy grid, window layout, attenuation
curves (photoelectric E^-3 plus Klein-Nishina, the Gd K-edge jump), the
Kramers-like source and the phantoms' material levels, for the 64x64, 256x256
and 512x512 single solves, the 64-solve mixed batch and the 16-request mixed
served stream.  These are the inputs every parity test and benchmark draws
from, so a drifted generator would silently change what is measured.
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs


def test_energy_grid_and_windows():
    E = inputs.energies_keV()
    assert E[0] == 20.0 and E[-1] == 120.0 and E.size == 101 and np.all(np.diff(E) == 1.0)
    assert inputs.window_edges(4) == (20.0, 40.0, 50.0, 65.0, 120.0)
    assert inputs.window_edges(5) == (20.0, 40.0, 50.0, 65.0, 80.0, 120.0)
    R = inputs.window_responses(E, 16)
    # Gaussian roll-off of 5 keV: half height at an edge, inner edges jittered by at most 1 keV
    assert R.shape == (16, 101, 4)
    # the windows tile the grid wherever both outer edges (20, 120 keV) are 4 sigma away
    assert np.allclose(R.sum(axis=2)[:, 20:81], 1.0, atol=1e-4)
    i65 = int(np.where(E == 65.0)[0][0])
    assert np.all(np.abs(R[:, i65, 3] - 0.5) < 0.1)                   # 65 keV lies within 1 keV of the edge
    assert np.all(R[:, 0, 0] > R[:, 0, 1])                            # 20 keV belongs to the first window


def test_attenuation_curves():
    E = inputs.energies_keV()
    mu = inputs.mu_curves(E)
    assert mu.shape == (3, 101) and np.all(mu > 0.0)
    for m in range(3):   # monotone decrease away from the Gd K edge
        d = np.diff(mu[m])
        if m == 2:
            k = int(np.where(E >= inputs.GD_K_EDGE_KEV)[0][0])
            assert mu[2, k] > 3.0 * mu[2, k - 1]                      # the jump at 50.2 keV
            d = np.delete(d, k - 1)
        assert np.all(d < 0.0)
    # the photoelectric term scales as E^-3: without Compton, mu(60) / mu(30) = 1/8
    kn = inputs.klein_nishina_total(np.array([30.0, 60.0]))
    pe = (mu[1, 40] - inputs.MU_B["Al"] * kn[1] / kn[0]) / (mu[1, 10] - inputs.MU_B["Al"])
    assert pe == pytest.approx(1.0 / 8.0, rel=1e-12)


def test_source_spectrum_is_kramers_like():
    E = inputs.energies_keV()
    phi = inputs.source_spectrum(E)
    assert phi.sum() == pytest.approx(1.0) and phi[-1] == 0.0 and np.all(phi[:-1] > 0.0)
    sp = inputs.make_spectra(8, 1e5)
    assert np.allclose(sp.s.sum(axis=1), 1.0) and np.all(sp.s >= 0.0)
    assert np.allclose(sp.N.sum(axis=1), 1e5 * np.sum(phi[None, :, None] *
                                                      inputs.window_responses(E, 8), axis=(1, 2)))


def _check_ellipse_phantom(f, gd_levels):
    assert f.shape[1] == 3
    assert set(np.unique(np.round(f[:, 0], 6))) >= {0.0, 1.0}
    assert f[:, 1].max() == pytest.approx(1.0)                        # Al inserts replace PMMA
    assert f[:, 2].max() == pytest.approx(max(gd_levels))             # Gd at 0.1-2 % inside PMMA
    assert np.all(f[:, 2] <= 0.02 + 1e-12) and np.all(f >= 0.0)


@pytest.mark.parametrize("name,n,views,bins,photons,iters", [
    ("small_64", 64, 128, 128, 1e5, 200),
    ("medium_256", 256, 512, 512, 1e5, 500),
    ("large_512", 512, 1024, 1024, 1e6, 1000),
])
def test_named_workloads(name, n, views, bins, photons, iters):
    w = inputs.workload(name)
    g = w.geom
    assert (g.n, g.pixel_mm, g.n_views, g.n_bins) == (n, 0.5, views, bins)
    assert (g.sid_mm, g.sdd_mm, g.arc_deg) == (500.0, 1000.0, 360.0)
    assert w.photons_per_ray == photons and w.n_iters == iters and w.noise_seed is not None
    assert w.spectra.s.shape == (bins, 101, 4)
    if name == "small_64":   # PMMA disk of radius 14 mm, two Al and two Gd inserts (0.1 %, 1 %)
        assert w.f_true[:, 2].max() == pytest.approx(0.01)
        assert np.sum(w.f_true[:, 0] > 0.5) * 0.25 == pytest.approx(np.pi * 14.0**2, rel=0.05)
    else:
        _check_ellipse_phantom(w.f_true, (0.001, 0.002, 0.005, 0.01, 0.015, 0.02))


def test_batch_workloads_follow_the_mixed_batch_recipe():
    ws = inputs.batch_workloads(64)
    assert len(ws) == 64
    assert {w.geom.n for w in ws} == {128, 192, 256, 384, 512}
    assert all(90 <= w.geom.n_views <= 720 and w.geom.n_bins == w.geom.n_views for w in ws)
    assert all(1e4 <= w.photons_per_ray <= 1e6 for w in ws)
    assert len({w.noise_seed for w in ws}) == 64
    assert len({w.f_true.tobytes() for w in ws[:8]}) == 8            # phantoms of their own


def test_served_requests_follow_the_stream_recipe():
    rs = inputs.served_requests(16)
    assert len(rs) == 16
    assert {w.geom.n for w in rs} <= {128, 192, 256, 384, 512}
    assert all(90 <= w.geom.n_views <= 1024 and w.geom.n_bins == w.geom.n_views for w in rs)
    assert all(200 <= w.n_iters <= 500 for w in rs)
    assert all(1e4 <= w.photons_per_ray <= 1e6 for w in rs)
    again = inputs.served_requests(16)
    assert [w.n_iters for w in again] == [w.n_iters for w in rs]      # seeded
