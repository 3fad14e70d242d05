"""GPU parity of the projector X, its adjoint and the counts model against the FP64 oracle.

  * footprints (which pixels each ray meets, which rays meet each pixel) are
    bit-exact against the oracle's Siddon traversal;
  * the forward and back-projection kernels use identical weights (the
    ray-driven and pixel-driven footprint dumps agree exactly);
  * FP32 projections agree with the FP64 oracle within 2e-6 relative, and the
    FP32 counts model of Eq. (finalModel) within 1e-5 relative; a pixel's
    back-projection may in addition carry the FP32 error of each weight it
    sums, bounded per ray by the bound the kernels use (see _weight_bound).
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEOMS = {
    "g8": inputs.make_geometry(8, 0.5, 12, 10),
    "g8_aligned": inputs.make_geometry(8, 0.5, 4, 9),
    # odd bin count: the central rays of the four axis views run along the x = 0 and
    # y = 0 grid lines, so every pixel they pass is decided by the FP64 table (~2n entries)
    "g64_aligned": inputs.make_geometry(64, 0.5, 8, 65),
    "g12_short": inputs.make_geometry(12, 0.3, 9, 20, sid_mm=100.0, sdd_mm=180.0, arc_deg=200.0,
                                      start_deg=17.0),
    "small_64": inputs.make_geometry(64, 0.5, 128, 128),
    "odd_37": inputs.make_geometry(37, 0.7, 45, 61, start_deg=90.0),
}


@pytest.fixture(scope="module")
def lib():
    from paper_1801_06263_gb300 import _lib
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _lib.load()


def _weight_bound(orc, geom, l):
    """Bound on |FP32 weight - exact weight| for any pixel of ray l: two plane
    parameters per chord, each within 2^-23 (R + |B|)(5.83 / |d_axis| + 4) (R the
    image circumradius, B the foot point).  Axis-parallel rays are decided
    entirely by the FP64 table, so only the rounding of the weight remains."""
    S, D = orc.ray_endpoints(geom, l // geom.n_bins, l % geom.n_bins)
    d = (D - S) / np.linalg.norm(D - S)
    if np.any(d == 0.0):
        return 2.0 ** -24 * geom.pixel_mm * np.sqrt(2.0)
    B = S - (S @ d) * d
    r_img = geom.n * geom.pixel_mm / np.sqrt(2.0)
    return 2.0 * max(2.0 ** -23 * (r_img + np.linalg.norm(B)) * (5.83 / abs(c) + 4.0) for c in d)


def _backprojection_slack(orc, geom, y):
    """Per pixel and channel: sum over its rays of |y_l| times ray l's weight bound."""
    out = np.zeros((geom.n_pixels, y.shape[1]))
    for l in range(geom.n_rays):
        pix, _ = orc.siddon(geom, l // geom.n_bins, l % geom.n_bins)
        out[pix] += np.abs(y[l]) * _weight_bound(orc, geom, l)
    return out


def _ctx(geom, spectra=None):
    from paper_1801_06263_gb300 import Reconstructor
    sp = spectra or inputs.make_spectra(geom.n_bins, 1e5)
    return Reconstructor(geom, sp, 1e-7)


def _ray_footprints(R, geom, cap):
    L = geom.n_rays
    cnt = torch.zeros(L, dtype=torch.int32, device="cuda")
    idx = torch.zeros((L, cap), dtype=torch.int32, device="cuda")
    wt = torch.zeros((L, cap), dtype=torch.float32, device="cuda")
    from paper_1801_06263_gb300 import osscir_footprint_rays
    osscir_footprint_rays(R.handle, 0, L, cap, cnt, idx, wt)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), idx.cpu().numpy(), wt.cpu().numpy()


def _pixel_footprints(R, geom, cap):
    P = geom.n_pixels
    cnt = torch.zeros(P, dtype=torch.int32, device="cuda")
    idx = torch.zeros((P, cap), dtype=torch.int32, device="cuda")
    wt = torch.zeros((P, cap), dtype=torch.float32, device="cuda")
    from paper_1801_06263_gb300 import osscir_footprint_pixels
    osscir_footprint_pixels(R.handle, 0, P, cap, cnt, idx, wt)
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), idx.cpu().numpy(), wt.cpu().numpy()


@pytest.mark.parametrize("name", list(GEOMS))
def test_footprint_bit_exact_and_weights(lib, orc, name):
    geom = GEOMS[name]
    R = _ctx(geom)
    cap = 2 * geom.n + 4
    cnt, idx, wt = _ray_footprints(R, geom, cap)
    for l in range(geom.n_rays):
        pix, ln = orc.siddon(geom, l // geom.n_bins, l % geom.n_bins)
        got = idx[l, :cnt[l]]
        assert cnt[l] == pix.size, (name, l)
        order = np.argsort(got)
        assert np.array_equal(got[order], np.sort(pix)), (name, l)
        want = ln[np.argsort(pix)]
        np.testing.assert_allclose(wt[l, :cnt[l]][order], want, rtol=0, atol=2e-4 * geom.pixel_mm)
    R.close()


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_and_adjoint_use_identical_weights(lib, name):
    geom = GEOMS[name]
    R = _ctx(geom)
    cap_r, cap_p = 2 * geom.n + 4, 8 * geom.n_views
    rc, ri, rw = _ray_footprints(R, geom, cap_r)
    pc, pi, pw = _pixel_footprints(R, geom, cap_p)
    assert pc.max() <= cap_p
    ray_pairs = {(l, int(k)): float(w) for l in range(geom.n_rays)
                 for k, w in zip(ri[l, :rc[l]], rw[l, :rc[l]])}
    pix_pairs = {(int(l), k): float(w) for k in range(geom.n_pixels)
                 for l, w in zip(pi[k, :pc[k]], pw[k, :pc[k]])}
    assert ray_pairs.keys() == pix_pairs.keys()
    assert all(ray_pairs[key] == pix_pairs[key] for key in ray_pairs)   # bitwise equal weights
    R.close()


@pytest.mark.parametrize("name", list(GEOMS))
def test_forward_backproject_match_oracle(lib, orc, name):
    geom = GEOMS[name]
    R = _ctx(geom)
    x, _ = inputs.random_state(geom, 5)
    x4 = np.concatenate([np.abs(x), np.ones((geom.n_pixels, 1))], axis=1)
    rng = np.random.default_rng(6)
    y4 = rng.uniform(0.0, 1.0, size=(geom.n_rays, 4))
    xt = torch.tensor(x4, dtype=torch.float32, device="cuda")
    yt = torch.tensor(y4, dtype=torch.float32, device="cuda")
    g = R.forward(xt).cpu().double().numpy()
    img = R.backproject(yt).cpu().double().numpy()
    torch.cuda.synchronize()
    g_ref = orc.forward(geom, x4.astype(np.float32).astype(np.float64))
    img_ref = orc.backproject(geom, y4.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(g, g_ref, rtol=2e-6, atol=2e-6 * np.abs(g_ref).max())
    slack = _backprojection_slack(orc, geom, y4)
    assert np.all(np.abs(img - img_ref) <= 2e-6 * np.abs(img_ref).max() + 2e-6 * np.abs(img_ref) + slack)
    # adjoint identity of the FP32 pair
    xs = rng.normal(size=(geom.n_pixels, 4))
    ys = rng.normal(size=(geom.n_rays, 4))
    gx = R.forward(torch.tensor(xs, dtype=torch.float32, device="cuda")).cpu().double().numpy()
    by = R.backproject(torch.tensor(ys, dtype=torch.float32, device="cuda")).cpu().double().numpy()
    lhs = float(np.sum(gx * ys.astype(np.float32)))
    rhs = float(np.sum(xs.astype(np.float32) * by))
    scale = float(np.sum(np.abs(gx) * np.abs(ys)))
    assert abs(lhs - rhs) <= 1e-6 * scale
    R.close()


@pytest.mark.parametrize("name", ["small_64", "odd_37"])
def test_counts_model_matches_oracle(lib, orc, name):
    geom = GEOMS[name]
    sp = inputs.make_spectra(geom.n_bins, 1e5)
    R = _ctx(geom, sp)
    f = inputs.disk_phantom(geom, radius_mm=0.45 * geom.n * geom.pixel_mm,
                            insert_mm=0.08 * geom.n * geom.pixel_mm)
    f4 = np.concatenate([f, np.zeros((geom.n_pixels, 1))], axis=1).astype(np.float32)
    chat = R.simulate(torch.tensor(f4, device="cuda")).cpu().double().numpy()
    # the oracle sees the library's FP32 copies of the inputs
    sp32 = inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                          sp.N.astype(np.float32).astype(np.float64),
                          sp.mu.astype(np.float32).astype(np.float64))
    ref = orc.counts(geom, sp32, f4[:, :3].astype(np.float64))
    np.testing.assert_allclose(chat, ref, rtol=1e-5, atol=0)
    R.close()
