"""Edge cases and the largest workload on the GPU, against the FP64 oracle.

  * degenerate sizes: one pixel, one view, one detector bin, ragged sizes that
    fill no tile or warp evenly;
  * rays that miss the image (their dual is kept, Sec. 2 reading) and pixels
    that no ray sees (they keep x);
  * all-zero counts (D_TPL terms reduce to c^, Eq. DTPL with 0 log 0 = 0);
  * large_512 (512 x 512, 1024 views x 1024 bins) at full size: footprints of
    200 sampled rays bit-exact against the oracle's Siddon traversal, their FP32
    weights within the kernels' error bound, simulated counts of 50 sampled
    rays within 1e-5 of the oracle's, and two iterations that stay finite.
    (The iterates at this size are compared with the oracle's over 100
    iterations in test_gpu_full_solve.py.)
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sp32(sp):
    return inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                          sp.N.astype(np.float32).astype(np.float64), sp.mu.astype(np.float32).astype(np.float64))


def _solve(geom, sp, c, lam, n_it):
    from paper_1801_06263_gb300 import Reconstructor
    R = Reconstructor(geom, sp, lam)
    R.set_counts(torch.tensor(np.ascontiguousarray(c, np.float32), device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    y = R.get_state()[2].cpu().double().numpy()
    d = R.dtpl(1)
    R.close()
    return x, y, d


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


GEOMS = [
    inputs.make_geometry(1, 2.0, 1, 1),                     # one pixel, one view, one bin
    inputs.make_geometry(3, 1.0, 1, 5),                     # one view
    inputs.make_geometry(5, 0.7, 7, 1),                     # one detector bin per view
    inputs.make_geometry(13, 0.6, 29, 33, start_deg=33.0),  # nothing is a multiple of a tile or warp
]


@pytest.mark.parametrize("gi", range(len(GEOMS)))
def test_degenerate_sizes_match_oracle(orc, gi):
    geom = GEOMS[gi]
    sp = inputs.make_spectra(geom.n_bins, 2e4)
    s32 = _sp32(sp)
    f = np.tile([[0.8, 0.1, 0.004]], (geom.n_pixels, 1))
    c = inputs.poisson_counts(orc.counts(geom, s32, f), 5).astype(np.float32)
    x, y, d = _solve(geom, sp, c, 1e-6, 20)
    st, hist = orc.mocca(geom, s32, c.astype(np.float64), 20, 1e-6)
    scale = np.abs(st.x).max(axis=0) + 1e-30
    assert (np.abs(x - st.x) <= 1e-4 * scale).all()
    assert abs(d - hist[-1]) <= 1e-5 * abs(hist[-1])


def test_rays_missing_the_image_keep_their_dual(orc):
    # a detector four times wider than needed: most rays miss the image
    geom = inputs.make_geometry(8, 0.5, 6, 40, bin_mm=4 * inputs.default_bin_mm(8, 0.5, 40))
    sp = inputs.make_spectra(geom.n_bins, 2e4)
    s32 = _sp32(sp)
    f = np.tile([[0.9, 0.0, 0.0]], (geom.n_pixels, 1))
    c = inputs.poisson_counts(orc.counts(geom, s32, f), 6).astype(np.float32)
    ones = orc.forward(geom, np.ones(geom.n_pixels))
    miss = ones == 0
    assert miss.sum() > geom.n_rays // 2
    x, y, _ = _solve(geom, sp, c, 1e-6, 10)
    assert np.all(y[miss] == 0.0)                 # y_0 = 0 is kept where Sigma^-1 = 0
    st, _ = orc.mocca(geom, s32, c.astype(np.float64), 10, 1e-6)
    assert np.all(st.y[miss] == 0.0)
    assert (np.abs(x - st.x) <= 1e-4 * (np.abs(st.x).max(axis=0) + 1e-30)).all()


def test_zero_counts(orc):
    geom = inputs.make_geometry(6, 0.8, 8, 10)
    sp = inputs.make_spectra(geom.n_bins, 2e4)
    s32 = _sp32(sp)
    c = np.zeros((geom.n_rays, 4), np.float32)
    x, y, d = _solve(geom, sp, c, 1e-6, 5)
    st, hist = orc.mocca(geom, s32, c.astype(np.float64), 5, 1e-6)
    assert np.isfinite(d) and abs(d - hist[-1]) <= 1e-5 * abs(hist[-1])
    assert (np.abs(x - st.x) <= 1e-4 * (np.abs(st.x).max(axis=0) + 1e-30)).all()


def test_large_512_full_size(orc):
    from paper_1801_06263_gb300 import Reconstructor, osscir_footprint_rays
    w = inputs.workload("large_512")
    R = Reconstructor(w.geom, w.spectra, 10 ** -8.5)
    assert R.n_rays == 1024 * 1024 and R.n_pixels == 512 * 512
    rng = np.random.default_rng(1)
    cap = 2 * w.geom.n + 4
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    idx = torch.zeros((1, cap), dtype=torch.int32, device="cuda")
    wt = torch.zeros((1, cap), dtype=torch.float32, device="cuda")
    r_img = w.geom.n * w.geom.pixel_mm / np.sqrt(2.0)
    for l in rng.choice(R.n_rays, size=200, replace=False):
        osscir_footprint_rays(R.handle, int(l), 1, cap, cnt, idx, wt)
        n = int(cnt.item())
        pix, ln = orc.siddon(w.geom, int(l) // w.geom.n_bins, int(l) % w.geom.n_bins)
        order = np.argsort(idx[0, :n].cpu().numpy())
        assert np.array_equal(idx[0, :n].cpu().numpy()[order], np.sort(pix))
        got = wt[0, :n].cpu().double().numpy()[order]
        want = ln[np.argsort(pix)]
        # each FP32 weight lies within the error bound the kernels use for this ray:
        # 2^-23 (R + |B|)(5.83 / |d_axis| + 4) per plane, two planes per chord
        S, D = orc.ray_endpoints(w.geom, int(l) // w.geom.n_bins, int(l) % w.geom.n_bins)
        d = (D - S) / np.linalg.norm(D - S)
        B = S - (S @ d) * d
        e = [2.0 ** -23 * (r_img + np.linalg.norm(B)) * (5.83 / abs(c) + 4.0) for c in d]
        assert np.all(np.abs(got - want) <= 2.0 * max(e))
        # telescoping: the sum carries the two end planes' errors and ~700 FP32 additions
        assert abs(got.sum() - want.sum()) <= 4e-6 * want.sum() + 2.0 * max(e)
    # simulated counts at full size against the oracle on sampled rays
    f4 = torch.zeros((R.n_pixels, 4), device="cuda")
    f4[:, :3] = torch.tensor(w.f_true, device="cuda")
    chat = R.simulate(f4).cpu().double().numpy()
    s32 = _sp32(w.spectra)
    for l in rng.choice(R.n_rays, size=50, replace=False):
        pix, ln = orc.siddon(w.geom, int(l) // w.geom.n_bins, int(l) % w.geom.n_bins)
        g = (ln[:, None] * w.f_true.astype(np.float32)[pix]).sum(axis=0)
        t = orc.ray_terms(s32, int(l) % w.geom.n_bins, g)
        np.testing.assert_allclose(chat[l], t["chat"], rtol=1e-5)
    # two MOCCA iterations at full size run and stay finite
    R.set_counts(torch.poisson(torch.tensor(chat, dtype=torch.float32, device="cuda")).contiguous())
    R.step(2)
    assert np.isfinite(R.dtpl(1))
    assert torch.isfinite(R.maps()).all()
    R.close()
