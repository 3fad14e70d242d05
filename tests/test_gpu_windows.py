"""Window variants against the FP64 oracle (Sec. 1 contrasts the paper's four
overlapping realistic windows with an earlier simulation of five ideal ones):

  * four ideal windows (sharp edges, no overlap): 200 MOCCA iterations of small_64,
    per material within 1e-4 relative L2;
  * five windows (20-40-50-65-80-120 keV, ideal and overlapping), stored as
    float[L][8] per ray: the expected counts (padding zero), 200 iterations of
    small_64 within 1e-4 per material and D_TPL within 1e-5, the split of a solve
    by views, checkpoint/resume bit for bit, the host-buffer reconstruction
    bit-identical to the device path, and the forms that take four windows only
    (batched, served, nested) refusing five."""
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


# ---------------------------------------------------------------- five windows

def _five(geom, ideal=True):
    return inputs.make_spectra(geom.n_bins, 1e5, ideal_windows=ideal, n_windows=5)


def _f4(f):
    t = torch.zeros((f.shape[0], 4), dtype=torch.float32, device="cuda")
    t[:, :3] = torch.tensor(f, dtype=torch.float32, device="cuda")
    return t


@pytest.mark.parametrize("ideal", [True, False])
def test_five_window_counts_match_oracle(orc, ideal):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor
    geom = inputs.make_geometry(40, 0.5, 48, 56)
    sp = _five(geom, ideal)
    f = inputs.disk_phantom(geom, radius_mm=7.0, insert_mm=1.5).astype(np.float32)
    R = Reconstructor(geom, sp, 1e-7)
    assert (R.n_windows, R.window_stride) == (5, 8)
    got = R.simulate(_f4(f)).cpu().double().numpy()
    R.close()
    assert got.shape == (geom.n_rays, 8)
    want = orc.counts(geom, _sp32(sp), f.astype(np.float64))
    np.testing.assert_allclose(got[:, :5], want, rtol=1e-5)
    assert (got[:, 5:] == 0).all()


@pytest.mark.parametrize("ideal", [True, False])
def test_mocca_with_five_windows_matches_oracle(orc, ideal):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor
    w = inputs.workload("small_64")
    sp = _five(w.geom, ideal)
    s32 = _sp32(sp)
    c = inputs.poisson_counts(orc.counts(w.geom, s32, w.f_true), w.noise_seed)
    n_it, lam = 200, 1e-7
    R = Reconstructor(w.geom, sp, lam)
    R.set_counts(torch.tensor(c, dtype=torch.float32, device="cuda"))   # [L, 5], padded by the binding
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    d = R.dtpl(1)
    _, _, y, it = R.get_state()
    R.close()
    st, hist = orc.mocca(w.geom, s32, c.astype(np.float32).astype(np.float64), n_it, lam)
    rel = np.linalg.norm(x - st.x, axis=0) / np.linalg.norm(st.x, axis=0)
    tag = "ideal" if ideal else "overlapping"
    print(f"\nfive {tag} windows: rel L2 after {n_it} iterations PMMA {rel[0]:.2e} Al {rel[1]:.2e} Gd {rel[2]:.2e}")
    assert it == n_it
    assert np.all(rel < 1e-4), rel
    assert abs(d - hist[-1]) <= 1e-5 * hist[-1]
    y = y.cpu().double().numpy()
    assert (y[:, 5:] == 0).all()
    ry = np.linalg.norm(y[:, :5] - st.y) / np.linalg.norm(st.y)
    assert ry < 1e-4, ry


def test_five_window_checkpoint_split_and_host_path(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Reconstructor, _lib
    geom = inputs.make_geometry(48, 0.5, 64, 72)
    sp = _five(geom)
    f = inputs.disk_phantom(geom, radius_mm=8.0, insert_mm=1.8)
    lam = 1e-7
    A = Reconstructor(geom, sp, lam)
    c = _lib.osscir_poisson_noise(A.simulate(_f4(f)), 11)   # [L, 8]: the padding stays zero
    assert (c[:, 5:] == 0).all()
    A.set_counts(c)
    A.step(15)
    x, xbar, y, it = A.get_state()
    A.step(15)
    ref = A.maps().cpu().numpy()
    B = Reconstructor(geom, sp, lam)
    B.set_counts(c)
    B.set_state(x, xbar, y, it)
    B.step(15)
    assert np.array_equal(B.maps().cpu().numpy(), ref)
    # host buffers through osscir_reconstruct: the device path's result bit for bit
    ch = c.cpu().pin_memory()
    out = torch.zeros((geom.n_pixels, 4), dtype=torch.float32).pin_memory()
    _lib.osscir_reconstruct(B.handle, ch, 30, out)
    assert np.array_equal(out.numpy(), ref)
    # split by views: two halves, channels added, the primal step from the sum
    C = Reconstructor(geom, sp, lam)
    C.set_counts(c)
    P = geom.n_pixels
    for _ in range(30):
        chans = []
        for v0, v1 in ((0, geom.n_views // 2), (geom.n_views // 2, geom.n_views)):
            ch9 = torch.zeros((9, P), dtype=torch.float32, device="cuda")
            _lib.osscir_mocca_partial(C.handle, v0, v1, ch9)
            chans.append(ch9)
        _lib.osscir_mocca_apply(C.handle, chans[0] + chans[1])
    xs = C.maps().cpu().double().numpy()[:, :3]
    rel = np.linalg.norm(xs - ref[:, :3], axis=0) / np.linalg.norm(ref[:, :3], axis=0)
    assert np.all(rel < 1e-5), rel
    for R in (A, B, C):
        R.close()


def test_five_windows_are_refused_where_four_are_required():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_06263_gb300 import Batch, Reconstructor, _lib
    geom = inputs.make_geometry(16, 0.5, 16, 20)
    sp = _five(geom)
    R = Reconstructor(geom, sp, 1e-7)
    with pytest.raises(_lib.OsscirError) as e:
        Batch([R])
    assert e.value.status == _lib.OSSCIR_E_INVALID
    R.close()
    srv = _lib.osscir_server_create(1 << 30, 2)
    try:
        with pytest.raises(_lib.OsscirError) as e:
            _lib.osscir_submit(srv, geom, sp.s, sp.N, sp.mu, 1e-7, np.zeros((geom.n_rays, 8), np.float32), 5)
        assert e.value.status == _lib.OSSCIR_E_INVALID
    finally:
        _lib.osscir_server_destroy(srv)
