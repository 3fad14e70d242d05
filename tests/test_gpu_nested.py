"""GPU parity of nested (inner/outer) MOCCA against the FP64 oracle.

The nested form (Sec. 3 mentions it and sets it aside for the single loop)
builds each ray's local convex model in an outer iteration and keeps it for
the next inner - 1 iterations, which are primal-dual steps on that fixed model:
the dual prox at u = y + Sigma alpha (X xbar - g0), with the stored alpha in K
and in the step matrix T.  The oracle takes the same steps in FP64 from the
stored Hessian; the GPU keeps the prox as its 4 x 4 linear map.  Tolerances
are those of the single-loop parity tests (1e-4 relative L2 per material after
many iterations; 2e-5 of the largest entry after one outer and one inner step).
"""
import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_L2 = 1e-4


def _sp32(sp):
    return inputs.Spectra(sp.energies, sp.s.astype(np.float32).astype(np.float64),
                          sp.N.astype(np.float32).astype(np.float64),
                          sp.mu.astype(np.float32).astype(np.float64))


def _rel(a, b):
    return [float(np.linalg.norm(a[:, m] - b[:, m]) / np.linalg.norm(b[:, m])) for m in range(3)]


@pytest.fixture(scope="module")
def small(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = inputs.workload("small_64")
    s32 = _sp32(w.spectra)
    c = inputs.poisson_counts(orc.counts(w.geom, s32, w.f_true), w.noise_seed).astype(np.float32)
    return w, s32, c


def _recon(geom, sp, lam, **kw):
    from paper_1801_06263_gb300 import Reconstructor
    return Reconstructor(geom, sp, lam, **kw)


@pytest.mark.parametrize("inner", [2, 4])
def test_one_outer_and_inner_steps_from_random_state(orc, inner):
    """inner iterations from a random state (one outer, inner - 1 inner): duals and
    maps element by element against the oracle."""
    geom = inputs.make_geometry(20, 0.6, 24, 30)
    sp = inputs.make_spectra(geom.n_bins, 5e4)
    s32 = _sp32(sp)
    f = inputs.disk_phantom(geom, radius_mm=5.0, insert_mm=1.0)
    c = inputs.poisson_counts(orc.counts(geom, s32, f), 3).astype(np.float32)
    rng = np.random.default_rng(40 + inner)
    x = (f + rng.normal(scale=0.05, size=f.shape) * np.array([1.0, 0.3, 0.003])).astype(np.float32)
    xbar = (x + rng.normal(scale=0.02, size=f.shape) * np.array([1.0, 0.3, 0.003])).astype(np.float32)
    y = rng.normal(scale=300.0, size=(geom.n_rays, 4)).astype(np.float32)
    lam = 3e-7
    R = _recon(geom, sp, lam, inner=inner)
    pad = lambda a: torch.tensor(np.concatenate([a, np.zeros((a.shape[0], 1), np.float32)], 1), device="cuda")
    R.set_counts(torch.tensor(c, device="cuda"))
    R.set_state(pad(x), pad(xbar), torch.tensor(y, device="cuda"), 0)
    R.step(inner)
    gx, _, gy, it = R.get_state()
    d1 = R.dtpl(1)
    R.close()
    st = orc.State(geom)
    st.x[:], st.xbar[:], st.y[:] = x, xbar, y
    st, hist = orc.mocca(geom, s32, c.astype(np.float64), inner, lam, st, inner=inner)
    gy = gy.cpu().double().numpy()
    np.testing.assert_allclose(gy, st.y, rtol=0, atol=2e-5 * np.abs(st.y).max())
    gx = gx.cpu().double().numpy()[:, :3]
    for m in range(3):
        np.testing.assert_allclose(gx[:, m], st.x[:, m], rtol=0, atol=2e-5 * np.abs(st.x[:, m]).max())
    # D_TPL of the last outer iteration (the only one in this call)
    assert abs(d1 - hist[0]) <= 1e-5 * hist[0]
    assert it == inner


@pytest.mark.parametrize("inner", [2, 4])
def test_small_64_nested_iterates_match_oracle(orc, small, inner):
    w, s32, c = small
    lam, n_it = 1e-7, 120
    R = _recon(w.geom, w.spectra, lam, inner=inner)
    R.set_counts(torch.tensor(c, device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    d_gpu = R.dtpl(1)
    R.close()
    st, hist = orc.mocca(w.geom, s32, c.astype(np.float64), n_it, lam, inner=inner)
    errs = _rel(x, st.x)
    print(f"inner={inner}: rel L2 after {n_it} iterations PMMA {errs[0]:.2e} Al {errs[1]:.2e} Gd {errs[2]:.2e}")
    assert max(errs) < REL_L2, errs
    last_outer = (n_it - 1) // inner * inner
    assert abs(d_gpu - hist[last_outer]) <= 1e-5 * hist[last_outer]


def test_cycle_continues_across_calls_and_restarts_on_resume(orc, small):
    """step(3) + step(5) is step(8) bit for bit (the cycle runs on across calls);
    after set_state the next iteration is an outer one, as in a new oracle call."""
    w, s32, c = small
    lam, inner = 1e-7, 4
    ct_ = torch.tensor(c, device="cuda")
    A = _recon(w.geom, w.spectra, lam, inner=inner)
    A.set_counts(ct_)
    A.step(8)
    xa = A.maps().cpu().numpy()
    A.set_counts(ct_)
    A.step(3)
    A.step(5)
    assert np.array_equal(A.maps().cpu().numpy(), xa)
    # resume: 6 iterations, save, restore into another context, 6 more
    A.set_counts(ct_)
    A.step(6)
    x, xbar, y, it = A.get_state()
    A.close()
    B = _recon(w.geom, w.spectra, lam, inner=inner)
    B.set_counts(ct_)
    B.set_state(x, xbar, y, it)
    B.step(6)
    xb = B.maps().cpu().double().numpy()[:, :3]
    B.close()
    st, _ = orc.mocca(w.geom, s32, c.astype(np.float64), 6, lam, inner=inner)
    st, _ = orc.mocca(w.geom, s32, c.astype(np.float64), 6, lam, st, inner=inner)
    assert max(_rel(xb, st.x)) < REL_L2


def test_inner_one_is_the_single_loop(small):
    w, _, c = small
    ct_ = torch.tensor(c, device="cuda")
    out = []
    for kw in ({}, {"inner": 1}, {"inner": 0}):
        R = _recon(w.geom, w.spectra, 1e-7, **kw)
        R.set_counts(ct_)
        R.step(12)
        out.append(R.maps().cpu().numpy())
        R.close()
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_nested_solves_are_neither_batched_nor_served(small):
    from paper_1801_06263_gb300 import Batch, OsscirError, _lib as L
    w, _, c = small
    R = _recon(w.geom, w.spectra, 1e-7, inner=3)
    with pytest.raises(OsscirError) as e:
        Batch([R])
    assert e.value.status == L.OSSCIR_E_INVALID
    R.close()
    srv = L.osscir_server_create(1 << 30, 1)
    try:
        sp = w.spectra
        with pytest.raises(OsscirError) as e:
            L.osscir_submit(srv, w.geom, sp.s, sp.N, sp.mu, 1e-7, c, 10, inner=3)
        assert e.value.status == L.OSSCIR_E_INVALID
    finally:
        L.osscir_server_destroy(srv)


@pytest.mark.parametrize("variant", ["gradient", "nonnegative", "diagonal"])
def test_nested_variants_match_oracle(orc, small, variant):
    """Nested MOCCA with the zero-curvature model (inner = 3, an iteration count
    that is not a multiple of it), with nonnegativity (inner = 4) and with the
    diagonal SPC (inner = 2), against the oracle's nested iterates."""
    w, s32, c = small
    inf = float("inf")
    gpu_kw, orc_kw, lam, n_it, inner = {
        "gradient": ({"model": 1}, {"model": "gradient"}, 3e-8, 61, 3),
        "nonnegative": ({"box": ((0.0, 0.0, 0.0), (inf, inf, inf))},
                        {"box": ((0.0, 0.0, 0.0), (inf, inf, inf))}, 1e-7, 60, 4),
        "diagonal": ({"spc": 1}, {"spc": "diagonal"}, 1e-6, 30, 2),
    }[variant]
    R = _recon(w.geom, w.spectra, lam, inner=inner, **gpu_kw)
    R.set_counts(torch.tensor(c, device="cuda"))
    R.step(n_it)
    x = R.maps().cpu().double().numpy()[:, :3]
    R.close()
    st, _ = orc.mocca(w.geom, s32, c.astype(np.float64), n_it, lam, inner=inner, **orc_kw)
    errs = _rel(x, st.x)
    print(f"nested {variant}: rel L2 after {n_it} iterations PMMA {errs[0]:.2e} Al {errs[1]:.2e} Gd {errs[2]:.2e}")
    assert max(errs) < REL_L2, errs
