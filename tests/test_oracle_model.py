"""Pins for the oracle's counts model, objective and derivatives (Sec. 2).

Ties Eq. (finalModel), Eq. (DTPL), the gradient Z^T A^T r and the per-ray
Hessian -Z^T diag(B^T r) Z + Z^T A^T diag(c^ + r) A Z to closed forms and to
central finite differences, and checks the sign facts the paper relies on
(sum_i s = 1, softexp'' <= softexp', A >= 0, C = A - B >= 0).
"""
import math

import numpy as np
import pytest

from paper_1801_06263_gb300 import inputs


@pytest.fixture(scope="module")
def spectra():
    return inputs.make_spectra(6, 1e5)


def test_spectral_response_is_normalised(spectra):
    np.testing.assert_allclose(spectra.s.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert (spectra.s >= 0).all() and (spectra.N > 0).all()


def test_zero_line_integrals_give_incident_counts(orc, spectra):
    for b in range(6):
        t = orc.ray_terms(spectra, b, np.zeros(3))
        np.testing.assert_allclose(t["chat"], spectra.N[b], rtol=1e-15, atol=0)


def _delta_spectra(nE, j):
    sp = inputs.make_spectra(2, 1e5)
    s = np.zeros_like(sp.s)
    s[:, j, :] = 1.0
    return inputs.Spectra(sp.energies, s, sp.N.copy(), sp.mu.copy())


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_delta_spectrum_closed_form(orc, sign):
    """One-hot s: c^_w = N_w softexp(-p_j) with p_j = mu_j . g (Eq. finalModel)."""
    j = 37
    sp = _delta_spectra(101, j)
    g = sign * np.array([3.0, 0.4, 0.01])
    p = float(sp.mu[:, j] @ g)
    t = orc.ray_terms(sp, 1, g)
    want = math.exp(-p) if p >= 0 else 1.0 - p
    np.testing.assert_allclose(t["chat"], sp.N[1] * want, rtol=1e-14)


def test_softexp_is_c1_at_zero(orc):
    """c^ is continuous with a continuous derivative where -p crosses 0."""
    j = 10
    sp = _delta_spectra(101, j)
    u = sp.mu[:, j] / np.linalg.norm(sp.mu[:, j])
    p_of = lambda t: float(sp.mu[:, j] @ (t * u))
    eps = 1e-7
    f = lambda t: orc.ray_terms(sp, 0, t * u)["chat"][0]
    left, mid, right = f(-eps), f(0.0), f(eps)
    assert abs(left - mid) < 1e-5 * mid and abs(right - mid) < 1e-5 * mid
    dl = (mid - f(-2 * eps)) / eps
    dr = (f(2 * eps) - mid) / eps
    assert abs(dl - dr) < 1e-4 * abs(dl)
    assert p_of(1.0) > 0


def test_A_and_C_nonnegative(orc, spectra):
    rng = np.random.default_rng(3)
    for _ in range(20):
        g = rng.normal(scale=5.0, size=3)
        t = orc.ray_terms(spectra, 2, g, with_AB=True)
        assert (t["A"] >= 0).all()
        assert (t["A"] - t["B"] >= -1e-300).all()


def test_dtpl_zero_at_data_and_positive_elsewhere(orc):
    c = np.array([10.0, 0.0, 3.5, 1e4])
    assert orc.dtpl(c, np.where(c > 0, c, 1e-300)) < 1e-12
    chat = np.array([12.0, 2.0, 3.0, 9e3])
    d = orc.dtpl(c, chat)
    want = sum((ch - cc - cc * math.log(ch / cc)) if cc > 0 else ch for ch, cc in zip(chat, c))
    assert abs(d - want) < 1e-12 * want and d > 0


def _tiny_problem(seed=5):
    geom = inputs.make_geometry(6, 0.8, 5, 8)
    sp = inputs.make_spectra(geom.n_bins, 2e4)
    f = inputs.disk_phantom(geom, radius_mm=2.0, insert_mm=0.6, gd_levels=(0.004, 0.008))
    rng = np.random.default_rng(seed)
    cbar_true = None
    return geom, sp, f, rng, cbar_true


def test_gradient_matches_finite_differences(orc):
    geom, sp, f_true, rng, _ = _tiny_problem()
    c = inputs.poisson_counts(orc.counts(geom, sp, f_true), 9)
    f = f_true + rng.normal(scale=0.05, size=f_true.shape) * np.array([1.0, 0.3, 0.002])
    d0, grad = orc.objective(geom, sp, c, f)
    fd = np.zeros_like(f)
    for k in range(geom.n_pixels):
        for m in range(3):
            h = 1e-6 * max(1.0, abs(f[k, m]))
            fp = f.copy(); fp[k, m] += h
            fm = f.copy(); fm[k, m] -= h
            fd[k, m] = (orc.objective(geom, sp, c, fp, with_grad=False)
                        - orc.objective(geom, sp, c, fm, with_grad=False)) / (2 * h)
    scale = np.abs(grad).max()
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ray_hessian_matches_finite_differences(orc, spectra, seed):
    """H = d(grad_g)/dg for one ray, with grad_g = alpha^T r (Sec. 2), in both
    softexp branches (negative g makes -p positive for some energies)."""
    rng = np.random.default_rng(seed)
    g = np.array([20.0, 1.0, 0.02]) * rng.uniform(-0.2, 1.0, size=3)
    c = spectra.N[3] * rng.uniform(0.05, 0.6, size=4)
    t = orc.ray_terms(spectra, 3, g, c)
    H = t["H"]
    fd = np.zeros((3, 3))
    for m in range(3):
        h = 1e-6 * max(1.0, abs(g[m]))
        gp = g.copy(); gp[m] += h
        gm = g.copy(); gm[m] -= h
        fd[:, m] = (orc.ray_terms(spectra, 3, gp, c)["grad"] - orc.ray_terms(spectra, 3, gm, c)["grad"]) / (2 * h)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())
    np.testing.assert_allclose(H, fd, rtol=0, atol=2e-6 * np.abs(H).max())


def test_ray_gradient_matches_dtpl_finite_difference(orc, spectra):
    rng = np.random.default_rng(8)
    g = np.array([15.0, 0.5, 0.01])
    c = spectra.N[4] * rng.uniform(0.1, 0.5, size=4)
    t = orc.ray_terms(spectra, 4, g, c)
    for m in range(3):
        h = 1e-6 * max(1.0, abs(g[m]))
        gp = g.copy(); gp[m] += h
        gm = g.copy(); gm[m] -= h
        dp = orc.dtpl(c, orc.ray_terms(spectra, 4, gp, c)["chat"])
        dm = orc.dtpl(c, orc.ray_terms(spectra, 4, gm, c)["chat"])
        assert abs((dp - dm) / (2 * h) - t["grad"][m]) <= 1e-6 * np.abs(t["grad"]).max()


# ---------------------------------------------------------------- the standard exp model (Eq. fullModel)

@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_exp_model_delta_spectrum_closed_form(orc, sign):
    """One-hot s: c^_w = N_w exp(-p_j) for either sign of p_j, and A = B = the one-hot
    response (exp' = exp'' = exp), so alpha_w = mu_j (Eq. fullModel, Eq. aeq)."""
    j = 37
    sp = _delta_spectra(101, j)
    g = sign * np.array([3.0, 0.4, 0.01])
    p = float(sp.mu[:, j] @ g)
    t = orc.ray_terms(sp, 1, g, with_AB=True, counts_model="exp")
    np.testing.assert_allclose(t["chat"], sp.N[1] * math.exp(-p), rtol=1e-14)
    np.testing.assert_allclose(t["alpha"], np.tile(sp.mu[:, j], (4, 1)), rtol=1e-14)
    np.testing.assert_allclose(t["A"], t["B"], rtol=0, atol=1e-15)


def test_models_agree_where_line_integrals_are_nonnegative(orc, spectra):
    """softexp(x) = exp(x) for x <= 0: with p_i >= 0 for every energy both models give
    the same counts, alpha and Hessian; with some p_i < 0 they differ."""
    g = np.array([12.0, 0.7, 0.01])
    c = spectra.N[2] * 0.3
    a = orc.ray_terms(spectra, 2, g, c)
    b = orc.ray_terms(spectra, 2, g, c, counts_model="exp")
    for k in ("chat", "alpha", "H"):
        np.testing.assert_array_equal(a[k], b[k])
    gn = -g
    a = orc.ray_terms(spectra, 2, gn, c)
    b = orc.ray_terms(spectra, 2, gn, c, counts_model="exp")
    assert np.all(b["chat"] > a["chat"])   # exp(x) > 1 + x for x > 0


@pytest.mark.parametrize("seed", [0, 1])
def test_exp_model_hessian_matches_finite_differences(orc, spectra, seed):
    """The per-ray Hessian -Z^T diag(B^T r) Z + Z^T A^T diag(c^ + r) A Z under exp, where
    B = A (so C = A - B = 0), against central differences of the gradient."""
    rng = np.random.default_rng(seed)
    g = np.array([20.0, 1.0, 0.02]) * rng.uniform(-0.2, 1.0, size=3)
    c = spectra.N[3] * rng.uniform(0.05, 0.6, size=4)
    t = orc.ray_terms(spectra, 3, g, c, with_AB=True, counts_model="exp")
    np.testing.assert_allclose(t["A"], t["B"], rtol=0, atol=1e-15)
    fd = np.zeros((3, 3))
    for m in range(3):
        h = 1e-6 * max(1.0, abs(g[m]))
        gp = g.copy(); gp[m] += h
        gm = g.copy(); gm[m] -= h
        fd[:, m] = (orc.ray_terms(spectra, 3, gp, c, counts_model="exp")["grad"]
                    - orc.ray_terms(spectra, 3, gm, c, counts_model="exp")["grad"]) / (2 * h)
    np.testing.assert_allclose(t["H"], fd, rtol=0, atol=2e-6 * np.abs(t["H"]).max())


def test_exp_model_gradient_matches_dtpl_finite_differences(orc):
    geom, sp, f_true, rng, _ = _tiny_problem()
    c = inputs.poisson_counts(orc.counts(geom, sp, f_true, counts_model="exp"), 9)
    f = f_true + rng.normal(scale=0.05, size=f_true.shape) * np.array([1.0, 0.3, 0.002])
    f[0] = -0.2   # a pixel with negative values, so that some p_i < 0
    d0, grad = orc.objective(geom, sp, c, f, counts_model="exp")
    fd = np.zeros_like(f)
    for k in range(geom.n_pixels):
        for m in range(3):
            h = 1e-6 * max(1.0, abs(f[k, m]))
            fp = f.copy(); fp[k, m] += h
            fm = f.copy(); fm[k, m] -= h
            fd[k, m] = (orc.objective(geom, sp, c, fp, with_grad=False, counts_model="exp")
                        - orc.objective(geom, sp, c, fm, with_grad=False, counts_model="exp")) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-6 * np.abs(grad).max())


# ---------------------------------------------------------------- ideal, non-overlapping windows

def test_ideal_windows_partition_the_energies():
    """Sharp windows: each energy lies in exactly one window, s sums to 1 per window."""
    R = inputs.window_responses(inputs.energies_keV(), 5, ideal=True)
    assert set(np.unique(R)) == {0.0, 1.0}
    assert (R.sum(axis=2) == 1.0).all()
    assert np.array_equal(R[0], R[4])   # the same response in every detector bin
    sp = inputs.make_spectra(5, 1e5, ideal_windows=True)
    assert ((sp.s > 0).sum(axis=2) <= 1).all()
    np.testing.assert_allclose(sp.s.sum(axis=1), 1.0, rtol=0, atol=1e-14)


def test_overlap_worsens_the_conditioning(orc):
    """The overlapping realistic windows make alpha^T alpha worse conditioned than
    ideal sharp windows on the same rays (the effect the paper attributes to the
    realistic response, Sec. 1)."""
    geom = inputs.make_geometry(32, 0.5, 16, 48)
    f = inputs.disk_phantom(geom, radius_mm=6.0, insert_mm=1.5)
    g = orc.forward(geom, f)
    real = inputs.make_spectra(geom.n_bins, 1e5)
    ideal = inputs.make_spectra(geom.n_bins, 1e5, ideal_windows=True)
    for l in (geom.n_bins // 2, 3 * geom.n_bins + 20, 9 * geom.n_bins + 30):
        b = l % geom.n_bins
        assert g[l, 0] > 0
        cond = [np.linalg.cond(orc.ray_terms(sp, b, g[l])["alpha"].T @ orc.ray_terms(sp, b, g[l])["alpha"])
                for sp in (real, ideal)]
        assert cond[0] > 1.2 * cond[1], cond


def test_five_ideal_windows_split_the_last_four_window_bin(orc):
    """Sharp windows are additive over disjoint energy ranges: with the same source
    and photons, the five-window layout equals the four-window one in the first
    three windows, and its last two windows (65-80 and 80-120 keV) add up to the
    four-window 65-120 keV window, for any maps (Eq. fullModel is linear in the
    per-energy photon flux)."""
    geom = inputs.make_geometry(12, 0.8, 8, 20)
    f = inputs.disk_phantom(geom, radius_mm=3.5, insert_mm=1.0)
    for counts_model in ("softexp", "exp"):
        c4 = orc.counts(geom, inputs.make_spectra(geom.n_bins, 1e5, ideal_windows=True), f,
                        counts_model=counts_model)
        c5 = orc.counts(geom, inputs.make_spectra(geom.n_bins, 1e5, ideal_windows=True, n_windows=5), f,
                        counts_model=counts_model)
        np.testing.assert_allclose(c5[:, :3], c4[:, :3], rtol=1e-13, atol=0)
        np.testing.assert_allclose(c5[:, 3] + c5[:, 4], c4[:, 3], rtol=1e-13, atol=0)
        assert (c5[:, 3] > 0).all() and (c5[:, 4] > 0).all()


def test_five_ideal_windows_partition_the_energies():
    R = inputs.window_responses(inputs.energies_keV(), 3, ideal=True, n_windows=5)
    assert R.shape[2] == 5 and (R.sum(axis=2) == 1.0).all()
    E = inputs.energies_keV()
    assert (R[0, (E >= 65) & (E < 80), 3] == 1).all() and (R[0, E >= 80, 4] == 1).all()
