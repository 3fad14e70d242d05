"""Pins for the oracle's mu-PC basis change (Sec. 1 and 2): orthonormal
transformed curves, unchanged line integrals, an exact round trip of the maps,
and the same counts model in the transformed basis."""
import numpy as np

from paper_1801_06263_gb300 import inputs


def test_mu_pc_orthonormal_and_invariant(orc):
    sp = inputs.make_spectra(8, 1e4)
    mu_t, M = orc.mu_pc(sp.mu)
    np.testing.assert_allclose(mu_t @ mu_t.T, np.eye(3), atol=1e-10)   # cond(mu mu^T) ~ 1e6
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
    np.testing.assert_allclose(M @ M @ (sp.mu @ sp.mu.T), np.eye(3), atol=1e-8)   # M^2 = (mu mu^T)^-1
    rng = np.random.default_rng(0)
    f = rng.normal(size=(50, 3))
    f_t = orc.maps_to_basis(f, M)
    np.testing.assert_allclose(f_t @ mu_t, f @ sp.mu, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(orc.maps_from_basis(f_t, M), f, rtol=1e-12, atol=1e-12)
    # the transformed problem has the same counts model (Eq. finalModel)
    geom = inputs.make_geometry(6, 0.8, 5, 8)
    sp8 = inputs.make_spectra(geom.n_bins, 1e4)
    mu_t8, M8 = orc.mu_pc(sp8.mu)
    f8 = np.abs(rng.normal(size=(geom.n_pixels, 3))) * np.array([0.5, 0.1, 0.002])
    a = orc.counts(geom, sp8, f8)
    b = orc.counts(geom, sp8, orc.maps_to_basis(f8, M8), mu=mu_t8)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_mu_pc_of_orthonormal_curves_is_identity(orc):
    # curves that are already orthonormal need no change of basis
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(40, 3)))
    mu_t, M = orc.mu_pc(Q.T)
    np.testing.assert_allclose(M, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(mu_t, Q.T, atol=1e-12)


def test_weighted_mu_pc_is_orthonormal_in_its_inner_product(orc):
    sp = inputs.make_spectra(8, 1e4)
    phi = np.linspace(1.0, 3.0, sp.mu.shape[1])
    mu_t, M = orc.mu_pc(sp.mu, weights=phi)
    np.testing.assert_allclose((mu_t * phi) @ mu_t.T, np.eye(3), atol=1e-10)
    np.testing.assert_allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())
