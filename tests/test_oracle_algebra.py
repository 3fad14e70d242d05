"""Pins for the oracle's small dense algebra: the 3x3 eigen-decomposition and
negative-curvature removal, the small linear solves, the per-ray dual step and
the per-pixel primal step (Sec. 2), against LAPACK (numpy) and scipy."""
import numpy as np
import pytest
import scipy.optimize


def _sym(rng, scales):
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return Q @ np.diag(scales) @ Q.T


CASES = [(1.0, 2.0, 3.0), (1e7, 1e2, 4.0), (5.0, 5.0, -1.0), (1e4, -3.0, 1e-3), (-2.0, -1.0, -1e-6),
         (0.0, 0.0, 0.0), (7.0, 7.0, 7.0)]


@pytest.mark.parametrize("scales", CASES)
def test_eig_sym3_matches_lapack(orc, scales):
    rng = np.random.default_rng(abs(hash(scales)) % 2**32)
    H = _sym(rng, scales)
    lam, V = orc.eig_sym3(H)
    nrm = max(np.abs(H).max(), 1e-300)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(H), rtol=0, atol=1e-13 * nrm + 1e-300)
    np.testing.assert_allclose(V @ np.diag(lam) @ V.T, H, rtol=0, atol=1e-13 * nrm + 1e-300)
    np.testing.assert_allclose(V.T @ V, np.eye(3), rtol=0, atol=1e-13)


@pytest.mark.parametrize("scales", CASES)
def test_clip_psd3(orc, scales):
    rng = np.random.default_rng(1 + abs(hash(scales)) % 2**32)
    H = _sym(rng, scales)
    Hp = orc.clip_psd3(H)
    w, V = np.linalg.eigh(H)
    want = V @ np.diag(np.maximum(w, 0)) @ V.T
    nrm = max(np.abs(H).max(), 1e-300)
    np.testing.assert_allclose(Hp, want, rtol=0, atol=1e-13 * nrm + 1e-300)
    assert np.linalg.eigvalsh(Hp).min() >= -1e-13 * nrm
    if min(scales) >= 0:
        np.testing.assert_allclose(Hp, H, rtol=0, atol=1e-13 * nrm + 1e-300)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_solve_matches_lapack(orc, n):
    rng = np.random.default_rng(n)
    M = rng.normal(size=(n, n)) + n * np.eye(n)
    b = rng.normal(size=n)
    np.testing.assert_allclose(orc.solve(M, b), np.linalg.solve(M, b), rtol=1e-13, atol=1e-13)


def _ray(rng, nw=4):
    alpha = np.abs(rng.normal(size=(nw, 3))) * np.array([0.03, 0.1, 20.0])
    H = _sym(rng, (3e4, 50.0, -0.5))
    r = rng.normal(scale=100.0, size=nw)
    sinv = rng.uniform(0.5, 5.0, size=nw)
    y = rng.normal(scale=50.0, size=nw)
    return alpha, H, r, sinv, y


@pytest.mark.parametrize("nw", [4, 5])
@pytest.mark.parametrize("seed", range(5))
def test_dual_step_is_the_prox_of_the_local_model(orc, seed, nw):
    """y' solves the optimality condition of the preconditioned dual prox of
    Q(z) = r^T (z - z0) + 1/2 (z - z0)^T W (z - z0):  y' = r + W Sigma^-1 (y - y')."""
    rng = np.random.default_rng(seed)
    alpha, H, r, sinv, y = _ray(rng, nw)
    Hp = orc.clip_psd3(H)
    yp = orc.dual_update(alpha, Hp, r, sinv, y)
    G = np.linalg.pinv(alpha)
    W = G.T @ Hp @ G
    step = sinv * (y - yp)
    resid = yp - r - W @ step
    # W is ill-conditioned (cond(alpha)^2): measure the residual on the scale of its terms
    scale = np.abs(r).max() + np.abs(yp).max() + np.abs(W).max() * np.abs(step).max()
    assert np.abs(resid).max() <= 1e-11 * scale


def test_dual_step_without_curvature_returns_residual(orc):
    rng = np.random.default_rng(7)
    alpha, H, r, sinv, y = _ray(rng)
    np.testing.assert_allclose(orc.dual_update(alpha, H, r, sinv, y, model="gradient"), r,
                               rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("nw", [4, 5])
@pytest.mark.parametrize("seed", range(3))
def test_separable_dual_step_is_the_windowwise_prox(orc, seed, nw):
    """W = diag(c) makes the W x W prox separable: y'_w = r_w + c_w / (c_w + sigma_w) (y_w - r_w),
    sigma_w = 1 / (Sigma^-1)_w, which the oracle's general solve must reproduce."""
    rng = np.random.default_rng(20 + seed)
    alpha, H, r, sinv, y = _ray(rng, nw)
    c = rng.uniform(10.0, 1e5, size=nw)
    yp = orc.dual_update(alpha, np.zeros((3, 3)), r, sinv, y, model="separable", c=c)
    sig = 1.0 / sinv
    np.testing.assert_allclose(yp, r + c / (c + sig) * (y - r), rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_dual_step_keeps_rays_outside_the_image(orc):
    rng = np.random.default_rng(8)
    alpha, H, r, sinv, y = _ray(rng)
    sinv[2] = 0.0
    np.testing.assert_array_equal(orc.dual_update(alpha, H, r, sinv, y), y)


@pytest.mark.parametrize("seed", range(4))
def test_primal_step_unconstrained(orc, seed):
    rng = np.random.default_rng(seed)
    T = _sym(rng, (1e3, 1.0, 1e-3))
    v = rng.normal(size=3)
    x = rng.normal(size=3)
    want = x - np.linalg.solve(T + 1e-12 * np.trace(T) * np.eye(3), v)
    # cond(T) = 1e6: both solves agree to cond * eps of the solution's scale
    np.testing.assert_allclose(orc.primal_update(T, v, x), want, rtol=0,
                               atol=1e-9 * np.abs(want).max())


def test_primal_step_unseen_pixel_keeps_x(orc):
    x = np.array([0.3, -0.1, 0.02])
    np.testing.assert_array_equal(orc.primal_update(np.zeros((3, 3)), np.ones(3), x), x)


BOXES = {
    "unit": (np.zeros(3), np.ones(3)),
    "nonnegative": (np.zeros(3), np.full(3, np.inf)),
    "half_open_mixed": (np.array([-np.inf, 0.0, -0.5]), np.array([0.5, np.inf, np.inf])),
}


@pytest.mark.parametrize("box", list(BOXES))
@pytest.mark.parametrize("seed", range(8))
def test_primal_step_box_matches_bounded_qp(orc, seed, box):
    rng = np.random.default_rng(100 + seed)
    T = _sym(rng, (50.0, 2.0, 0.1))
    v = rng.normal(scale=3.0, size=3)
    x = rng.uniform(0, 1, size=3)
    lo, hi = BOXES[box]
    got = orc.primal_update(T, v, x, box=(lo, hi))
    Tr = T + 1e-12 * np.trace(T) * np.eye(3)
    t = x - np.linalg.solve(Tr, v)
    obj = lambda z: 0.5 * (z - t) @ Tr @ (z - t)
    res = scipy.optimize.minimize(obj, np.clip(t, lo, hi), jac=lambda z: Tr @ (z - t),
                                  bounds=[(None if np.isinf(a) else a, None if np.isinf(b) else b)
                                          for a, b in zip(lo, hi)], method="L-BFGS-B",
                                  options=dict(ftol=1e-15, gtol=1e-12, maxiter=1000))
    assert (got >= lo).all() and (got <= hi).all()
    assert obj(got) <= obj(res.x) + 1e-10
    np.testing.assert_allclose(got, res.x, atol=1e-5)


@pytest.mark.parametrize("nw", [4, 5])
@pytest.mark.parametrize("seed", range(4))
def test_dual_step_in_an_orthonormal_basis_of_alpha(orc, seed, nw):
    """The identity the GPU's dual step is built on: with R the Cholesky factor of
    alpha^T alpha and Q = alpha R^-1, W = G^T H+ G = Q M Q^T with M = R^-T H+ R^-1,
    and the prox y' = y - Sigma (W + Sigma)^-1 (y - r) equals r + Q z with
    (I + M S) z = M Q^T Sigma^-1 (y - r), S = Q^T Sigma^-1 Q.  Written out here in
    FP64 and compared with the oracle's prox."""
    rng = np.random.default_rng(40 + seed)
    alpha, H, r, sinv, y = _ray(rng, nw)
    Hp = orc.clip_psd3(H)
    R = np.linalg.cholesky(alpha.T @ alpha).T
    Q = alpha @ np.linalg.inv(R)
    np.testing.assert_allclose(Q.T @ Q, np.eye(3), atol=1e-12)
    M = np.linalg.inv(R).T @ Hp @ np.linalg.inv(R)
    S = (Q.T * sinv) @ Q
    z = np.linalg.solve(np.eye(3) + M @ S, M @ (Q.T @ (sinv * (y - r))))
    want = orc.dual_update(alpha, Hp, r, sinv, y)
    # both sides are FP64 on a problem with cond(alpha^T alpha) up to ~1e7 (these alpha
    # scales): they agree to a few 1e-9 relative, the conditioning's share of FP64
    np.testing.assert_allclose(r + Q @ z, want, rtol=0, atol=1e-8 * np.abs(want).max())
    # M has the inertia of H (Sylvester's law), so a test on M picks the Hessians to clip
    M0 = np.linalg.inv(R).T @ H @ np.linalg.inv(R)
    assert (np.linalg.eigvalsh(M0) < 0).sum() == (np.linalg.eigvalsh(H) < 0).sum()
