"""Pins for the oracle's MOCCA iteration with the m-block-diagonal SPC (Sec. 2).

  * one iteration equals an independent dense matrix-form restatement;
  * the step matrices satisfy the CPPD condition M = [[T^-1, -K^T], [-K, Sigma^-1]] >= 0;
  * the block SPC iterates are invariant under a rotation of the material
    basis, the diagonal SPC iterates are not (Sec. 2);
  * with monochromatic windows D_TPL is convex and MOCCA reaches the scipy minimiser;
  * noiseless data made with the reconstruction's own model (Sec. 3): D_TPL falls by > 1e8 and the maps
    approach the truth;
  * box constraints hold at every iterate; results do not depend on the thread count.
"""
import numpy as np
import pytest
import scipy.optimize

from paper_1801_06263_gb300 import inputs
import _dense


def _tiny(seed=0, n=5, views=4, bins=7, n_windows=4, ideal=False):
    geom = inputs.make_geometry(n, 0.9, views, bins, bin_mm=None)
    sp = inputs.make_spectra(geom.n_bins, 3e4, seed=seed + 3, n_windows=n_windows, ideal_windows=ideal)
    f = inputs.disk_phantom(geom, radius_mm=1.8, insert_mm=0.5, gd_levels=(0.005, 0.01))
    return geom, sp, f


def _random_state(geom, seed, nw=4):
    rng = np.random.default_rng(seed)
    x = np.abs(rng.normal(size=(geom.n_pixels, 3))) * np.array([0.8, 0.3, 0.004])
    xbar = x + rng.normal(size=x.shape) * np.array([0.05, 0.02, 0.0005])
    y = rng.normal(scale=200.0, size=(geom.n_rays, nw))
    return x, xbar, y


@pytest.mark.parametrize("spc,model,n_windows,ideal", [("block", "hessian", 4, False), ("block", "gradient", 4, False),
                                                       ("diagonal", "hessian", 4, False),
                                                       ("block", "hessian", 5, True), ("block", "hessian", 5, False),
                                                       ("diagonal", "hessian", 5, True)])
def test_one_iteration_matches_dense_restatement(orc, spc, model, n_windows, ideal):
    geom, sp, f = _tiny(n_windows=n_windows, ideal=ideal)
    c = inputs.poisson_counts(orc.counts(geom, sp, f), 4)
    x, xbar, y = _random_state(geom, 1, n_windows)
    X = _dense.dense_X(geom)
    lam = 3e-6
    want_x, want_xbar, want_y = _dense.one_iteration(geom, sp, X, c, x, xbar, y, lam, spc, model)
    st = orc.State(geom, n_windows)
    st.x[:], st.xbar[:], st.y[:] = x, xbar, y
    st, _ = orc.mocca(geom, sp, c, 1, lam, st, spc=spc, model=model)
    np.testing.assert_allclose(st.y, want_y, rtol=0, atol=1e-8 * np.abs(want_y).max())
    for m in range(3):
        sc = np.abs(want_x[:, m]).max()
        np.testing.assert_allclose(st.x[:, m], want_x[:, m], rtol=0, atol=1e-7 * sc)
        np.testing.assert_allclose(st.xbar[:, m], want_xbar[:, m], rtol=0, atol=1e-7 * sc)


@pytest.mark.parametrize("n_windows", [4, 5])
@pytest.mark.parametrize("spc", ["block", "diagonal"])
def test_step_condition_M_is_psd(orc, spc, n_windows):
    geom, sp, f = _tiny(1, n=6, views=5, bins=8, n_windows=n_windows, ideal=n_windows == 5)
    lam = 2.7e-4
    sinv, Tinv, alpha = orc.step_matrices(geom, sp, f, lam, spc=spc)
    X = _dense.dense_X(geom)
    L, P, nw = geom.n_rays, geom.n_pixels, n_windows
    K = np.zeros((nw * L, 3 * P))
    for w in range(nw):
        for m in range(3):
            K[w * L:(w + 1) * L, m * P:(m + 1) * P] = alpha[:, w, m][:, None] * X
    Ti = np.zeros((3 * P, 3 * P))
    for k in range(P):
        idx = [m * P + k for m in range(3)]
        Ti[np.ix_(idx, idx)] = Tinv[k]
    Si = np.diag(sinv.T.reshape(-1))
    M = np.block([[Ti, -K.T], [-K, Si]])
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1e-10 * np.abs(ev).max()
    if spc == "block":   # Sigma^-1 written out from its definition over the dense K
        want = lam * np.array([[np.sum(np.sqrt(sum(K[w * L + l, m * P:(m + 1) * P] ** 2 for m in range(3))))
                                for w in range(nw)] for l in range(L)])
        np.testing.assert_allclose(sinv, want, rtol=1e-12, atol=0)


def _rotation(seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return Q * np.sign(np.linalg.det(Q))


@pytest.mark.parametrize("spc,invariant", [("block", True), ("diagonal", False)])
def test_rotation_invariance(orc, spc, invariant):
    geom, sp, f = _tiny(2, n=6, views=6, bins=8)
    c = orc.counts(geom, sp, f)
    R = _rotation(5)
    mu_rot = R @ sp.mu                      # mu'_i = R mu_i  and  f' = R f keep Z f fixed
    lam = 1e-6
    st, _ = orc.mocca(geom, sp, c, 25, lam, spc=spc)
    st_r, _ = orc.mocca(geom, sp, c, 25, lam, spc=spc, mu=mu_rot)
    back = st_r.x @ R                       # R^T x'
    rel = np.linalg.norm(back - st.x) / np.linalg.norm(st.x)
    if invariant:
        assert rel < 1e-9, rel
    else:
        assert rel > 1e-3, rel


def test_convex_monochromatic_case_reaches_minimiser(orc):
    """One energy per window: c^_w = N_w softexp(-mu_w . g), so D_TPL is convex
    in f.  On a well-posed tiny problem (16 views, well-separated mu) MOCCA must
    reach the minimiser that scipy's BFGS finds from the truth."""
    geom = inputs.make_geometry(4, 1.0, 16, 12)
    base = inputs.make_spectra(geom.n_bins, 5e3)
    E = base.energies
    s = np.zeros_like(base.s)
    idx = [int(np.argmin(np.abs(E - e))) for e in (28.0, 45.0, 58.0, 85.0)]
    for w, i in enumerate(idx):
        s[:, i, w] = 1.0
    mu = np.zeros_like(base.mu)
    mu[:, idx] = [[0.30, 0.22, 0.18, 0.15], [0.60, 0.20, 0.10, 0.06], [0.20, 0.10, 0.60, 0.30]]
    sp = inputs.Spectra(E, s, base.N, mu)
    f_true = np.tile(np.array([[0.9, 0.4, 0.3]]), (geom.n_pixels, 1))
    c = inputs.poisson_counts(orc.counts(geom, sp, f_true), 21)
    fun = lambda v: orc.objective(geom, sp, c, v.reshape(-1, 3))
    res = scipy.optimize.minimize(lambda v: fun(v)[0], f_true.ravel(), jac=lambda v: fun(v)[1].ravel(),
                                  method="BFGS", options=dict(gtol=1e-10, maxiter=5000))
    d_star, g_star = fun(res.x)
    assert np.abs(g_star).max() < 1e-6          # stationary, hence the global minimiser
    f_star = res.x.reshape(-1, 3)
    st, hist = orc.mocca(geom, sp, c, 2000, 1e-3)
    d_mocca = orc.objective(geom, sp, c, st.x, with_grad=False)
    assert abs(d_mocca - d_star) <= 1e-10 * d_star
    assert np.linalg.norm(st.x - f_star) <= 1e-7 * np.linalg.norm(f_star)


@pytest.mark.parametrize("counts_model", ["softexp", "exp"])
def test_noiseless_inverse_crime_converges(orc, counts_model):
    w = inputs.workload("tiny_16")
    c = orc.counts(w.geom, w.spectra, w.f_true, counts_model=counts_model)
    st, hist = orc.mocca(w.geom, w.spectra, c, 3000, 1e-6, counts_model=counts_model)
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 1e-8 * hist[0]
    # after a burn-in the objective decreases (checked on a coarse grid)
    grid = hist[200::100]
    assert np.all(np.diff(grid) < 0)
    errs = [np.linalg.norm(st.x[:, m] - w.f_true[:, m]) / np.linalg.norm(w.f_true[:, m]) for m in range(3)]
    assert max(errs) < 0.06, errs
    # stationarity: the gradient Z^T A^T r shrinks by orders of magnitude
    _, g0 = orc.objective(w.geom, w.spectra, c, np.zeros_like(w.f_true), counts_model=counts_model)
    _, g1 = orc.objective(w.geom, w.spectra, c, st.x, counts_model=counts_model)
    assert np.linalg.norm(g1) < 1e-3 * np.linalg.norm(g0)


@pytest.mark.parametrize("lo,hi", [((0.0, 0.0, 0.0), (1.0, 0.8, 0.012)),
                                   ((0.0, 0.0, 0.0), (np.inf, np.inf, np.inf))])   # a box; nonnegativity
def test_box_constraint_holds_every_iteration(orc, lo, hi):
    geom, sp, f = _tiny(3, n=6, views=6, bins=8)
    c = inputs.poisson_counts(orc.counts(geom, sp, f), 8)
    st = None
    for _ in range(30):
        st, _ = orc.mocca(geom, sp, c, 1, 1e-6, st, box=(lo, hi))
        assert (st.x >= np.array(lo)).all() and (st.x <= np.array(hi)).all()


def test_thread_count_does_not_change_results(orc):
    w = inputs.workload("tiny_16")
    c = inputs.poisson_counts(orc.counts(w.geom, w.spectra, w.f_true), 3)
    n0 = orc.max_threads()
    try:
        orc.set_threads(1)
        a, ha = orc.mocca(w.geom, w.spectra, c, 20, 1e-6)
        orc.set_threads(4)
        b, hb = orc.mocca(w.geom, w.spectra, c, 20, 1e-6)
    finally:
        orc.set_threads(n0)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.y, b.y)
    np.testing.assert_array_equal(ha, hb)


# ---------------------------------------------------------------- nested (inner/outer) MOCCA

def _convex_case(orc):
    geom = inputs.make_geometry(4, 1.0, 16, 12)
    base = inputs.make_spectra(geom.n_bins, 5e3)
    E = base.energies
    s = np.zeros_like(base.s)
    idx = [int(np.argmin(np.abs(E - e))) for e in (28.0, 45.0, 58.0, 85.0)]
    for w, i in enumerate(idx):
        s[:, i, w] = 1.0
    mu = np.zeros_like(base.mu)
    mu[:, idx] = [[0.30, 0.22, 0.18, 0.15], [0.60, 0.20, 0.10, 0.06], [0.20, 0.10, 0.60, 0.30]]
    sp = inputs.Spectra(E, s, base.N, mu)
    f_true = np.tile(np.array([[0.9, 0.4, 0.3]]), (geom.n_pixels, 1))
    c = inputs.poisson_counts(orc.counts(geom, sp, f_true), 21)
    return geom, sp, f_true, c


@pytest.mark.parametrize("inner", [2, 5])
def test_nested_mocca_reaches_the_minimiser(orc, inner):
    """Nested MOCCA (a new local model every `inner` iterations) reaches the same
    convex D_TPL minimiser that scipy's BFGS finds from the truth."""
    geom, sp, f_true, c = _convex_case(orc)
    fun = lambda v: orc.objective(geom, sp, c, v.reshape(-1, 3))
    res = scipy.optimize.minimize(lambda v: fun(v)[0], f_true.ravel(), jac=lambda v: fun(v)[1].ravel(),
                                  method="BFGS", options=dict(gtol=1e-10, maxiter=5000))
    d_star = fun(res.x)[0]
    f_star = res.x.reshape(-1, 3)
    st, hist = orc.mocca(geom, sp, c, 2000, 1e-3, inner=inner)
    assert np.all(np.isfinite(hist))
    assert abs(orc.objective(geom, sp, c, st.x, with_grad=False) - d_star) <= 1e-10 * d_star
    assert np.linalg.norm(st.x - f_star) <= 1e-7 * np.linalg.norm(f_star)


def test_frozen_model_solves_the_local_quadratic(orc):
    """With a single outer iteration (inner = all iterations) the primal-dual steps
    minimise the local convex model built at f0 = 0: D(f0) + r^T K f + 1/2 f^T K^T W K f
    with the per-ray W = G^T H+ G, i.e. f = -(K^T W K)^-1 K^T r.  K, r and W come from
    the dense restatement (tests/_dense.py), not from the oracle."""
    geom, sp, f_true, c = _convex_case(orc)
    X = _dense.dense_X(geom)
    L, P, nE = geom.n_rays, geom.n_pixels, sp.s.shape[1]
    M = _dense.model_matrices(geom, sp, X, np.zeros((P, 3)), c)
    K, r, A, B = M["K"], M["r"], M["A"], M["B"]
    Btr = B.T @ r
    cvec = M["chat"] + r
    W = np.zeros((4 * L, 4 * L))
    for l in range(L):
        rows = [w * L + l for w in range(4)]
        if not np.any(X[l]):
            continue
        k0 = int(np.flatnonzero(X[l])[0])
        alpha = K[rows][:, [m * P + k0 for m in range(3)]] / X[l, k0]
        Zl = sp.mu.T
        seg = slice(l * nE, (l + 1) * nE)
        Al = A[rows][:, seg]
        H = -Zl.T @ np.diag(Btr[seg]) @ Zl + Zl.T @ Al.T @ np.diag(cvec[rows]) @ Al @ Zl
        lamH, V = np.linalg.eigh(H)
        G = np.linalg.pinv(alpha)
        W[np.ix_(rows, rows)] = G.T @ (V @ np.diag(np.maximum(lamH, 0)) @ V.T) @ G
    f_q = np.linalg.solve(K.T @ W @ K, -K.T @ r).reshape(3, P).T
    n = 2000
    st, _ = orc.mocca(geom, sp, c, n, 1e-3, inner=n)
    assert np.linalg.norm(st.x - f_q) <= 1e-8 * np.linalg.norm(f_q)


def test_inner_one_is_the_single_loop(orc):
    geom, sp, f = _tiny(2)
    c = inputs.poisson_counts(orc.counts(geom, sp, f), 4)
    a, ha = orc.mocca(geom, sp, c, 25, 1e-6)
    b, hb = orc.mocca(geom, sp, c, 25, 1e-6, inner=1)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and np.array_equal(ha, hb)


def test_gauss_newton_curvature_equals_the_hessian_at_zero_residual(orc):
    """The per-ray Hessian of Sec. 2 is sum_w c_w alpha_w alpha_w^T minus a term
    weighted by the residual r = c - c^; with noiseless counts at the expansion
    point (c = c^(f), xbar = f) that term vanishes, so one iteration with the
    Gauss-Newton curvature (model 2) equals one with the clipped Hessian
    (model 0, nothing to clip)."""
    from paper_1801_06263_gb300 import inputs
    geom = inputs.make_geometry(12, 0.5, 16, 14)
    sp = inputs.make_spectra(geom.n_bins, 1e4)
    f = inputs.disk_phantom(geom, radius_mm=2.5, insert_mm=0.6)
    c = orc.counts(geom, sp, f)
    y0 = np.random.default_rng(4).normal(scale=30.0, size=(geom.n_rays, 4))   # W acts on y - r = y
    out = []
    for model in ("hessian", "gauss_newton", "gradient"):
        st = orc.State(geom)
        st.x[:] = f
        st.xbar[:] = f
        st.y[:] = y0
        st, _ = orc.mocca(geom, sp, c, 1, 1e-6, st, model=model)
        out.append((st.x.copy(), st.y.copy()))
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-9, atol=1e-9 * np.abs(out[0][1]).max())
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-9, atol=1e-9 * np.abs(out[0][0]).max())
    # and the curvature does act here: without it (W = 0) the step is different
    assert np.abs(out[2][1] - out[0][1]).max() > 1e-3 * np.abs(out[0][1]).max()


def test_five_ideal_windows_converge(orc):
    """The ideal five-window response (Sec. 1: the earlier one-step simulation
    that converged readily) on noiseless data made with the model itself: D_TPL
    falls by more than 1e8 and the maps approach the truth."""
    w = inputs.workload("tiny_16")
    sp = inputs.make_spectra(w.geom.n_bins, 1e5, ideal_windows=True, n_windows=5)
    c = orc.counts(w.geom, sp, w.f_true)
    assert c.shape == (w.geom.n_rays, 5)
    st, hist = orc.mocca(w.geom, sp, c, 2000, 3e-6)   # a step ratio at which four windows diverge here
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 1e-8 * hist[0]
    errs = [np.linalg.norm(st.x[:, m] - w.f_true[:, m]) / np.linalg.norm(w.f_true[:, m]) for m in range(3)]
    assert max(errs) < 0.06, errs
