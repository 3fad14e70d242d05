"""Dense, matrix-form restatement of one MOCCA iteration for tiny problems.

Independent of the oracle (no shared code): it builds X by clipping every ray
against every pixel, forms Z, A(f0), B(f0) and K(f0) = A Z as the dense
matrices of Sec. 2, and takes the step with numpy's linear algebra.  The tests
compare the oracle's per-ray loops against it.
"""
import math

import numpy as np


def ray_endpoints(geom, v, b):
    th = math.radians(geom.start_deg + v * geom.arc_deg / geom.n_views)
    c, s = math.cos(th), math.sin(th)
    u = (b - 0.5 * (geom.n_bins - 1)) * geom.bin_mm
    S = np.array([geom.sid_mm * c, geom.sid_mm * s])
    D = np.array([(geom.sid_mm - geom.sdd_mm) * c - u * s, (geom.sid_mm - geom.sdd_mm) * s + u * c])
    return S, D


def dense_X(geom):
    """X[l, k]: length of ray l inside pixel k (clip; lengths <= 1e-9 h dropped)."""
    n, h = geom.n, geom.pixel_mm
    x0 = -0.5 * n * h
    edges = x0 + np.arange(n + 1) * h
    X = np.zeros((geom.n_rays, n * n))
    for l in range(geom.n_rays):
        S, D = ray_endpoints(geom, l // geom.n_bins, l % geom.n_bins)
        d = D - S
        nrm = float(np.hypot(*d))
        for iy in range(n):
            for ix in range(n):
                t0, t1, ok = 0.0, 1.0, True
                for a, (lo, hi) in enumerate(((edges[ix], edges[ix + 1]), (edges[iy], edges[iy + 1]))):
                    if d[a] == 0.0:
                        ok &= lo <= S[a] < hi
                        continue
                    ta, tb = (lo - S[a]) / d[a], (hi - S[a]) / d[a]
                    t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
                ln = (t1 - t0) * nrm
                if ok and ln > 1e-9 * h:
                    X[l, iy * n + ix] = ln
    return X


def sexp(x, order):
    if order == 0:
        return np.where(x <= 0, np.exp(np.minimum(x, 0)), x + 1.0)
    if order == 1:
        return np.where(x <= 0, np.exp(np.minimum(x, 0)), 1.0)
    return np.where(x <= 0, np.exp(np.minimum(x, 0)), 0.0)


def model_matrices(geom, sp, X, f0, c):
    """Dense Z, A, B, K, c^, r at the expansion point f0 ([P,3]).

    Row index of data space: w * L + l;  column index of image space: m * P + k;
    (l, i) index of the Z-space: l * nE + i.
    """
    L, P, nE, nw = geom.n_rays, geom.n_pixels, sp.s.shape[1], sp.s.shape[2]
    mu = sp.mu
    Z = np.zeros((L * nE, 3 * P))
    for m in range(3):
        Z[:, m * P:(m + 1) * P] = np.kron(X, mu[m][:, None])    # rows (l, i)
    zf = Z @ f0.T.reshape(-1)                                    # (Zf)_{l,i}
    e0, e1, e2 = sexp(-zf, 0), sexp(-zf, 1), sexp(-zf, 2)
    bins = np.arange(L) % geom.n_bins
    A = np.zeros((nw * L, L * nE))
    B = np.zeros((nw * L, L * nE))
    chat = np.zeros(nw * L)
    for w in range(nw):
        for l in range(L):
            s = sp.s[bins[l], :, w]
            seg = slice(l * nE, (l + 1) * nE)
            den = float(s @ e0[seg])
            A[w * L + l, seg] = s * e1[seg] / den
            B[w * L + l, seg] = s * e2[seg] / den
            chat[w * L + l] = sp.N[bins[l], w] * den
    cvec = c.T.reshape(-1)                                        # (w, l) ordering
    r = cvec - chat
    K = A @ Z
    return dict(Z=Z, A=A, B=B, K=K, chat=chat, r=r, c=cvec)


def one_iteration(geom, sp, X, c, x, xbar, y, lam, spc="block", model="hessian"):
    """One MOCCA iteration in matrix form (reading of the step in the oracle header)."""
    L, P, nE, nw = geom.n_rays, geom.n_pixels, sp.s.shape[1], sp.s.shape[2]
    M = model_matrices(geom, sp, X, xbar, c)
    K, r, Z, A, B = M["K"], M["r"], M["Z"], M["A"], M["B"]
    Btr = B.T @ r
    cvec = M["chat"] + r
    # per-ray clipped Hessian in the ray's line integrals g (3x3)
    ynew = y.copy()
    for l in range(L):
        rows = [w * L + l for w in range(nw)]
        Kl = K[rows]                                          # [W, 3P]
        if not np.any(X[l]):
            continue
        k0 = int(np.flatnonzero(X[l])[0])
        alpha = Kl[:, [m * P + k0 for m in range(3)]] / X[l, k0]   # K_{wl,mk} = alpha_wm X_lk
        Zl = sp.mu.T                                          # d(Zf)_{l,i}/dg_m = mu_{m,i}
        seg = slice(l * nE, (l + 1) * nE)
        Al = A[rows][:, seg]
        H = -Zl.T @ np.diag(Btr[seg]) @ Zl + Zl.T @ Al.T @ np.diag(cvec[rows]) @ Al @ Zl
        lamH, V = np.linalg.eigh(H)
        Hp = V @ np.diag(np.maximum(lamH, 0)) @ V.T
        if spc == "block":
            sinv = lam * np.array([np.sum(np.sqrt(sum(Kl[w, m * P:(m + 1) * P] ** 2 for m in range(3))))
                                   for w in range(nw)])
        else:
            sinv = lam * np.abs(Kl).sum(axis=1)
        Sig = np.diag(1.0 / sinv)
        if model == "hessian":
            G = np.linalg.pinv(alpha)
            W = G.T @ Hp @ G
        else:
            W = np.zeros((nw, nw))
        yl = y[l]
        ynew[l] = yl - Sig @ np.linalg.solve(W + Sig, yl - r[rows])
    yv = ynew.T.reshape(-1)
    v = (K.T @ yv).reshape(3, P).T
    xn = x.copy()
    for k in range(P):
        cols = [m * P + k for m in range(3)]
        Kk = K[:, cols]                                       # [W L, 3]
        if spc == "block":
            nrm = np.sqrt((Kk ** 2).sum(axis=1))
            ok = nrm > 0
            Tinv = (Kk[ok].T * (1.0 / nrm[ok])) @ Kk[ok] / lam
        else:
            Tinv = np.diag(np.abs(Kk).sum(axis=0) / lam)
        tr = np.trace(Tinv)
        if tr <= 0:
            continue
        xn[k] = x[k] - np.linalg.solve(Tinv + 1e-12 * tr * np.eye(3), v[k])
    return xn, 2 * xn - x, ynew
