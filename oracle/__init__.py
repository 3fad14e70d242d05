"""FP64 CPU oracle for MOCCA with m-block-diagonal step-preconditioning.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The GPU library
never calls it and the two share no code: the oracle is the plain, slow,
obviously correct double-precision statement of what the library computes,
written from the paper (arXiv:1801.06263, Sec. 2, Eqs. fullModel, finalModel,
DTPL, aeq and the m-block SPC) with the readings stated in ``mocca_oracle.c``.

Pins (tests/test_oracle_*.py) tie it to things other than itself: a brute-force
clipper, closed-form chords, the adjoint identity, closed-form counts, finite
differences, LAPACK eigen-decompositions, the step condition M >= 0, rotation
invariance, convex special cases solved by scipy, and noiseless convergence.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "mocca_oracle.c"), os.path.join(_HERE, "noise_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


class _Geom(ct.Structure):
    _fields_ = [("n", ct.c_int), ("pixel_mm", ct.c_double), ("n_views", ct.c_int),
                ("arc_deg", ct.c_double), ("start_deg", ct.c_double), ("n_bins", ct.c_int),
                ("bin_mm", ct.c_double), ("sid_mm", ct.c_double), ("sdd_mm", ct.c_double)]


class _Spectra(ct.Structure):
    _fields_ = [("n_energies", ct.c_int), ("s", _dp), ("N", _dp), ("mu", _dp), ("exp_model", ct.c_int),
                ("n_windows", ct.c_int)]


class _Params(ct.Structure):
    _fields_ = [("lambda_", ct.c_double), ("use_box", ct.c_int), ("lo", ct.c_double * 3),
                ("hi", ct.c_double * 3), ("spc", ct.c_int), ("model", ct.c_int), ("inner", ct.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP over rays/pixels)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-fPIC", "-shared", *_SRCS, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        L = _lib
        L.orc_siddon.argtypes = [ct.POINTER(_Geom), ct.c_int, ct.c_int, _ip, _dp, ct.c_int]
        L.orc_siddon.restype = ct.c_int
        L.orc_ray_endpoints.argtypes = [ct.POINTER(_Geom), ct.c_int, ct.c_int, _dp, _dp]
        L.orc_forward.argtypes = [ct.POINTER(_Geom), _dp, ct.c_int, _dp]
        L.orc_backproject.argtypes = [ct.POINTER(_Geom), _dp, ct.c_int, _dp]
        L.orc_ray_terms.argtypes = [ct.POINTER(_Spectra), ct.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                    _dp, _dp, _dp]
        L.orc_counts.argtypes = [ct.POINTER(_Geom), ct.POINTER(_Spectra), _dp, _dp]
        L.orc_dtpl.argtypes = [ct.c_int, _dp, _dp]
        L.orc_dtpl.restype = ct.c_double
        L.orc_objective.argtypes = [ct.POINTER(_Geom), ct.POINTER(_Spectra), _dp, _dp, _dp]
        L.orc_objective.restype = ct.c_double
        L.orc_solve.argtypes = [ct.c_int, _dp, _dp, _dp]
        L.orc_solve.restype = ct.c_int
        L.orc_eig_sym3.argtypes = [_dp, _dp, _dp]
        L.orc_clip_psd3.argtypes = [_dp, _dp]
        L.orc_dual_update.argtypes = [ct.c_int, _dp, _dp, _dp, _dp, ct.c_int, _dp, _dp, _dp]
        L.orc_dual_update.restype = ct.c_int
        L.orc_primal_update.argtypes = [_dp, _dp, _dp, ct.c_int, _dp, _dp, _dp]
        L.orc_primal_update.restype = ct.c_int
        L.orc_step_matrices.argtypes = [ct.POINTER(_Geom), ct.POINTER(_Spectra),
                                        ct.POINTER(_Params), _dp, _dp, _dp, _dp]
        L.orc_mocca.argtypes = [ct.POINTER(_Geom), ct.POINTER(_Spectra), ct.POINTER(_Params), _dp,
                                _dp, _dp, _dp, ct.c_int, _dp]
        L.orc_mocca.restype = ct.c_int
        L.orc_set_threads.argtypes = [ct.c_int]
        L.orc_philox4x32_10.argtypes = [ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint32)]
        L.orc_poisson_draw.argtypes = [ct.c_double, ct.c_uint32, ct.POINTER(ct.c_uint32)]
        L.orc_poisson_draw.restype = ct.c_double
        L.orc_poisson_noise.argtypes = [ct.c_int, _dp, ct.c_uint64, _dp]
        L.orc_max_threads.restype = ct.c_int
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _geom(g) -> _Geom:
    return _Geom(g.n, g.pixel_mm, g.n_views, g.arc_deg, g.start_deg, g.n_bins, g.bin_mm,
                 g.sid_mm, g.sdd_mm)


class _SpecHolder:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, sp, mu=None, counts_model="softexp"):
        self.s = _f64(sp.s)
        self.N = _f64(sp.N)
        self.mu = _f64(sp.mu if mu is None else mu)
        self.nw = self.s.shape[2]
        self.c = _Spectra(self.s.shape[1], _ptr(self.s), _ptr(self.N), _ptr(self.mu),
                          {"softexp": 0, "exp": 1}[counts_model], self.nw)


def _params(lam, use_box=False, lo=(0, 0, 0), hi=(0, 0, 0), spc="block", model="hessian", inner=1):
    return _Params(float(lam), int(bool(use_box)), (ct.c_double * 3)(*lo), (ct.c_double * 3)(*hi),
                   {"block": 0, "diagonal": 1}[spc], MODELS[model], int(inner))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------- geometry / X

def ray_endpoints(geom, v, b):
    S = np.zeros(2)
    D = np.zeros(2)
    lib().orc_ray_endpoints(ct.byref(_geom(geom)), int(v), int(b), _ptr(S), _ptr(D))
    return S, D


def siddon(geom, v, b):
    cap = 2 * geom.n + 4
    pix = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap)
    cnt = lib().orc_siddon(ct.byref(_geom(geom)), int(v), int(b),
                           pix.ctypes.data_as(_ip), _ptr(ln), cap)
    return pix[:cnt].copy(), ln[:cnt].copy()


def forward(geom, f):
    f = _f64(f)
    C = 1 if f.ndim == 1 else f.shape[1]
    g = np.zeros((geom.n_rays, C))
    lib().orc_forward(ct.byref(_geom(geom)), _ptr(f), C, _ptr(g))
    return g[:, 0] if f.ndim == 1 else g


def backproject(geom, rf):
    rf = _f64(rf)
    C = 1 if rf.ndim == 1 else rf.shape[1]
    img = np.zeros((geom.n_pixels, C))
    lib().orc_backproject(ct.byref(_geom(geom)), _ptr(rf), C, _ptr(img))
    return img[:, 0] if rf.ndim == 1 else img


# --------------------------------------------------------------------------- counts model

def counts(geom, spectra, f, mu=None, counts_model="softexp"):
    """Expected counts c^(f), [L, W] (Eq. finalModel; counts_model="exp": Eq. fullModel)."""
    sh = _SpecHolder(spectra, mu, counts_model)
    f = _f64(f)
    chat = np.zeros((geom.n_rays, sh.nw))
    lib().orc_counts(ct.byref(_geom(geom)), ct.byref(sh.c), _ptr(f), _ptr(chat))
    return chat


def ray_terms(spectra, b, g, c=None, with_AB=False, mu=None, counts_model="softexp"):
    sh = _SpecHolder(spectra, mu, counts_model)
    nE, nw = sh.s.shape[1], sh.nw
    g = _f64(g)
    cw = None if c is None else _f64(c)
    out = {k: np.zeros(sz) for k, sz in
           (("chat", nw), ("r", nw), ("alpha", 3 * nw), ("grad", 3), ("H", 9))}
    A = np.zeros(nw * nE) if with_AB else None
    B = np.zeros(nw * nE) if with_AB else None
    lib().orc_ray_terms(ct.byref(sh.c), int(b), _ptr(g), _ptr(cw), _ptr(out["chat"]),
                        _ptr(out["r"]), _ptr(out["alpha"]), _ptr(out["grad"]), _ptr(out["H"]),
                        _ptr(A), _ptr(B))
    out["alpha"] = out["alpha"].reshape(nw, 3)
    out["H"] = out["H"].reshape(3, 3)
    if with_AB:
        out["A"] = A.reshape(nw, nE)
        out["B"] = B.reshape(nw, nE)
    return out


def dtpl(c, chat):
    c = _f64(c).ravel()
    chat = _f64(chat).ravel()
    return float(lib().orc_dtpl(c.size, _ptr(c), _ptr(chat)))


def objective(geom, spectra, c, f, with_grad=True, mu=None, counts_model="softexp"):
    sh = _SpecHolder(spectra, mu, counts_model)
    c = _f64(c)
    f = _f64(f)
    grad = np.zeros((geom.n_pixels, 3)) if with_grad else None
    d = lib().orc_objective(ct.byref(_geom(geom)), ct.byref(sh.c), _ptr(c), _ptr(f), _ptr(grad))
    return (float(d), grad) if with_grad else float(d)


# --------------------------------------------------------------------------- small algebra

def solve(M, rhs):
    M = _f64(M)
    rhs = _f64(rhs)
    x = np.zeros(rhs.size)
    st = lib().orc_solve(rhs.size, _ptr(M), _ptr(rhs), _ptr(x))
    if st:
        raise np.linalg.LinAlgError("singular")
    return x


def eig_sym3(H):
    H = _f64(H)
    lam = np.zeros(3)
    V = np.zeros(9)
    lib().orc_eig_sym3(_ptr(H), _ptr(lam), _ptr(V))
    return lam, V.reshape(3, 3)


def clip_psd3(H):
    H = _f64(H)
    Hp = np.zeros(9)
    lib().orc_clip_psd3(_ptr(H), _ptr(Hp))
    return Hp.reshape(3, 3)


MODELS = {"hessian": 0, "gradient": 1, "gauss_newton": 2, "separable": 3}


def dual_update(alpha, Hp, r, sigma_inv, y, model="hessian", c=None):
    """Dual step of one ray; c (the window counts) is needed by model="separable"."""
    alpha = _f64(alpha).reshape(-1, 3)
    nw = alpha.shape[0]
    out = np.zeros(nw)
    cw = _f64(np.zeros(nw) if c is None else c)
    st = lib().orc_dual_update(nw, _ptr(alpha), _ptr(_f64(Hp)), _ptr(_f64(r)),
                               _ptr(_f64(sigma_inv)), MODELS[model], _ptr(cw),
                               _ptr(_f64(y)), _ptr(out))
    if st:
        raise np.linalg.LinAlgError("singular dual system")
    return out


def primal_update(Tinv, v, x, box=None):
    out = np.zeros(3)
    lo = _f64(box[0] if box else np.zeros(3))
    hi = _f64(box[1] if box else np.zeros(3))
    st = lib().orc_primal_update(_ptr(_f64(Tinv)), _ptr(_f64(v)), _ptr(_f64(x)),
                                 int(box is not None), _ptr(lo), _ptr(hi), _ptr(out))
    if st:
        raise np.linalg.LinAlgError("singular primal system")
    return out


# --------------------------------------------------------------------------- MOCCA

def step_matrices(geom, spectra, xbar, lam, spc="block", mu=None, counts_model="softexp"):
    sh = _SpecHolder(spectra, mu, counts_model)
    P = _params(lam, spc=spc)
    xbar = _f64(xbar)
    sinv = np.zeros((geom.n_rays, sh.nw))
    Tinv = np.zeros((geom.n_pixels, 9))
    alpha = np.zeros((geom.n_rays, 3 * sh.nw))
    lib().orc_step_matrices(ct.byref(_geom(geom)), ct.byref(sh.c), ct.byref(P), _ptr(xbar),
                            _ptr(sinv), _ptr(Tinv), _ptr(alpha))
    return sinv, Tinv.reshape(-1, 3, 3), alpha.reshape(-1, sh.nw, 3)


class State:
    """MOCCA state: x = x_n [P,3], xbar = 2 x_n - x_{n-1} [P,3], y = y_n [L,W]."""

    def __init__(self, geom, n_windows=4):
        self.x = np.zeros((geom.n_pixels, 3))
        self.xbar = np.zeros((geom.n_pixels, 3))
        self.y = np.zeros((geom.n_rays, n_windows))
        self.n = 0

    def copy(self):
        s = State.__new__(State)
        s.x, s.xbar, s.y, s.n = self.x.copy(), self.xbar.copy(), self.y.copy(), self.n
        return s


def mocca(geom, spectra, c, n_iters, lam, state=None, *, box=None, spc="block",
          model="hessian", mu=None, counts_model="softexp", inner=1):
    """Run n_iters MOCCA iterations from `state` (zeros if None); returns
    (state, dtpl_history) with dtpl_history[i] = D_TPL(c, c^(xbar_i)).
    counts_model="exp" replaces softexp by exp (the standard model, Eq. fullModel).
    inner=k > 1: nested MOCCA, a new local model every k iterations of this call
    (the first iteration of a call is always an outer one; see orc_mocca)."""
    sh = _SpecHolder(spectra, mu, counts_model)
    st = State(geom, sh.nw) if state is None else state
    assert st.y.shape == (geom.n_rays, sh.nw)
    lo, hi = (box if box is not None else ((0, 0, 0), (0, 0, 0)))
    P = _params(lam, box is not None, tuple(lo), tuple(hi), spc, model, inner)
    c = _f64(c)
    hist = np.zeros(n_iters)
    for arr in (st.x, st.xbar, st.y):
        assert arr.flags.c_contiguous and arr.dtype == np.float64
    rc = lib().orc_mocca(ct.byref(_geom(geom)), ct.byref(sh.c), ct.byref(P), _ptr(c),
                         _ptr(st.x), _ptr(st.xbar), _ptr(st.y), int(n_iters), _ptr(hist))
    if rc:
        raise np.linalg.LinAlgError("singular small system inside MOCCA")
    st.n += n_iters
    return st, hist


# --------------------------------------------------------------------------- mu-PC basis change

def mu_pc(mu, weights=None):
    """mu-PC (Sec. 1 and 2): (mu_t, M) with mu_t = M mu, whose rows are
    orthonormal over the energy grid in the inner product sum_i weights_i a_i b_i
    (Euclidean when weights is None), and M = (mu diag(weights) mu^T)^(-1/2), the
    symmetric choice (the paper leaves the orthogonalisation to Barber et al.
    2016).  numpy's eigh is the step."""
    mu = np.asarray(mu, dtype=np.float64)
    wts = np.ones(mu.shape[1]) if weights is None else np.asarray(weights, dtype=np.float64)
    w, V = np.linalg.eigh((mu * wts) @ mu.T)
    M = V @ np.diag(w ** -0.5) @ V.T
    return M @ mu, M


def maps_to_basis(f, M):
    """Maps in the mu-PC basis, f' = M^-1 f per pixel (f [P, 3]), so that mu_t^T f' = mu^T f."""
    return np.asarray(f, dtype=np.float64) @ np.linalg.inv(M).T


def maps_from_basis(f_t, M):
    """Maps in the original basis, f = M f' per pixel."""
    return np.asarray(f_t, dtype=np.float64) @ np.asarray(M).T


# --------------------------------------------------------------------------- seeded Poisson noise

def philox4x32_10(ctr, key):
    """Philox4x32-10 of four 32-bit counter words under two key words (noise_oracle.c)."""
    c = (ct.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ct.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (ct.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, out)
    return [int(v) for v in out]


def poisson_noise(chat, seed: int):
    """c ~ Poisson(chat) elementwise (any shape), sample i (in C order) drawn from
    counter (i, t, 0, 0) under key (seed mod 2^32, seed / 2^32)."""
    chat = _f64(chat)
    out = np.zeros_like(chat)
    lib().orc_poisson_noise(int(chat.size), _ptr(chat), ct.c_uint64(int(seed)), _ptr(out))
    return out
