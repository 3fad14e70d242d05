"""mu-preconditioning (mu-PC) of the material basis (Sec. 1 and Sec. 2).

mu-PC replaces the material basis by one whose attenuation curves are
orthonormal functions of energy and then runs MOCCA with the diagonal
step-preconditioner on the transformed problem; the maps are transformed back
afterwards.  With mu' = M mu and f' = M^-T f the line integrals are unchanged
(mu'^T f' = mu^T f).  The paper does not state which orthogonalisation is
used; this reading takes the Euclidean inner product over the energy grid and
the symmetric choice M = (mu mu^T)^(-1/2).
"""
from __future__ import annotations

import numpy as np


def mu_pc(mu: np.ndarray):
    """Return (mu_t, M) with mu_t = M mu having orthonormal rows, M = (mu mu^T)^(-1/2)."""
    mu = np.asarray(mu, dtype=np.float64)
    w, V = np.linalg.eigh(mu @ mu.T)
    M = V @ np.diag(w ** -0.5) @ V.T
    return M @ mu, M


def maps_to_basis(f: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Maps in the transformed basis: f' = M^-T f (per pixel, f of shape [P, 3])."""
    return np.asarray(f) @ np.linalg.inv(M)


def maps_from_basis(f_t: np.ndarray, M: np.ndarray) -> np.ndarray:
    """Maps in the original basis: f = M^T f' (per pixel)."""
    return np.asarray(f_t) @ M
