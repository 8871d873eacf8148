"""Lanczos lowest eigenpair with full reorthogonalisation (oracle).

The paper diagonalises each targeted superblock with the Lanczos method
(Sec. 3.3, refs. Lanczos 1950 and Pettifor & Weaire 1985) and needs only the
operation x += H y.  It gives no tolerance, cap or reorthogonalisation rule;
the readings used here:

* start vector: the given (seeded N(0,1)) vector, normalised;
* every new Krylov vector is orthogonalised against all previous ones with
  classical Gram-Schmidt applied twice (CGS2), in float64;
* alpha_j = <v_j, H v_j> (the j-th Gram-Schmidt coefficient of both passes),
  beta_j = || w || after reorthogonalisation;
* stop when beta_j |s_j| <= tol * max(1, |theta|), where (theta, s) is the
  lowest eigenpair of the tridiagonal T_j and s_j its last component
  (the residual norm of the Ritz pair), or when beta_j falls below
  1e-14 * max(1, |theta|) (invariant subspace: theta is exact), or at max_iter;
* T_j is diagonalised with LAPACK's symmetric tridiagonal solver.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class LanczosResult:
    e0: float
    psi: np.ndarray
    iters: int
    residual: float
    converged: bool
    breakdown: bool
    alphas: np.ndarray
    betas: np.ndarray


def tridiag_lowest(alphas, betas):
    """Lowest eigenpair of the symmetric tridiagonal matrix with diagonal
    ``alphas`` and off-diagonal ``betas`` (len(alphas) - 1)."""
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)
    if len(a) == 1:
        return float(a[0]), np.array([1.0])
    w, v = sla.eigh_tridiagonal(a, b, select="i", select_range=(0, 0))
    s = v[:, 0]
    if s[0] < 0:
        s = -s
    return float(w[0]), s


def lanczos_ground(matvec, v0, tol=1e-12, max_iter=300) -> LanczosResult:
    v0 = np.asarray(v0, dtype=np.float64)
    D = v0.shape[0]
    max_iter = int(min(max_iter, D))
    V = np.zeros((max_iter + 1, D))
    V[0] = v0 / np.linalg.norm(v0)
    alphas, betas = [], []
    theta, s = 0.0, np.array([1.0])
    resid = np.inf
    converged = breakdown = False
    j = 0
    for j in range(max_iter):
        w = matvec(V[j])
        h1 = V[: j + 1] @ w
        w = w - V[: j + 1].T @ h1
        h2 = V[: j + 1] @ w
        w = w - V[: j + 1].T @ h2
        alphas.append(h1[j] + h2[j])
        beta = float(np.linalg.norm(w))
        theta, s = tridiag_lowest(alphas, betas)
        resid = beta * abs(s[-1])
        scale = max(1.0, abs(theta))
        if beta < 1e-14 * scale or j + 1 == D:
            breakdown = True
            converged = True
            break
        if resid <= tol * scale:
            converged = True
            break
        betas.append(beta)
        V[j + 1] = w / beta
    k = len(alphas)
    psi = V[:k].T @ s
    psi /= np.linalg.norm(psi)
    return LanczosResult(theta, psi, k, float(resid), converged, breakdown,
                         np.array(alphas), np.array(betas))


def rayleigh(matvec, psi):
    """<psi|H|psi> / <psi|psi> and the residual norm ||H psi - theta psi|| / ||psi||."""
    psi = np.asarray(psi, dtype=np.float64)
    n2 = float(psi @ psi)
    w = matvec(psi)
    th = float(psi @ w) / n2
    res = float(np.linalg.norm(w - th * psi)) / np.sqrt(n2)
    return th, res
