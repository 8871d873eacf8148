"""Exact diagonalisation of a whole lattice in one symmetry sector (oracle).

Brute force: the full lattice Hamiltonian from explicit Kronecker products of
site operators (oracle.models), restricted to the states with the requested
quantum numbers (paper Sec. 3.2: H is block diagonal in the effective quantum
number), lowest eigenpair by dense ``eigh`` or sparse ``eigsh``.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import models


def lowest(H, dense_max=3000):
    n = H.shape[0]
    if n <= dense_max:
        M = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
        w, v = sla.eigh(M)
        return float(w[0]), v[:, 0]
    w, v = spla.eigsh(H, k=1, which="SA", tol=1e-14, maxiter=100000)
    return float(w[0]), v[:, 0]


def heisenberg_ed(L, n_up=None, J1=1.0, J2=0.0):
    """Ground energy of the open J1-J2 chain in the sector N_up (default L/2)."""
    if n_up is None:
        n_up = L // 2
    bonds = models.chain_bonds(L, nnn=(J2 != 0.0))
    H, parts, q = models.heisenberg_lattice(L, bonds, {1: J1, 2: J2})
    idx = np.nonzero(q == n_up)[0]
    Hs = H.tocsr()[idx][:, idx]
    return lowest(Hs)[0]


def heisenberg_ed_parts(L, n_up, J1, J2):
    """Ground energy and <psi|H_class|psi> for the J1 and J2 parts (used for
    finite-difference and Hellmann-Feynman pins)."""
    bonds = models.chain_bonds(L, nnn=True)
    H, parts, q = models.heisenberg_lattice(L, bonds, {1: J1, 2: J2})
    idx = np.nonzero(q == n_up)[0]
    Hs = H.tocsr()[idx][:, idx]
    e, v = lowest(Hs)
    ev = {k: float(v @ (parts[k].tocsr()[idx][:, idx] @ v)) for k in parts}
    return e, ev


def hubbard_ed(L, n_up, n_dn, t=1.0, U=4.0, geometry="chain", t_rung=None):
    if geometry == "chain":
        bonds = [(i, i + 1, "t") for i in range(L - 1)]
        tb = {"t": t}
    else:
        bonds = models.ladder_bonds(L)
        tb = {"leg": t, "rung": t if t_rung is None else t_rung}
    H, parts, nu, nd = models.hubbard_lattice(L, bonds, tb, U)
    idx = np.nonzero((nu == n_up) & (nd == n_dn))[0]
    Hs = H.tocsr()[idx][:, idx]
    return lowest(Hs)[0]
