"""Site operators and whole-lattice Hamiltonians (oracle).

Paper Sec. 1: site bases C = {up, dn} (spin-1/2 Heisenberg) and
C = {e, up, dn, updn} (Hubbard).  Paper Sec. 4.1: the Hubbard model
sum t_ij c^dag_i c_j + sum U_i n_up n_dn + sum V_i n_i and the Heisenberg
model sum J_ij S_i . S_j.

Readings (the paper is silent on these):
* hopping enters as H = -t sum_<ij>,sigma (c^dag_i c_j + h.c.);
* fermion signs: Jordan-Wigner order by site label, |updn> = c^dag_up c^dag_dn|e>;
* effective quantum number (Sec. 3.2, q = sum_a q~_a Q^a): Heisenberg
  q = N_up; Hubbard q = N_up + Q N_dn with Q = L + 1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------- sites


def heisenberg_site():
    """Spin-1/2 site, basis order (up, dn)."""
    Sz = np.diag([0.5, -0.5])
    Sp = np.array([[0.0, 1.0], [0.0, 0.0]])  # S^+ |dn> = |up>
    n_up = np.array([1, 0])
    return dict(Sz=Sz, Sp=Sp, Sm=Sp.T.copy(), I=np.eye(2), n_up=n_up,
                n_dn=1 - n_up, d=2, fermion=False)


def hubbard_site():
    """Hubbard site, basis order (e, up, dn, updn) with |updn> = c^dag_up c^dag_dn |e>."""
    c_up = np.zeros((4, 4))
    c_up[0, 1] = 1.0   # c_up |up> = |e>
    c_up[2, 3] = 1.0   # c_up c^dag_up c^dag_dn |e> = |dn>
    c_dn = np.zeros((4, 4))
    c_dn[0, 2] = 1.0   # c_dn |dn> = |e>
    c_dn[1, 3] = -1.0  # c_dn c^dag_up c^dag_dn |e> = -|up>
    n_up = np.array([0, 1, 0, 1])
    n_dn = np.array([0, 0, 1, 1])
    F = np.diag((-1.0) ** (n_up + n_dn))
    return dict(c_up=c_up, c_dn=c_dn, F=F, I=np.eye(4),
                nn=np.diag((n_up * n_dn).astype(float)),
                n_up=n_up, n_dn=n_dn, d=4, fermion=True)


# ------------------------------------------------------------ geometries


def chain_bonds(L, nnn=False):
    """Open chain: nearest-neighbour bonds (i, i+1), class 'J1' or 't';
    with nnn=True also (i, i+2) of class 'J2'."""
    b = [(i, i + 1, 1) for i in range(L - 1)]
    if nnn:
        b += [(i, i + 2, 2) for i in range(L - 2)]
    return b


def ladder_bonds(L):
    """Two-leg ladder, site i = 2*x + leg: rungs (2x, 2x+1) class 'rung',
    legs (i, i+2) class 'leg' (reading of the paper's n-leg ladder geometry
    with one site added per DMRG step)."""
    b = []
    for i in range(L):
        if i % 2 == 0 and i + 1 < L:
            b.append((i, i + 1, "rung"))
        if i + 2 < L:
            b.append((i, i + 2, "leg"))
    return b


# ------------------------------------------------ whole-lattice operators


def _embed(ops_per_site, L):
    """Sparse kron of a list of L single-site matrices."""
    out = sp.csr_matrix(np.array([[1.0]]))
    for o in ops_per_site:
        out = sp.kron(out, sp.csr_matrix(o), format="csr")
    return out


def lattice_fermion_c(L, i, spin, site=None):
    """c_{i,spin} on L Hubbard sites with the Jordan-Wigner string F on j < i."""
    s = site or hubbard_site()
    ops = [s["F"]] * i + [s["c_" + spin]] + [s["I"]] * (L - i - 1)
    return _embed(ops, L)


def heisenberg_lattice(L, bonds, couplings):
    """Terms of sum_b J_class(b) S_i . S_j as a dict class -> sparse matrix
    (unit coupling), plus the quantum number q = N_up of every basis state."""
    s = heisenberg_site()
    d = 2
    H = {}
    for (i, j, cls) in bonds:
        def op(Oi, Oj):
            ops = [s["I"]] * L
            ops[i] = Oi
            ops[j] = Oj
            return _embed(ops, L)
        h = op(s["Sz"], s["Sz"]) + 0.5 * (op(s["Sp"], s["Sm"]) + op(s["Sm"], s["Sp"]))
        H[cls] = H.get(cls, 0) + h
    q = np.zeros(d ** L, dtype=np.int64)
    for i in range(L):
        ops = [np.ones(d)] * L
        ops[i] = s["n_up"].astype(float)
        v = np.array([1.0])
        for o in ops:
            v = np.kron(v, o)
        q += v.astype(np.int64)
    total = sum(couplings[k] * H[k] for k in H)
    return total, H, q


def hubbard_lattice(L, bonds, t_by_class, U):
    """H = -sum_b t_class(b) sum_sigma (c^dag_i c_j + h.c.) + U sum_i n_up n_dn.
    Returns (H, parts {'t': unit hopping part (with its minus sign), 'U': sum nn},
    n_up per state, n_dn per state)."""
    s = hubbard_site()
    Hhop = {}
    for (i, j, cls) in bonds:
        for spin in ("up", "dn"):
            ci = lattice_fermion_c(L, i, spin, s)
            cj = lattice_fermion_c(L, j, spin, s)
            h = ci.T @ cj
            Hhop[cls] = Hhop.get(cls, 0) - (h + h.T)
    HU = 0
    for i in range(L):
        ops = [s["I"]] * L
        ops[i] = s["nn"]
        HU = HU + _embed(ops, L)
    nu = np.zeros(4 ** L, dtype=np.int64)
    nd = np.zeros(4 ** L, dtype=np.int64)
    for i in range(L):
        a = np.array([1.0])
        b = np.array([1.0])
        for k in range(L):
            a = np.kron(a, s["n_up"] if k == i else np.ones(4))
            b = np.kron(b, s["n_dn"] if k == i else np.ones(4))
        nu += a.astype(np.int64)
        nd += b.astype(np.int64)
    H = sum(t_by_class[k] * Hhop[k] for k in Hhop) + U * HU
    parts = dict(Hhop)
    parts["U"] = HU
    return H, parts, nu, nd
