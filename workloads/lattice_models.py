"""Model descriptors of the device DMRG driver (input data only).

A model is given to the library as data (paper Sec. 4.1: the Hubbard and
Heisenberg models; Sec. 1: the site bases): the site basis with the
effective quantum number and fermion parity of each state, the site
operators kept at block boundaries, on-site terms, the lattice as bond rules
(bonds (p, p + delta) of a coupling class for every p with p % mod == rem),
and the unit-coupling bond Hamiltonian as a sum of coef * op(O_a at i) *
op(O_b at j), i < j, op = transpose or not.  Nothing here does any
arithmetic of the method.

Conventions (the same physics as the oracle's own, independent model code):
* Heisenberg site basis (up, dn), q = N_up; S^z S^z + (S^+ S^- + S^- S^+)/2
  with S^- = (S^+)^T.  Target q = L/2 (S_z = 0).
* Hubbard site basis (e, up, dn, updn) with |updn> = c^dag_up c^dag_dn |e>,
  q = N_up + Q N_dn; hopping -t (c^dag_i c_j + c^dag_j c_i) per spin, written
  with the i-first operators: -t (c_i^T c_j) + t (c_i c_j^T) (the second is
  c^dag_j c_i after anticommuting the two Jordan-Wigner operators).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


@dataclass
class ModelDesc:
    site_q: np.ndarray
    site_parity: np.ndarray
    op_names: List[str]
    ops: np.ndarray                       # [n_ops][d][d]
    op_fermion: np.ndarray
    class_names: List[str]
    couplings: np.ndarray
    onsite_class: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int32))
    onsite: np.ndarray = field(default_factory=lambda: np.zeros((0, 1, 1)))
    bond_rules: np.ndarray = field(default_factory=lambda: np.zeros((0, 4), dtype=np.int32))
    bond_terms: List[Tuple[float, int, int, int, int]] = field(default_factory=list)
    density: float = 1.0
    Q: int = 0

    @property
    def d(self) -> int:
        return int(len(self.site_q))


def heisenberg_chain(J1: float = 1.0, J2: float = 0.0) -> ModelDesc:
    """Open spin-1/2 chain, J1 nearest and (J2 != 0) next-nearest neighbours."""
    Sz = np.diag([0.5, -0.5])
    Sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    classes, g, rules = ["J1"], [J1], [[1, 0, 1, 0]]
    if J2 != 0.0:
        classes.append("J2")
        g.append(J2)
        rules.append([2, 1, 1, 0])
    return ModelDesc(site_q=np.array([1, 0], dtype=np.int64), site_parity=np.zeros(2, dtype=np.int32),
                     op_names=["Sz", "Sp"], ops=np.stack([Sz, Sp]), op_fermion=np.zeros(2, dtype=np.int32),
                     class_names=classes, couplings=np.array(g, dtype=np.float64),
                     bond_rules=np.array(rules, dtype=np.int32),
                     bond_terms=[(1.0, 0, 0, 0, 0), (0.5, 1, 0, 1, 1), (0.5, 1, 1, 1, 0)],
                     density=1.0, Q=0)


def _hubbard_site():
    cu = np.zeros((4, 4))
    cu[0, 1] = 1.0   # c_up |up> = |e>
    cu[2, 3] = 1.0   # c_up |updn> = |dn>
    cd = np.zeros((4, 4))
    cd[0, 2] = 1.0   # c_dn |dn> = |e>
    cd[1, 3] = -1.0  # c_dn |updn> = -|up>
    nn = np.diag([0.0, 0.0, 0.0, 1.0])
    return cu, cd, nn


_HOP = [(-1.0, 0, 1, 0, 0), (1.0, 0, 0, 0, 1), (-1.0, 1, 1, 1, 0), (1.0, 1, 0, 1, 1)]


def _hubbard(classes, g, rules, density, Q):
    cu, cd, nn = _hubbard_site()
    iu = classes.index("U")
    return ModelDesc(site_q=np.array([0, 1, Q, Q + 1], dtype=np.int64),
                     site_parity=np.array([0, 1, 1, 0], dtype=np.int32),
                     op_names=["c_up", "c_dn"], ops=np.stack([cu, cd]), op_fermion=np.ones(2, dtype=np.int32),
                     class_names=classes, couplings=np.array(g, dtype=np.float64),
                     onsite_class=np.array([iu], dtype=np.int32), onsite=nn[None].copy(),
                     bond_rules=np.array(rules, dtype=np.int32), bond_terms=list(_HOP),
                     density=density, Q=Q)


def hubbard_chain(t: float = 1.0, U: float = 4.0, density: float = 1.0, Q: int = 65) -> ModelDesc:
    """Open Hubbard chain; classes (t, U)."""
    return _hubbard(["t", "U"], [t, U], [[1, 0, 1, 0]], density, Q)


def hubbard_ladder(t_leg: float = 1.0, t_rung: float = 1.0, U: float = 8.0, density: float = 1.0,
                   Q: int = 65) -> ModelDesc:
    """Two-leg Hubbard ladder, site i = 2 x + leg: rungs (2x, 2x + 1), legs
    (i, i + 2); classes (t_leg, t_rung, U)."""
    return _hubbard(["t_leg", "t_rung", "U"], [t_leg, t_rung, U], [[2, 0, 1, 0], [1, 1, 2, 0]], density, Q)
