"""Independent brute-force lattice Hamiltonians in an occupation-number basis.

Test-side helpers, written without the oracle's Kronecker/Jordan-Wigner
machinery: states are bit strings, spin flips and hoppings are bit
operations, and the fermion sign of c^dag_i c_j is (-1)^(number of occupied
orbitals of the same spin strictly between i and j) with the orbitals of
one spin species ordered by site.  The spectrum does not depend on the
ordering convention, so these pin the oracle's energies.
"""
from itertools import combinations

import numpy as np


def _states(L, n):
    return [sum(1 << i for i in c) for c in combinations(range(L), n)]


def heisenberg_matrix(L, bonds, n_up):
    """bonds: [(i, j, J)].  Bit 1 = spin up."""
    st = _states(L, n_up)
    idx = {s: k for k, s in enumerate(st)}
    H = np.zeros((len(st), len(st)))
    for k, s in enumerate(st):
        for (i, j, J) in bonds:
            bi, bj = (s >> i) & 1, (s >> j) & 1
            H[k, k] += J * (0.25 if bi == bj else -0.25)
            if bi != bj:
                t = s ^ (1 << i) ^ (1 << j)
                H[idx[t], k] += 0.5 * J
    return H


def _hop(bits, i, j):
    """c^dag_i c_j on one spin species; returns (new_bits, sign) or None."""
    if not (bits >> j) & 1:
        return None
    if i != j and (bits >> i) & 1:
        return None
    lo, hi = min(i, j), max(i, j)
    between = bin(bits & (((1 << hi) - 1) ^ ((1 << (lo + 1)) - 1))).count("1")
    new = (bits ^ (1 << j)) | (1 << i)
    return new, (-1.0) ** between


def hubbard_matrix(L, bonds, U, n_up, n_dn):
    """H = -sum_(i,j,t) t (c^dag_i c_j + h.c.) per spin + U sum n_up n_dn."""
    ups, dns = _states(L, n_up), _states(L, n_dn)
    basis = [(u, d) for u in ups for d in dns]
    idx = {s: k for k, s in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    for k, (u, d) in enumerate(basis):
        H[k, k] += U * bin(u & d).count("1")
        for (i, j, t) in bonds:
            for (a, b) in ((i, j), (j, i)):
                r = _hop(u, a, b)
                if r is not None:
                    H[idx[(r[0], d)], k] += -t * r[1]
                r = _hop(d, a, b)
                if r is not None:
                    H[idx[(u, r[0])], k] += -t * r[1]
    return H


def lowest(H):
    return float(np.linalg.eigvalsh(H)[0])
