"""Derivatives of the superblock product and of the ground energy (oracle).

Not in the paper, which computes energies only; these follow from linear
algebra on H = sum_k c_k A_k (x) B_k (paper Sec. 3.3):

* y = H psi is linear in psi and in every c_k, so for a cotangent g:
  dL/dpsi = H^T g  and  dL/dc_k = <g, (A_k (x) B_k) psi>.
* Hellmann-Feynman: for a normalised eigenvector psi of a symmetric H,
  dE0/dc_k = <psi, (A_k (x) B_k) psi> / <psi, psi>.
* Couplings enter as c_k = mult_k * g_class(k), so
  dE0/dg = sum_{k in class} mult_k dE0/dc_k.
"""
from __future__ import annotations

import numpy as np

from . import superblock as osb


def apply_H_backward(sb, psi, g, b=0):
    """Returns (dpsi, dc) for y = H psi with cotangent g (batch member b)."""
    return osb.apply_HT(sb, g, b), osb.term_products(sb, g, psi)


def hf_grad(sb, psi):
    psi = np.asarray(psi, dtype=np.float64)
    return osb.term_products(sb, psi, psi) / float(psi @ psi)


def coupling_grad(sb, dE_dc):
    out = np.zeros(len(sb.class_names))
    for k in range(sb.n_terms):
        out[sb.term_class[k]] += sb.term_mult[k] * dE_dc[k]
    return out


def central_fd(fn, x0, h=1e-5):
    """Central finite differences of a scalar function of a vector."""
    x0 = np.asarray(x0, dtype=np.float64)
    g = np.zeros_like(x0)
    for i in range(len(x0)):
        xp = x0.copy()
        xm = x0.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (fn(xp) - fn(xm)) / (2 * h)
    return g
