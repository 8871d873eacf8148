"""Local density of states by the continued-fraction method (oracle).

Test infrastructure: imported only by tests, the smoke check and the bench's
CPU-baseline leg.

Paper Sec. "DmrgSolver and the infinite DMRG algorithm" defines the local
density of states of the ground state psi as the time integral of
<psi| c_i^dag(t) c_i |psi> e^{i w t} and, in its closing notes, computes it
from the continued fraction of the Lanczos coefficients of the superblock
Hamiltonian (Hallberg 1995) over an energy window with a broadening.  The
readings used here (the printed formula carries the 2 pi of the time
integral and only the removal part; the figure shows both sides of the
Fermi level):

* removal part, normalised to <n_i>:
      A_<(w) = sum_n |<n|c_i|psi>|^2 delta(w - (E0 - E_n)),
  the resolvent of H in the N - 1 particle sector started from
  phi = c_i |psi>:  A_<(w) = -Im G_phi(E0 - w + i eta) / pi;
* addition part:  A_>(w) = sum_m |<m|c_i^dag|psi>|^2 delta(w - (E_m - E0))
  = -Im G_chi(E0 + w + i eta) / pi with chi = c_i^dag |psi> (N + 1);
* N_i(w) = A_<(w) + A_>(w), a sum of Lorentzians of half width eta; its
  integral is <c_i c_i^dag> + <c_i^dag c_i> = 1 per spin;
* G_v(z) = <v|(z - H)^-1|v> = |v|^2 / (z - a_0 - b_0^2 / (z - a_1 - b_1^2 /
  (... / (z - a_{k-1})))) with a_j, b_j the Lanczos diagonal and
  off-diagonal (b_j couples Krylov vectors j and j + 1) from v / |v|.

`lanczos_coefficients` is the ground-state solver's iteration (oracle.lanczos:
classical Gram-Schmidt applied twice against every Krylov vector) without its
stopping test; it stops early only at an invariant subspace.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from workloads.superblock import transition

from . import dmrg as odmrg
from . import models
from . import superblock as osb


def lanczos_coefficients(matvec, v0, n):
    """|v0|^2 and the first k <= n Lanczos coefficients from v0 / |v0|:
    alphas[0..k), betas[0..k-1) (betas[j] couples vectors j and j + 1)."""
    v0 = np.asarray(v0, dtype=np.float64)
    norm2 = float(v0 @ v0)
    D = v0.shape[0]
    n = int(min(n, D))
    V = np.zeros((n + 1, D))
    V[0] = v0 / np.sqrt(norm2)
    alphas, betas = [], []
    for j in range(n):
        w = matvec(V[j])
        h1 = V[: j + 1] @ w
        w = w - V[: j + 1].T @ h1
        h2 = V[: j + 1] @ w
        w = w - V[: j + 1].T @ h2
        alphas.append(float(h1[j] + h2[j]))
        beta = float(np.linalg.norm(w))
        scale = max(1.0, abs(alphas[-1]))
        if j + 1 == n or beta < 1e-14 * scale:
            break
        betas.append(beta)
        V[j + 1] = w / beta
    return norm2, np.array(alphas), np.array(betas)


def continued_fraction(norm2, alphas, betas, z):
    """G(z) = <v|(z - H)^-1|v> from the Lanczos coefficients of v, for an
    array of complex z, evaluated from the deepest level up."""
    z = np.asarray(z, dtype=np.complex128)
    k = len(alphas)
    t = z - alphas[k - 1]
    for j in range(k - 2, -1, -1):
        t = z - alphas[j] - betas[j] ** 2 / t
    return norm2 / t


def spectral_sum(energies, weights, z):
    """sum_m w_m / (z - E_m): the resolvent from a spectral decomposition."""
    z = np.asarray(z, dtype=np.complex128)
    return (np.asarray(weights)[None, :] / (z[:, None] - np.asarray(energies)[None, :])).sum(axis=1)


def ldos_from_fractions(cf_hole, cf_particle, e0, omega, eta):
    """(A_<, A_>) on the grid omega from the two continued fractions, each a
    tuple (norm2, alphas, betas); a missing part (None) counts as zero."""
    omega = np.asarray(omega, dtype=np.float64)
    out = []
    for cf, z in ((cf_hole, e0 - omega + 1j * eta), (cf_particle, e0 + omega + 1j * eta)):
        out.append(np.zeros_like(omega) if cf is None else -continued_fraction(*cf, z).imag / np.pi)
    return out[0], out[1]


def hubbard_ldos_ed(L, i, spin, n_up, n_dn, t, U, omega, eta, geometry="chain"):
    """Exact (A_<, A_>) of site i, spin `spin`, in the (n_up, n_dn) ground
    state of the open Hubbard chain or ladder: full diagonalisation of the
    N - 1 and N + 1 sectors, weights |<n|c|psi>|^2, Lorentzians of half width
    eta.  Also returns E0."""
    if geometry == "chain":
        bonds = [(a, a + 1, "t") for a in range(L - 1)]
        tb = {"t": t}
    else:
        bonds = models.ladder_bonds(L)
        tb = {"leg": t, "rung": t}
    H, _, nu, nd = models.hubbard_lattice(L, bonds, tb, U)
    H = H.tocsr()
    c = models.lattice_fermion_c(L, i, spin).tocsr()

    def sector(a, b):
        return np.nonzero((nu == a) & (nd == b))[0]

    i0 = sector(n_up, n_dn)
    w0, v0 = sla.eigh(H[i0][:, i0].toarray())
    e0, psi0 = float(w0[0]), v0[:, 0]
    full = np.zeros(H.shape[0])
    full[i0] = psi0
    d_up, d_dn = (1, 0) if spin == "up" else (0, 1)
    omega = np.asarray(omega, dtype=np.float64)
    parts = []
    for sgn, op in ((-1, c), (+1, c.T.tocsr())):
        idx = sector(n_up + sgn * d_up, n_dn + sgn * d_dn)
        if len(idx) == 0:
            parts.append(np.zeros_like(omega))
            continue
        phi = (op @ full)[idx]
        w, v = sla.eigh(H[idx][:, idx].toarray())
        weights = (v.T @ phi) ** 2
        z = (e0 - omega + 1j * eta) if sgn < 0 else (e0 + omega + 1j * eta)
        parts.append(-spectral_sum(w, weights, z).imag / np.pi)
    return parts[0], parts[1], e0


def free_chain_ldos(L, i, n_occ, t, omega, eta):
    """U = 0 open chain, closed form: single-particle orbitals
    phi_k(x) = sqrt(2 / (L + 1)) sin(k pi (x + 1) / (L + 1)), energies
    eps_k = -2 t cos(k pi / (L + 1)), k = 1 .. L; the n_occ lowest occupied.
    Removal weight |phi_k(i)|^2 at w = eps_k for occupied k, addition weight
    at w = eps_k for empty k."""
    k = np.arange(1, L + 1)
    eps = -2.0 * t * np.cos(k * np.pi / (L + 1))
    amp2 = 2.0 / (L + 1) * np.sin(k * np.pi * (i + 1) / (L + 1)) ** 2
    omega = np.asarray(omega, dtype=np.float64)
    lor = (eta / np.pi) / ((omega[:, None] - eps[None, :]) ** 2 + eta ** 2)
    occ = np.arange(L) < n_occ
    return (lor[:, occ] * amp2[occ]).sum(axis=1), (lor[:, ~occ] * amp2[~occ]).sum(axis=1)


def superblock_ldos_inputs(model, Sp, Ep, L_k, i, spin, couplings_batch=None):
    """For site i of S' (block-local operator c_i, Jordan-Wigner string inside
    S'; the full-lattice c_i is c_i (x) 1 because E' holds the higher labels):
    the superblocks of the N - 1 and N + 1 targets on the same S', E' and the
    transition containers of c_i (x) 1 (N -> N - 1) and c_i^dag (x) 1
    (N -> N + 1).  Returns {"hole": (sb, trans), "particle": (sb, trans)}."""
    Q = model.target(L_k)
    c = odmrg._ops_of(Sp, i)["c_" + spin]
    dq = 1 if spin == "up" else model.Q
    terms, names, tcls, tmult = odmrg.superblock_terms(model, Sp, Ep, L_k)
    classes = model.classes()
    if couplings_batch is None:
        couplings_batch = [[model.couplings[k] for k in classes]]
    g = np.atleast_2d(np.asarray(couplings_batch, dtype=np.float64))
    tci = np.array([classes.index(k) for k in tcls])
    coeffs = g[:, tci] * np.array(tmult)[None, :]
    secs_in = osb.target_sectors(Sp.q, Ep.q, Q)
    out = {}
    for part, A, Qo in (("hole", c, Q - dq), ("particle", c.T, Q + dq)):
        sb = osb.superblock_from_full(Sp.q, Ep.q, Qo, terms, coeffs[0], names)
        sb.coeffs = coeffs
        secs_out = osb.target_sectors(Sp.q, Ep.q, Qo)
        blocks = []
        for so, (_, iSo, iEo) in enumerate(secs_out):
            for si, (_, iSi, iEi) in enumerate(secs_in):
                if len(iEo) != len(iEi) or np.any(iEo != iEi):
                    continue
                a = A[np.ix_(iSo, iSi)]
                if np.any(a):
                    blocks.append((so, si, a, np.eye(len(iEo))))
        tr = transition([len(s[1]) for s in secs_out], [len(s[2]) for s in secs_out],
                        [len(s[1]) for s in secs_in], [len(s[2]) for s in secs_in], blocks,
                        batch=g.shape[0], name=("c" if part == "hole" else "c+") + f"_{i}{spin}")
        out[part] = (sb, tr)
    return out
