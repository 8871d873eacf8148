"""Superblock Hamiltonian: explicit Kronecker form and sector-blocked product.

Paper Sec. 3.3: for operators A on S' and B on E', (A (x) B) has entries
C[(a1,b1),(a2,b2)] = A[a1,a2] B[b1,b2], and the superblock basis is reordered
by effective quantum number (Sec. 3.2) so that H is block diagonal in q.
The Lanczos solver only needs x += H y (Sec. 3.3), done by the model in three
tasks: (i) x += H_system y, (ii) x += H_environment y, (iii) x += H_connection y.

Two independent forms are kept here so that each checks the other:

* ``explicit_H``: the plain definition.  Build sum_k c_k kron(A_k, B_k) over
  the whole S' (x) E' space and keep the rows and columns of the target
  sector, in the flat order of the wavefunction.
* ``apply_H``: the method.  With psi split into row-major blocks Psi_s of
  shape r_s x c_s, each (term, sector pair) acts as
  Y[s_out] += c_k * A_k[s_out,s_in] @ Psi[s_in] @ B_k[s_out,s_in].T,
  because (A (x) B) vec(Psi) = vec(A Psi B^T) for row-major vec.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads.superblock import Pair, Superblock


def target_sectors(qS, qE, Q):
    """Sectors of the target space: for each distinct q of S' (increasing),
    the S' states with that q and the E' states with Q - q (both in basis
    order).  Sectors where either side is empty are dropped."""
    qS = np.asarray(qS)
    qE = np.asarray(qE)
    out = []
    for q in sorted(set(qS.tolist())):
        iS = np.nonzero(qS == q)[0]
        iE = np.nonzero(qE == Q - q)[0]
        if len(iS) and len(iE):
            out.append((q, iS, iE))
    return out


def flat_index(qS, qE, Q):
    dimE = len(qE)
    idx = []
    for (q, iS, iE) in target_sectors(qS, qE, Q):
        idx.append((iS[:, None] * dimE + iE[None, :]).ravel())
    return np.concatenate(idx) if idx else np.zeros(0, dtype=np.int64)


def explicit_H(qS, qE, Q, terms, coeffs):
    """sum_k coeffs[k] kron(A_k, B_k) restricted to the target sector.
    ``terms`` is a list of (A_full or None, B_full or None); None = identity."""
    dS, dE = len(qS), len(qE)
    H = sp.csr_matrix((dS * dE, dS * dE))
    for (A, B), ck in zip(terms, coeffs):
        Am = sp.identity(dS, format="csr") if A is None else sp.csr_matrix(A)
        Bm = sp.identity(dE, format="csr") if B is None else sp.csr_matrix(B)
        H = H + ck * sp.kron(Am, Bm, format="csr")
    idx = flat_index(qS, qE, Q)
    return H[idx][:, idx]


def superblock_from_full(qS, qE, Q, terms, coeffs, names=None, zero_tol=0.0,
                         **extra) -> Superblock:
    """Cut full S' and E' operators into the sector blocks that the blocked
    product uses.  A pair is kept when both of its blocks have a nonzero entry
    (identity blocks always count as nonzero)."""
    secs = target_sectors(qS, qE, Q)
    r = np.array([len(s[1]) for s in secs])
    c = np.array([len(s[2]) for s in secs])
    pairs = []
    for k, (A, B) in enumerate(terms):
        for so, (_, iSo, iEo) in enumerate(secs):
            for si, (_, iSi, iEi) in enumerate(secs):
                if A is None:
                    if so != si:
                        continue
                    a = None
                else:
                    a = np.asarray(A[np.ix_(iSo, iSi)], dtype=np.float64)
                    if not np.any(np.abs(a) > zero_tol):
                        continue
                if B is None:
                    if so != si:
                        continue
                    b = None
                else:
                    b = np.asarray(B[np.ix_(iEo, iEi)], dtype=np.float64)
                    if not np.any(np.abs(b) > zero_tol):
                        continue
                pairs.append(Pair(k, so, si, a, b))
    sb = Superblock(r, c, np.atleast_2d(coeffs), pairs, list(names or []), **extra)
    sb.q_labels = np.array([s[0] for s in secs])
    return sb


def _blocks(sb: Superblock, v):
    off = sb.offsets()
    return [v[off[s]:off[s + 1]].reshape(sb.r[s], sb.c[s]) for s in range(sb.n_sectors)]


def apply_H(sb: Superblock, psi, b: int = 0):
    """y = H psi with the blocked rule Y[s_out] += c_k A Psi[s_in] B^T (paper
    Sec. 3.3, the on-the-fly superblock product; identity sides skipped)."""
    psi = np.asarray(psi, dtype=np.float64)
    X = _blocks(sb, psi)
    y = np.zeros(sb.dim)
    Y = _blocks(sb, y)
    for p in sb.pairs:
        T = X[p.s_in]
        if p.A is not None:
            T = p.A @ T
        if p.B is not None:
            T = T @ p.B.T
        Y[p.s_out] += sb.coeffs[b, p.term] * T
    return y


def apply_HT(sb: Superblock, g, b: int = 0):
    """H^T g: each pair contributes c_k A^T G[s_out] B to sector s_in."""
    G = _blocks(sb, np.asarray(g, dtype=np.float64))
    out = np.zeros(sb.dim)
    O = _blocks(sb, out)
    for p in sb.pairs:
        T = G[p.s_out]
        if p.A is not None:
            T = p.A.T @ T
        if p.B is not None:
            T = T @ p.B
        O[p.s_in] += sb.coeffs[b, p.term] * T
    return out


def term_products(sb: Superblock, g, psi):
    """d_k = <g, (A_k (x) B_k) psi> for every term k (no coefficient)."""
    G = _blocks(sb, np.asarray(g, dtype=np.float64))
    X = _blocks(sb, np.asarray(psi, dtype=np.float64))
    d = np.zeros(sb.n_terms)
    for p in sb.pairs:
        T = X[p.s_in]
        if p.A is not None:
            T = p.A @ T
        if p.B is not None:
            T = T @ p.B.T
        d[p.term] += float(np.sum(G[p.s_out] * T))
    return d


def dense_H(sb: Superblock, b: int = 0):
    """The D x D matrix of the blocked rule, one column per unit vector
    (tiny superblocks only)."""
    D = sb.dim
    M = np.zeros((D, D))
    e = np.zeros(D)
    for j in range(D):
        e[:] = 0.0
        e[j] = 1.0
        M[:, j] = apply_H(sb, e, b)
    return M


def matvec_flops(sb: Superblock) -> int:
    """Algorithmic flops of one product for one batch member, counting every
    stored block as dense and each two-GEMM pair in its cheaper order:
    min(2 r_o r_i c_i + 2 r_o c_i c_o, 2 r_i c_i c_o + 2 r_o r_i c_o)."""
    r, c = sb.r, sb.c
    f = 0
    for p in sb.pairs:
        ro, ri, co, ci = int(r[p.s_out]), int(r[p.s_in]), int(c[p.s_out]), int(c[p.s_in])
        if p.A is None:
            f += 2 * ro * ci * co
        elif p.B is None:
            f += 2 * ro * ri * co
        else:
            f += min(2 * ro * ri * ci + 2 * ro * ci * co, 2 * ri * ci * co + 2 * ro * ri * co)
    return f
