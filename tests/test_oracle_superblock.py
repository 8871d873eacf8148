"""Pins for the oracle's superblock: the blocked product against the explicit
Kronecker definition, symmetry, and exactness against whole-lattice ED."""
import numpy as np
import pytest

from oracle import dmrg, ed
from oracle import superblock as osb
from oracle import grad as ograd
from workloads.superblock import seeded_normal
from workloads.synthetic import random_sectored, ragged_small


def _dmrg_superblock(model, nS, nE, m=10**6):
    """Untruncated S' = first nS sites, E' = last nE sites of an (nS+nE)-site lattice."""
    S = dmrg.site_block(model)
    for _ in range(nS - 1):
        S = dmrg.grow(model, S, "left")
    E = dmrg.site_block(model)
    for _ in range(nE - 1):
        E = dmrg.grow(model, E, "right")
    sb, terms = dmrg.make_superblock(model, S, E, nS + nE)
    return sb, terms, S, E


CASES = [
    ("heis", lambda: dmrg.heisenberg_chain(), 3, 3),
    ("j1j2", lambda: dmrg.heisenberg_chain(1.0, 0.35), 4, 4),
    ("hub", lambda: dmrg.hubbard_chain(1.0, 4.0), 2, 3),
    ("ladder", lambda: dmrg.hubbard_ladder(1.0, 0.7, 6.0), 3, 3),
]


@pytest.mark.parametrize("name,mk,nS,nE", CASES)
def test_blocked_equals_explicit_kron(name, mk, nS, nE):
    model = mk()
    sb, terms, S, E = _dmrg_superblock(model, nS, nE)
    H = osb.explicit_H(S.q, E.q, model.target(nS + nE), terms, sb.coeffs[0])
    x = seeded_normal(3, sb.dim)
    assert np.allclose(osb.apply_H(sb, x), H @ x, atol=1e-13, rtol=0)
    # H is symmetric, and the transpose product agrees with H^T
    y = seeded_normal(4, sb.dim)
    assert abs(x @ osb.apply_H(sb, y) - osb.apply_H(sb, x) @ y) < 1e-11
    assert np.allclose(osb.apply_HT(sb, x), H.T @ x, atol=1e-13, rtol=0)


@pytest.mark.parametrize("name,L,nS", [("heis", 6, 3), ("hub", 4, 2), ("hub", 5, 3), ("j1j2", 8, 4), ("ladder", 6, 3)])
def test_untruncated_superblock_is_the_lattice(name, L, nS):
    """With no truncation (paper Sec. 1: m >= #V(S') keeps everything) the
    superblock ground energy is the whole-lattice ED energy."""
    if name == "heis":
        model, ref = dmrg.heisenberg_chain(), ed.heisenberg_ed(L)
    elif name == "j1j2":
        model, ref = dmrg.heisenberg_chain(1.0, 0.3), ed.heisenberg_ed(L, J1=1.0, J2=0.3)
    elif name == "hub":
        model = dmrg.hubbard_chain(1.0, 4.0, density=1.0)
        N = L - L % 2
        ref = ed.hubbard_ed(L, N // 2, N // 2, 1.0, 4.0)
    else:
        model = dmrg.hubbard_ladder(1.0, 1.0, 8.0)
        ref = ed.hubbard_ed(L, L // 2, L // 2, 1.0, 8.0, geometry="ladder")
    sb, terms, S, E = _dmrg_superblock(model, nS, L - nS)
    M = osb.dense_H(sb)
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M)[0] == pytest.approx(ref, abs=1e-10)


def _full_ops_from_blocks(sb, k):
    """Rebuild the full S' and E' operators of term k from its blocks; sector s
    has q_S = s and q_E = Q - s with Q = n_sectors (test-side construction)."""
    r, c = sb.r, sb.c
    oR = np.concatenate([[0], np.cumsum(r)])
    oC = np.concatenate([[0], np.cumsum(c)])
    A = np.zeros((oR[-1], oR[-1]))
    B = np.zeros((oC[-1], oC[-1]))
    ida = idb = False
    for p in sb.pairs:
        if p.term != k:
            continue
        if p.A is None:
            ida = True
        else:
            A[oR[p.s_out]:oR[p.s_out + 1], oR[p.s_in]:oR[p.s_in + 1]] = p.A
        if p.B is None:
            idb = True
        else:
            B[oC[p.s_out]:oC[p.s_out + 1], oC[p.s_in]:oC[p.s_in + 1]] = p.B
    return (None if ida else A), (None if idb else B)


def _explicit_from_blocks(sb, b=0):
    S = sb.n_sectors
    qS = np.repeat(np.arange(S), sb.r)
    qE = np.repeat(S - np.arange(S), sb.c)
    terms = []
    for k in range(sb.n_terms):
        A, B = _full_ops_from_blocks(sb, k)
        # a term whose pairs each reuse one (A, B) pair per sector pair is a
        # single kron only if no two pairs share a row/column range pattern
        terms.append((A, B))
    return osb.explicit_H(qS, qE, S, terms, sb.coeffs[b])


def test_blocked_equals_explicit_on_ragged_random():
    # every pair of one term has a distinct (s_out, s_in), so the term is the
    # single kron product of its full operators restricted to the target sector
    sb = ragged_small(seed=5, batch=2, tiny=True)
    sb.validate()
    for b in range(2):
        H = _explicit_from_blocks(sb, b)
        x = seeded_normal(11 + b, sb.dim)
        y = H @ x
        tol = 1e-13 * np.abs(y).max()
        assert np.abs(osb.apply_H(sb, x, b) - y).max() <= tol
        assert np.abs(osb.apply_HT(sb, x, b) - H.T @ x).max() <= tol


def test_blocked_equals_explicit_random_sectored_small():
    sb = random_sectored(seed=2, n_sectors=6, dmin=1, dmax=9, identity_terms=True)
    H = _explicit_from_blocks(sb)
    x = seeded_normal(5, sb.dim)
    assert np.allclose(osb.apply_H(sb, x), H @ x, atol=1e-12, rtol=0)


def test_term_products_and_backward_are_exact_derivatives():
    sb = ragged_small(seed=7)
    psi = seeded_normal(1, sb.dim)
    g = seeded_normal(2, sb.dim)
    dpsi, dc = ograd.apply_H_backward(sb, psi, g)
    # L(psi, c) = <g, H(c) psi> is bilinear: its derivative is its own slope
    L0 = g @ osb.apply_H(sb, psi)
    assert L0 == pytest.approx(float(dc @ sb.coeffs[0]), rel=1e-12)
    for k in range(sb.n_terms):
        c2 = sb.coeffs.copy()
        c2[0, k] += 1.0
        assert g @ osb.apply_H(sb.with_coeffs(c2), psi) - L0 == pytest.approx(dc[k], rel=1e-10, abs=1e-10)
    e = np.zeros(sb.dim)
    for j in range(0, sb.dim, 37):
        e[:] = 0
        e[j] = 1.0
        assert g @ osb.apply_H(sb, e) == pytest.approx(dpsi[j], rel=1e-12, abs=1e-12)


def test_empty_and_uncoupled_sectors_stay_zero():
    sb = ragged_small(seed=3)
    y = osb.apply_H(sb, seeded_normal(0, sb.dim))
    off = sb.offsets()
    assert np.all(y[off[6]:off[7]] == 0.0)  # sector 6 has no contributing term
    assert sb.r[3] * sb.c[3] == 0 and sb.r[4] * sb.c[4] == 0


def test_matvec_flops_hand_counted():
    """Algorithmic flop count pinned by hand on a 2-sector superblock:
    r = (2, 3), c = (4, 5); a multiply-add is 2 flops, blocks dense.

    * term 0, A (x) 1 on sector 0: A (2x2) times Psi_0 (2x4): 2*2*2*4 = 32
    * term 1, 1 (x) B on sector 1: Psi_1 (3x5) times B^T (5x5): 2*3*5*5 = 150
    * term 2, sector 1 -> 0, A (2x3), B (4x5):
        (A Psi_1) B^T: 2*2*3*5 + 2*2*5*4 = 60 + 80 = 140
        A (Psi_1 B^T): 2*3*5*4 + 2*2*3*4 = 120 + 48 = 168  -> 140
    * term 3, sector 0 -> 1, A (3x2), B (5x4):
        (A Psi_0) B^T: 2*3*2*4 + 2*3*4*5 = 48 + 120 = 168
        A (Psi_0 B^T): 2*2*4*5 + 2*3*2*5 = 80 + 60 = 140   -> 140
    total 32 + 150 + 140 + 140 = 462 per member.
    """
    from workloads.superblock import Pair, Superblock
    rng = np.random.default_rng(0)
    pairs = [Pair(0, 0, 0, rng.standard_normal((2, 2)), None),
             Pair(1, 1, 1, None, rng.standard_normal((5, 5))),
             Pair(2, 0, 1, rng.standard_normal((2, 3)), rng.standard_normal((4, 5))),
             Pair(3, 1, 0, rng.standard_normal((3, 2)), rng.standard_normal((5, 4)))]
    sb = Superblock([2, 3], [4, 5], np.ones((1, 4)), pairs)
    assert osb.matvec_flops(sb) == 462
    # each pair alone, with the order the count picks
    for p, want in zip(pairs, (32, 150, 140, 140)):
        assert osb.matvec_flops(Superblock([2, 3], [4, 5], np.ones((1, 4)), [p])) == want
    # and the product the count describes is the blocked rule itself
    x = rng.standard_normal(sb.dim)
    y = osb.apply_H(sb, x)
    X0, X1 = x[:8].reshape(2, 4), x[8:].reshape(3, 5)
    y0 = pairs[0].A @ X0 + pairs[2].A @ X1 @ pairs[2].B.T
    y1 = X1 @ pairs[1].B.T + pairs[3].A @ X0 @ pairs[3].B.T
    assert np.allclose(y, np.concatenate([y0.ravel(), y1.ravel()]), rtol=0, atol=1e-13)
