"""Pins for the oracle's Lanczos solver, DMRG driver and energy gradients."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dmrg, ed
from oracle import grad as ograd
from oracle import lanczos as olz
from oracle import superblock as osb
from tests import bruteforce as bf
from workloads.superblock import seeded_normal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("D,seed", [(1, 0), (7, 1), (300, 2), (2000, 3)])
def test_lanczos_matches_dense_eigh(D, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((D, D))
    M = M + M.T
    ref = np.linalg.eigvalsh(M)[0]
    res = olz.lanczos_ground(lambda v: M @ v, seeded_normal(seed, D), tol=1e-12, max_iter=D)
    assert res.converged
    assert res.e0 == pytest.approx(ref, abs=1e-12 * max(1, abs(ref)))
    th, rr = olz.rayleigh(lambda v: M @ v, res.psi)
    assert rr < 1e-9 * max(1, abs(ref))


def test_lanczos_breakdown_on_invariant_subspace():
    # start vector inside a 3-dimensional invariant subspace: exact after 3 steps
    M = np.diag([3.0, -1.0, 2.0, 5.0, -7.0, 9.0])
    v0 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    res = olz.lanczos_ground(lambda v: M @ v, v0, tol=1e-14)
    assert res.iters == 3 and res.breakdown
    assert res.e0 == pytest.approx(-1.0, abs=1e-14)


def test_tridiag_lowest_against_dense():
    rng = np.random.default_rng(0)
    a, b = rng.standard_normal(50), rng.standard_normal(49)
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    w, s = olz.tridiag_lowest(a, b)
    assert w == pytest.approx(np.linalg.eigvalsh(T)[0], abs=1e-13)
    assert np.allclose(T @ s, w * s, atol=1e-12)


def test_infinite_dmrg_without_truncation_is_exact():
    model = dmrg.heisenberg_chain()
    steps, _, _ = dmrg.infinite_dmrg(model, 10, m=10**6)
    for st in steps:
        bonds = [(i, i + 1, 1.0) for i in range(st.L - 1)]
        assert st.energy == pytest.approx(bf.lowest(bf.heisenberg_matrix(st.L, bonds, st.L // 2)), abs=1e-10)
        assert st.eps_S == pytest.approx(0.0, abs=1e-12)


def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "paper_test_run_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                L, e, nd = line.split()
                rows.append((int(L), float(e), int(nd)))
    return rows


def test_paper_test_run_energies():
    """The paper's test run (m = 64, density 1) prints four energies to five
    decimals; the infinite algorithm on the U = 1 Hubbard chain reproduces all."""
    model = dmrg.hubbard_chain(t=1.0, U=1.0, density=1.0)
    steps, _, _ = dmrg.infinite_dmrg(model, 10, m=64)
    got = {st.L: st.energy for st in steps}
    for (L, e, nd) in _golden():
        assert abs(got[L] - e) <= 0.5 * 10.0 ** (-nd) + 1e-12, (L, got[L], e)


@pytest.mark.slow
def test_heisenberg_16_sites_m32_finite():
    """Heisenberg chain L = 16, m = 32, infinite + 2 finite sweeps: variational
    (E_DMRG >= E_exact, W^T W = 1) and within the truncation error of exact."""
    bonds = [(i, i + 1, 1.0) for i in range(15)]
    exact = -6.911737145575
    # pin of the quoted exact value itself, by a bit-basis Lanczos (no oracle code)
    H = bf.heisenberg_matrix(16, bonds, 8)
    w = sla.eigh(H, eigvals_only=True, subset_by_index=(0, 0))[0]
    assert w == pytest.approx(exact, abs=1e-10)
    model = dmrg.heisenberg_chain()
    out = dmrg.finite_dmrg(model, 16, m=32, n_sweeps=2)
    fin = [st for st in out if st.L == 16]
    e_last = fin[-1].energy
    assert all(st.energy >= exact - 1e-10 for st in out if st.L == 16)
    assert e_last - exact < 2e-4
    # sweeps lower the energy at the middle split
    mids = [st.energy for st in fin if st.nS == 8]
    assert mids[-1] <= mids[0] + 1e-9


def _j1j2_superblock(L, J1, J2):
    model = dmrg.heisenberg_chain(J1, J2)
    S = dmrg.site_block(model)
    E = dmrg.site_block(model)
    for _ in range(L // 2 - 1):
        S = dmrg.grow(model, S, "left")
        E = dmrg.grow(model, E, "right")
    sb, _ = dmrg.make_superblock(model, S, E, L)
    return sb


@pytest.mark.parametrize("J2", [0.25, 0.5])
def test_hellmann_feynman_j1j2(J2):
    """dE0/dJ via Hellmann-Feynman on an untruncated J1-J2 superblock:
    Euler identity E0 = J1 dE/dJ1 + J2 dE/dJ2 (H is homogeneous of degree 1),
    agreement with central differences of exact energies, and the
    Majumdar-Ghosh values dE/dJ2 = 0, dE/dJ1 = -3L/8 at J2 = J1/2."""
    L = 10
    sb = _j1j2_superblock(L, 1.0, J2)
    res = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), seeded_normal(0, sb.dim), tol=1e-13)
    dEdc = ograd.hf_grad(sb, res.psi)
    g = ograd.coupling_grad(sb, dEdc)  # classes J1, J2
    assert res.e0 == pytest.approx(1.0 * g[0] + J2 * g[1], abs=1e-10)

    def E(x):
        bonds = [(i, i + 1, x[0]) for i in range(L - 1)] + [(i, i + 2, x[1]) for i in range(L - 2)]
        return bf.lowest(bf.heisenberg_matrix(L, bonds, L // 2))
    fd = ograd.central_fd(E, [1.0, J2], h=1e-5)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-7)
    if J2 == 0.5:
        assert g[1] == pytest.approx(0.0, abs=1e-9)
        assert g[0] == pytest.approx(-3 * L / 8, abs=1e-9)
