"""Pins of the oracle's local density of states (continued fraction of the
Lanczos coefficients; paper Sec. "DmrgSolver and the infinite DMRG algorithm"
and its closing notes on the continued-fraction method).

* the continued fraction of a full Krylov space is the resolvent from the
  spectral decomposition (random symmetric matrix: nothing of the model);
* U = 0: exact diagonalisation gives the free-fermion closed form
  sum_k |phi_k(i)|^2 Lorentzian(w - eps_k);
* sum rule: |c psi|^2 + |c^dag psi|^2 = 1 and the LDOS integrates to 1;
* the DMRG superblock route (c_i (x) 1 between the N and N -/+ 1 targets on
  the same S', E', Lanczos on the N -/+ 1 superblock, continued fraction)
  equals exact diagonalisation when nothing is truncated.
"""
import numpy as np
import pytest

from oracle import dmrg, ldos
from oracle import superblock as osb
from workloads.superblock import seeded_normal

OMEGA = np.linspace(-5.0, 5.0, 201)
ETA = 0.1


def test_full_krylov_fraction_is_the_resolvent():
    rng = np.random.default_rng(3)
    n = 40
    M = rng.standard_normal((n, n))
    H = 0.5 * (M + M.T)
    v = rng.standard_normal(n)
    norm2, a, b = ldos.lanczos_coefficients(lambda x: H @ x, v, n)
    assert len(a) == n and len(b) == n - 1 and norm2 == pytest.approx(v @ v)
    w, U = np.linalg.eigh(H)
    z = np.linspace(-6, 6, 97) + 0.05j
    g_cf = ldos.continued_fraction(norm2, a, b, z)
    g_ex = ldos.spectral_sum(w, (U.T @ v) ** 2, z)
    assert np.max(np.abs(g_cf - g_ex)) <= 1e-9 * np.max(np.abs(g_ex))


def test_invariant_subspace_stops_early():
    H = np.diag([1.0, 2.0, 3.0, 4.0, 5.0])
    v = np.array([1.0, 1.0, 0.0, 0.0, 0.0])
    norm2, a, b = ldos.lanczos_coefficients(lambda x: H @ x, v, 5)
    assert len(a) == 2 and len(b) == 1
    z = np.array([0.3 + 0.2j, 2.5 + 0.1j])
    assert np.allclose(ldos.continued_fraction(norm2, a, b, z), 1 / (z - 1) + 1 / (z - 2))


@pytest.mark.parametrize("i,spin", [(0, "up"), (2, "dn"), (5, "up")])
def test_free_fermions_closed_form(i, spin):
    L = 6
    h, p, e0 = ldos.hubbard_ldos_ed(L, i, spin, L // 2, L // 2, 1.0, 0.0, OMEGA, ETA)
    fh, fp = ldos.free_chain_ldos(L, i, L // 2, 1.0, OMEGA, ETA)
    assert np.max(np.abs(h - fh)) < 1e-12 and np.max(np.abs(p - fp)) < 1e-12
    eps = -2 * np.cos(np.arange(1, L + 1) * np.pi / (L + 1))
    assert e0 == pytest.approx(2 * np.sort(eps)[: L // 2].sum(), abs=1e-12)


def test_sum_rule():
    L = 6
    w = np.linspace(-60, 60, 240001)
    h, p, _ = ldos.hubbard_ldos_ed(L, 1, "up", L // 2, L // 2, 1.0, 4.0, w, 0.05)
    total = np.trapezoid(h + p, w)
    assert total == pytest.approx(1.0, abs=2e-3)  # Lorentzian tails beyond the window
    # half filling, particle-hole symmetric chain: <n_i up> = 1/2
    assert np.trapezoid(h, w) == pytest.approx(0.5, abs=2e-3)


@pytest.mark.parametrize("spin", ["up", "dn"])
def test_superblock_route_equals_ed(spin):
    L, U = 6, 2.0
    model = dmrg.hubbard_chain(1.0, U, Lmax=L)
    steps, _, _ = dmrg.infinite_dmrg(model, L, m=1000, keep_superblocks=True)
    last = steps[-1]
    Sp, Ep = last.blocks
    i = Sp.n - 1
    h_ed, p_ed, e0 = ldos.hubbard_ldos_ed(L, i, spin, L // 2, L // 2, 1.0, U, OMEGA, ETA)
    assert last.energy == pytest.approx(e0, abs=1e-10)
    inp = ldos.superblock_ldos_inputs(model, Sp, Ep, last.L, i, spin)
    cf = {}
    for part in ("hole", "particle"):
        sb, tr = inp[part]
        tr.validate()
        sb.validate()
        n_out = tr.meta["dim_out"]
        y = osb.apply_H(tr, np.concatenate([np.zeros(n_out), last.psi]))
        assert np.all(y[n_out:] == 0.0)
        cf[part] = ldos.lanczos_coefficients(lambda v: osb.apply_H(sb, v), y[:n_out], sb.dim)
    assert cf["hole"][0] + cf["particle"][0] == pytest.approx(1.0, abs=1e-12)
    h, p = ldos.ldos_from_fractions(cf["hole"], cf["particle"], last.energy, OMEGA, ETA)
    assert np.max(np.abs(h - h_ed)) < 1e-9 and np.max(np.abs(p - p_ed)) < 1e-9


def test_transition_container_layout():
    from workloads.superblock import transition
    r_out, c_out, r_in, c_in = [2, 3], [4, 1], [3, 2], [1, 4]
    A = seeded_normal(1, (2, 2))
    tr = transition(r_out, c_out, r_in, c_in, [(0, 1, A, np.eye(4))], batch=2)
    tr.validate()
    assert tr.n_sectors == 4 and tr.batch == 2 and tr.meta["dim_out"] == 11
    x = np.concatenate([np.zeros(11), seeded_normal(2, 3 + 8)])
    y = osb.apply_H(tr, x)
    off = tr.offsets()
    psi_in = x[off[3]:off[4]].reshape(2, 4)
    assert np.allclose(y[off[0]:off[1]].reshape(2, 4), A @ psi_in)
    assert np.all(y[off[1]:] == 0.0)


def test_grown_inputs_equal_ed():
    """The bench's input builder (isometry-grown blocks; here nothing is
    truncated) gives the N, N - 1 and N + 1 superblocks and the c (x) 1
    transitions on one growth: its densities equal exact diagonalisation."""
    from oracle import lanczos as olz
    from workloads.grown import grown_ldos_inputs
    L, U = 6, 2.0
    inp = grown_ldos_inputs(L, "chain", 3, 3, m=1000, cut=3, U_values=[U])
    sbN = inp["N"]
    r = olz.lanczos_ground(lambda v: osb.apply_H(sbN, v), seeded_normal(0, sbN.dim), tol=1e-12, max_iter=400)
    h_ed, p_ed, e0 = ldos.hubbard_ldos_ed(L, inp["site"], "up", 3, 3, 1.0, U, OMEGA, ETA)
    assert r.e0 == pytest.approx(e0, abs=1e-10)
    cf = {}
    for part in ("hole", "particle"):
        sb, tr = inp[part]
        tr.validate()
        sb.validate()
        n_out = tr.meta["dim_out"]
        y = osb.apply_H(tr, np.concatenate([np.zeros(n_out), r.psi]))
        cf[part] = ldos.lanczos_coefficients(lambda v: osb.apply_H(sb, v), y[:n_out], sb.dim)
    h, p = ldos.ldos_from_fractions(cf["hole"], cf["particle"], r.e0, OMEGA, ETA)
    assert np.max(np.abs(h - h_ed)) < 1e-9 and np.max(np.abs(p - p_ed)) < 1e-9
