"""Pins for the oracle's lattice models and exact diagonalisation."""
import os

import numpy as np
import pytest

from oracle import ed, models
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_two_site_singlet():
    # S_1.S_2 on two spins: singlet energy -3J/4
    assert ed.heisenberg_ed(2) == pytest.approx(-0.75, abs=1e-14)


def test_heisenberg_four_sites_closed_form():
    # open 4-site chain: E0 = -(3 + 2 sqrt 3)/4 (characteristic polynomial of the S=0 sector)
    assert ed.heisenberg_ed(4) == pytest.approx(-(3 + 2 * np.sqrt(3)) / 4, abs=1e-12)


@pytest.mark.parametrize("L", [6, 8, 10])
def test_heisenberg_vs_bit_basis(L):
    bonds = [(i, i + 1, 1.0) for i in range(L - 1)]
    assert ed.heisenberg_ed(L) == pytest.approx(bf.lowest(bf.heisenberg_matrix(L, bonds, L // 2)), abs=1e-11)


@pytest.mark.parametrize("L,J2", [(8, 0.25), (10, 0.4)])
def test_j1j2_vs_bit_basis(L, J2):
    bonds = [(i, i + 1, 1.0) for i in range(L - 1)] + [(i, i + 2, J2) for i in range(L - 2)]
    ref = bf.lowest(bf.heisenberg_matrix(L, bonds, L // 2))
    assert ed.heisenberg_ed(L, J1=1.0, J2=J2) == pytest.approx(ref, abs=1e-11)


@pytest.mark.parametrize("L", [8, 12])
def test_majumdar_ghosh_point(L):
    # J2 = J1/2, open chain with even L: the dimer product state is exact, E0 = -3 L J1 / 8
    assert ed.heisenberg_ed(L, J1=1.0, J2=0.5) == pytest.approx(-3 * L / 8, abs=1e-10)


@pytest.mark.parametrize("L", [2, 4, 6, 8])
def test_hubbard_free_fermions(L):
    # U = 0: E0 = 2 * sum of the L/2 lowest eps_k = -2 cos(k pi / (L+1)), k = 1..L
    eps = np.sort(-2 * np.cos(np.arange(1, L + 1) * np.pi / (L + 1)))
    assert ed.hubbard_ed(L, L // 2, L // 2, t=1.0, U=0.0) == pytest.approx(2 * eps[: L // 2].sum(), abs=1e-11)


@pytest.mark.parametrize("U", [1.0, 4.0, 8.0])
def test_hubbard_dimer_closed_form(U):
    # two sites, one up + one down electron: E0 = U/2 - sqrt(U^2/4 + 4 t^2)
    assert ed.hubbard_ed(2, 1, 1, t=1.0, U=U) == pytest.approx(U / 2 - np.sqrt(U * U / 4 + 4), abs=1e-12)


@pytest.mark.parametrize("L,nu,nd,U", [(4, 2, 2, 4.0), (6, 3, 3, 4.0), (6, 2, 3, 8.0)])
def test_hubbard_vs_bit_basis(L, nu, nd, U):
    bonds = [(i, i + 1, 1.0) for i in range(L - 1)]
    ref = bf.lowest(bf.hubbard_matrix(L, bonds, U, nu, nd))
    assert ed.hubbard_ed(L, nu, nd, t=1.0, U=U) == pytest.approx(ref, abs=1e-11)


def test_hubbard_ladder_vs_bit_basis():
    L = 6
    bonds = [(i, j, 1.0) for (i, j, _) in models.ladder_bonds(L)]
    ref = bf.lowest(bf.hubbard_matrix(L, bonds, 8.0, 3, 2))
    assert ed.hubbard_ed(L, 3, 2, t=1.0, U=8.0, geometry="ladder") == pytest.approx(ref, abs=1e-11)


def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "paper_test_run_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                L, e, nd = line.split()
                rows.append((int(L), float(e), int(nd)))
    return rows


@pytest.mark.parametrize("row", [r for r in _golden() if r[0] <= 8])
def test_hubbard_u1_matches_paper_test_run(row):
    # the paper prints the test-run energies to 5 decimals (Sec. Test Run, Note1)
    L, e, nd = row
    E = ed.hubbard_ed(L, L // 2, L // 2, t=1.0, U=1.0)
    assert abs(E - e) <= 0.5 * 10.0 ** (-nd) + 1e-12
