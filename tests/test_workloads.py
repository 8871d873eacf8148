"""Checks of the seeded input generators (not the oracle): the isometry-grown
superblocks are exact projections of the lattice Hamiltonian."""
import numpy as np
import pytest

from oracle import ed
from oracle import superblock as osb
from workloads.grown import grown_hubbard_superblock
from workloads.superblock import Superblock, seeded_normal
from workloads.synthetic import random_sectored, ragged_small


@pytest.mark.parametrize("geom,L,nu,nd,cut", [("ladder", 8, 3, 3, 4), ("ladder", 6, 3, 2, 3), ("chain", 6, 3, 3, 3)])
def test_grown_untruncated_is_exact(geom, L, nu, nd, cut):
    sb = grown_hubbard_superblock(L, geom, nu, nd, m=10**6, cut=cut, U_values=[8.0, 3.0])
    sb.validate()
    for b, U in enumerate([8.0, 3.0]):
        M = osb.dense_H(sb, b)
        assert np.allclose(M, M.T, atol=1e-12)
        ref = ed.hubbard_ed(L, nu, nd, t=1.0, U=U, geometry=geom)
        assert np.linalg.eigvalsh(M)[0] == pytest.approx(ref, abs=1e-10)


def test_grown_truncated_is_variational():
    L, nu, nd = 8, 3, 3
    sb = grown_hubbard_superblock(L, "ladder", nu, nd, m=12, cut=4, U_values=[8.0])
    M = osb.dense_H(sb)
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(M)[0] >= ed.hubbard_ed(L, nu, nd, 1.0, 8.0, geometry="ladder") - 1e-10


def test_npz_roundtrip(tmp_path):
    sb = ragged_small(seed=2, batch=3)
    p = tmp_path / "sb.npz"
    sb.save(str(p))
    sb2 = Superblock.load(str(p))
    x = seeded_normal(0, sb.dim)
    for b in range(3):
        assert np.array_equal(osb.apply_H(sb, x, b), osb.apply_H(sb2, x, b))


def test_random_sectored_shape():
    sb = random_sectored(seed=0)
    assert sb.n_sectors == 64 and sb.n_terms == 12 and len(sb.pairs) == 760
    assert sb.r.min() >= 16 and sb.r.max() <= 512
