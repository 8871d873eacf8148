"""The DMRG step on the device (paper Sec. 3.1, Fig. infiniteloop): block
growth with the operators in the product basis, superblock assembly, the
Lanczos ground state, the density matrices rho_S = Psi Psi^T and
rho_E = Psi^T Psi (Eqs. rhoSystem, rhoEnviron), batched symmetric
eigensolves, the global choice of the m most probable states, and the change
of basis W^T O W (Eq. transformation) -- through the C ABI (dmrg_sys_*)
against the oracle's DMRG driver and exact results.

* Without truncation (m >= every block dimension) each infinite step is the
  exact ground state of its lattice: energies equal exact diagonalisation
  to 1e-10.
* The paper's test run (U = 1 Hubbard chain, m = 64): the four printed
  energies to their five decimals.
* With truncation, the trajectories of the two drivers (same tie rule:
  eigenvalues within 1e-12 are equal, then (q, index)) give the same step
  energies to 1e-10 relative and the same kept counts, on Heisenberg L = 16,
  m = 32, Hubbard L = 12, m = 48, a J1-J2 chain and a two-leg ladder (bonds
  of reach 2, fermion signs across two sites).
* The superblock the device built at the last step, exported, gives the
  same E0 under the oracle's own Lanczos.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dmrg, ed, lanczos as olz, superblock as osb
from workloads import lattice_models as lm
from workloads.superblock import seeded_normal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    return binding


def compare(g_steps, o_steps, rel=1e-10):
    assert len(g_steps) == len(o_steps)
    for gs, os_ in zip(g_steps, o_steps):
        assert gs["status"] == 0
        assert gs["L"] == os_.L and gs["n_sys"] == os_.nS
        assert abs(gs["energy"] - os_.energy) <= rel * abs(os_.energy), (gs["L"], gs["n_sys"], gs["energy"], os_.energy)
        assert abs(gs["eps_S"] - os_.eps_S) <= 1e-9 and abs(gs["eps_E"] - os_.eps_E) <= 1e-9


def test_untruncated_heisenberg_equals_exact(gpu):
    g = gpu.GpuDmrg(lm.heisenberg_chain(), 10, m=10 ** 6)
    for st in g.infinite():
        assert st["status"] == 0 and st["eps_S"] == 0.0
        assert st["energy"] == pytest.approx(ed.heisenberg_ed(st["L"]), abs=1e-10)


def test_untruncated_hubbard_equals_exact(gpu):
    g = gpu.GpuDmrg(lm.hubbard_chain(1.0, 4.0), 8, m=10 ** 6)
    for st in g.infinite():
        n = st["L"] // 2
        assert st["energy"] == pytest.approx(ed.hubbard_ed(st["L"], n, n, 1.0, 4.0), abs=1e-10)


def test_paper_test_run_energies(gpu):
    rows = []
    with open(os.path.join(GOLDEN, "paper_test_run_energies.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                L, e, nd = line.split()
                rows.append((int(L), float(e), int(nd)))
    g = gpu.GpuDmrg(lm.hubbard_chain(1.0, 1.0), 10, m=64)
    got = {st["L"]: st["energy"] for st in g.infinite()}
    for (L, e, nd) in rows:
        assert abs(got[L] - e) <= 0.5 * 10.0 ** (-nd) + 1e-12, (L, got[L], e)


def test_heisenberg16_m32_infinite_and_sweep(gpu):
    g = gpu.GpuDmrg(lm.heisenberg_chain(), 16, m=32)
    gs = g.infinite() + g.sweeps(1)
    os_ = dmrg.finite_dmrg(dmrg.heisenberg_chain(), 16, m=32, n_sweeps=1)
    compare(gs, os_)
    exact = -6.911737145575
    assert all(s["energy"] >= exact - 1e-10 for s in gs if s["L"] == 16)
    assert gs[-1]["energy"] - exact < 1e-7


def test_hubbard12_m48_infinite_and_sweep(gpu):
    g = gpu.GpuDmrg(lm.hubbard_chain(1.0, 4.0), 12, m=48)
    gs = g.infinite() + g.sweeps(1)
    os_ = dmrg.finite_dmrg(dmrg.hubbard_chain(t=1.0, U=4.0), 12, m=48, n_sweeps=1)
    compare(gs, os_)
    # the exported last superblock under the oracle's own Lanczos
    sb, psi = g.last_superblock()
    ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), seeded_normal(3, sb.dim), tol=1e-12, max_iter=400)
    assert abs(ref.e0 - gs[-1]["energy"]) <= 1e-10 * abs(ref.e0)
    th, res = olz.rayleigh(lambda v: osb.apply_H(sb, v), psi)
    assert abs(th - gs[-1]["energy"]) <= 1e-10 * abs(th) and res <= 1e-9


def test_j1j2_chain_against_oracle(gpu):
    g = gpu.GpuDmrg(lm.heisenberg_chain(1.0, 0.35), 14, m=24)
    gs = g.infinite() + g.sweeps(1)
    os_ = dmrg.finite_dmrg(dmrg.heisenberg_chain(1.0, 0.35), 14, m=24, n_sweeps=1)
    compare(gs, os_)


def test_hubbard_ladder_against_oracle(gpu):
    g = gpu.GpuDmrg(lm.hubbard_ladder(1.0, 0.7, 6.0), 8, m=40)
    gs = g.infinite() + g.sweeps(1)
    os_ = dmrg.finite_dmrg(dmrg.hubbard_ladder(1.0, 0.7, 6.0), 8, m=40, n_sweeps=1)
    compare(gs, os_)
