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


@pytest.mark.parametrize("make,L,m", [(lambda: lm.hubbard_chain(1.0, 4.0), 12, 48),
                                      (lambda: lm.hubbard_ladder(1.0, 0.7, 6.0), 10, 48),
                                      (lambda: lm.heisenberg_chain(1.0, 0.35), 14, 24)])
def test_wavefunction_transformation_cuts_iterations(gpu, make, L, m):
    """Finite steps started from the previous ground state carried to the new
    basis (White's wavefunction transformation, the paper's closing notes):
    the same energies as random starts (to 1e-10), every finite step started
    from the transformed state, and fewer Lanczos iterations.  At the float64
    tolerance 1e-12 the transformed state's error (about the truncation
    error) still leaves most of the 12 decades to the Lanczos iteration, so
    the saving is a fraction of the random starts' count (0.67 of it on the
    L = 10 ladder), not an order of magnitude."""
    runs = {}
    for guess in (False, True):
        g = gpu.GpuDmrg(make(), L, m=m, guess=guess)
        g.infinite()
        runs[guess] = g.sweeps(2)
    rnd, gss = runs[False], runs[True]
    assert len(rnd) == len(gss)
    for a, b in zip(rnd, gss):
        assert a["status"] == 0 and b["status"] == 0
        assert abs(a["energy"] - b["energy"]) <= 1e-10 * abs(a["energy"])
        assert b["guessed"] == 1 and a["guessed"] == 0
    it_r = sum(s["iters"] for s in rnd)
    it_g = sum(s["iters"] for s in gss)
    assert it_g < 0.75 * it_r, (it_g, it_r)


@pytest.mark.slow
def test_config2_hubbard32_m200_two_sweeps(gpu):
    """Hubbard chain L = 32, U = 4, half filling, m = 200: the infinite
    algorithm and two finite sweeps on the device, end to end.  Every step
    converges; the sweeps lower the middle-split energy below the infinite
    phase's and the second sweep changes it by less than 1e-6 relative;
    the last superblock, exported, gives the same E0 under the oracle's own
    Lanczos (1e-10)."""
    g = gpu.GpuDmrg(lm.hubbard_chain(1.0, 4.0), 32, m=200, tol=1e-10, guess=True)
    inf = g.infinite()
    sw = g.sweeps(2)
    assert all(s["status"] == 0 for s in inf + sw)
    assert all(s["guessed"] == 1 for s in sw)
    e_inf = inf[-1]["energy"]
    mids = [s["energy"] for s in sw if s["n_sys"] == 16]
    assert mids[-1] <= e_inf + 1e-9
    assert abs(mids[-1] - mids[-3]) <= 1e-6 * abs(mids[-1])
    sb, psi = g.last_superblock()
    ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), seeded_normal(5, sb.dim), tol=1e-11, max_iter=600)
    assert abs(ref.e0 - sw[-1]["energy"]) <= 1e-10 * abs(ref.e0)


def test_batched_symmetric_eigensolver(gpu):
    """dmrg_sym_eig_batched against LAPACK on seeded matrices of every path:
    one block (n <= 110), a cluster of 16 blocks (111 <= n <= 448), one block
    over global memory (n > 448); random symmetric, and rank-deficient positive
    semidefinite (density matrices Psi Psi^T).  Eigenvalues to 1e-12 ||A||,
    V orthogonal to 1e-12, residual A V - V diag(w) to 1e-11 ||A||."""
    rng = np.random.default_rng(7)
    sizes = [1, 2, 3, 17, 64, 110, 111, 200, 333, 448, 470]
    mats = []
    for i, n in enumerate(sizes):
        if i % 2:
            X = rng.standard_normal((n, max(1, n // 3)))
            M = X @ X.T
            M /= np.trace(M)
        else:
            M = rng.standard_normal((n, n))
            M = M + M.T
        mats.append(M)
    out = gpu.sym_eig_batched([torch.from_numpy(M).cuda() for M in mats])
    for M, (w, V) in zip(mats, out):
        w, V = w.cpu().numpy(), V.cpu().numpy()
        n = M.shape[0]
        scale = max(1e-300, np.abs(M).max())
        ref = np.sort(np.linalg.eigvalsh(M))[::-1]
        assert np.all(np.diff(w) <= 0)
        assert np.abs(w - ref).max() <= 1e-12 * scale * max(1, np.sqrt(n)), n
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12 * max(1, np.sqrt(n)), n
        assert np.abs(M @ V - V * w[None, :]).max() <= 1e-11 * scale * max(1, np.sqrt(n)), n
