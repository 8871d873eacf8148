"""J1-J2 chain at L = 48, m = 400: a coupling sweep on the device.

The superblock is the last step of the oracle's infinite DMRG for the
J1-J2 chain at the Majumdar-Ghosh point J2 = J1/2 (L = 48, m = 400 kept
states, coupling-resolved block Hamiltonians).  At that point the ground
state is a product of nearest-neighbour singlets, which the kept basis holds
exactly, so E0 = -3L/8 = -18, dE0/dJ1 = -18 and dE0/dJ2 = 0.

On this fixed basis the six couplings J2 = 0, 0.1, .., 0.5 run as six batch
members of one superblock (operator blocks shared, coefficients per member):

* mixed-precision solve (TF32 products, float64 Lanczos) with float64 Newton
  refinement against the float64 solve: |dE0| <= 1e-8 |E0|;
* Hellmann-Feynman gradients dE0/dJ1, dE0/dJ2 (chain rule over the
  coupling-resolved terms) against central finite differences (h = 1e-5,
  1e-6 relative) of float64 energies -- the four shifted couplings of every member as 24 members
  of a second superblock -- against the oracle's gradient (its own DMRG
  ground state at J2 = 0.5, its formula on the device state elsewhere), and
  against the Euler identity E0 = J1 dE/dJ1 + J2 dE/dJ2;
* at J2 = 0.5 the Majumdar-Ghosh values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle import dmrg, grad as ograd
from workloads.superblock import seeded_normal

L, M = 48, 400
J2S = [0.0, 0.1, 0.2, 0.3, 0.4, 0.5]
H = 1e-5


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    model = dmrg.heisenberg_chain(1.0, 0.5, Lmax=L)
    steps, _, _ = dmrg.infinite_dmrg(model, L, m=M, keep_superblocks=True)
    last = steps[-1]
    return binding, last.superblock, last.psi, last.energy


def start(sb, batch):
    return torch.from_numpy(np.stack([seeded_normal(7, sb.dim)] * batch)).cuda()


def test_oracle_mg_energy(mg):
    _, sb, _, e = mg
    assert sb.class_names == ["J1", "J2"]
    assert e == pytest.approx(-3 * L / 8, abs=1e-9)


def test_j2_sweep_energies_and_gradients(mg):
    binding, sb0, psi_o, _ = mg
    sb = sb0.with_coeffs(sb0.coeffs_from_couplings([[1.0, j2] for j2 in J2S]))
    g = binding.GpuSuperblock(sb)
    B = len(J2S)
    # mixed solve + float64 refinement
    e_mx, psi, infos, st = g.lanczos_ground(start(sb, B), tol=1e-6, max_iter=400, prec="tf32",
                                           refine="newton", refine_tol=1e-11)
    assert st == 0, infos
    # float64 solve of the same members
    e_64, _, _, st = g.lanczos_ground(start(sb, B), tol=1e-12, max_iter=600)
    assert st == 0
    assert np.all(np.abs(e_mx - e_64) <= 1e-8 * np.abs(e_64))
    # Hellmann-Feynman gradients on the refined states
    dEdc = g.energy_grad(psi).cpu().numpy()
    grads = np.array([ograd.coupling_grad(sb, dEdc[b]) for b in range(B)])
    # Euler identity (H is homogeneous of degree one in the couplings)
    for b, j2 in enumerate(J2S):
        assert e_64[b] == pytest.approx(1.0 * grads[b, 0] + j2 * grads[b, 1], abs=1e-7)
    # central finite differences of float64 energies: 4 shifted couplings per member
    shifted = []
    for j2 in J2S:
        shifted += [[1.0 + H, j2], [1.0 - H, j2], [1.0, j2 + H], [1.0, j2 - H]]
    sbf = sb0.with_coeffs(sb0.coeffs_from_couplings(shifted))
    gf = binding.GpuSuperblock(sbf)
    ef, _, _, st = gf.lanczos_ground(start(sbf, len(shifted)), tol=1e-13, max_iter=600)
    assert st == 0
    ef = ef.reshape(B, 4)
    fd = np.stack([(ef[:, 0] - ef[:, 1]) / (2 * H), (ef[:, 2] - ef[:, 3]) / (2 * H)], axis=1)
    # 1e-6 relative, plus an absolute floor for dE0/dJ2 ~ 0 at the Majumdar-Ghosh
    # point: a central difference of energies each accurate to eps |E| errs by
    # at most eps |E| / h (rounding) + h^2 |E'''| / 6 (truncation, ~1e-10 here);
    # the float64 solves at tolerance 1e-13 give eps <= 1e-13, |E| <= 21, so
    # eps |E| / h <= 2.1e-7; the floor is 5e-7
    assert np.allclose(grads, fd, rtol=1e-6, atol=5e-7), np.abs(grads - fd).max()
    # the oracle's gradient formula on the device states
    P = psi.cpu().numpy()
    for b in range(B):
        og = ograd.coupling_grad(sb, ograd.hf_grad(sb.with_coeffs(sb.coeffs[b:b + 1]), P[b]))
        assert np.allclose(grads[b], og, rtol=1e-9, atol=1e-9)
    # at J2 = J1 / 2: the oracle's own ground state and the Majumdar-Ghosh values
    b = J2S.index(0.5)
    og = ograd.coupling_grad(sb, ograd.hf_grad(sb.with_coeffs(sb.coeffs[b:b + 1]), psi_o))
    assert np.allclose(grads[b], og, rtol=1e-8, atol=1e-8)
    assert e_mx[b] == pytest.approx(-3 * L / 8, abs=1e-8 * 18)
    assert grads[b, 0] == pytest.approx(-3 * L / 8, abs=1e-7)
    assert grads[b, 1] == pytest.approx(0.0, abs=1e-7)
