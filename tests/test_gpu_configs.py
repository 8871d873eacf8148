"""GPU parity on the workloads of the hot-path configurations.

* Hubbard chain L = 32, half filling, m = 200 (isometry-grown superblock):
  FP64 and BF16x3 products element by element; the mixed Lanczos with FP64
  refinement against the FP64 oracle, |dE0| <= 1e-8 |E0|, |dpsi| small.
* A superblock from the oracle's own finite DMRG (Hubbard L = 12, m = 48,
  one sweep): FP64 Lanczos within 1e-10 relative of the oracle.
* Synthetic batched product: 64 sectors, dims U{16..512}, 12 terms, 760
  pairs (D ~ 4.5e6): FP64, TF32 and BF16x3 products against the oracle.
* J1-J2 chain gradients: Hellmann-Feynman dE0/dJ1, dE0/dJ2 (chain rule over
  coupling-resolved terms) against central finite differences (h = 1e-5) of
  GPU FP64 energies, against the oracle's gradient, and the Euler identity
  E0 = J1 dE/dJ1 + J2 dE/dJ2; at J2 = J1/2 the Majumdar-Ghosh values.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dmrg, grad as ograd, lanczos as olz, superblock as osb
from workloads.grown import grown_hubbard_superblock
from workloads.superblock import Pair, Superblock, seeded_normal
from workloads.synthetic import random_sectored

GAMMA = {"tf32": 8 * 2.0 ** -11 + 1e-5, "bf16x3": 8 * 2.0 ** -16 + 2e-6}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    return torch.device("cuda:0")


def gpu_sb(sb):
    from paper_0902_3185_gb300.binding import GpuSuperblock
    return GpuSuperblock(sb)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def abs_sb(sb):
    pairs = [Pair(p.term, p.s_out, p.s_in, None if p.A is None else np.abs(p.A),
                  None if p.B is None else np.abs(p.B)) for p in sb.pairs]
    return Superblock(sb.r, sb.c, np.abs(sb.coeffs), pairs)


@pytest.fixture(scope="module")
def hub32():
    return grown_hubbard_superblock(32, "chain", 16, 16, m=200, U_values=[4.0], seed=2)


def test_hubbard32_m200_products(dev, hub32):
    sb = hub32
    g = gpu_sb(sb)
    X = seeded_normal(5, sb.dim)[None]
    ref = osb.apply_H(sb, X[0])
    y = g.apply_H(to_dev(X)).cpu().numpy()[0]
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    yb = g.apply_H(to_dev(X), prec="bf16x3").cpu().numpy()[0]
    bound = osb.apply_H(abs_sb(sb), np.abs(X[0]))
    assert np.all(np.abs(yb - ref) <= GAMMA["bf16x3"] * bound)


def test_hubbard32_m200_mixed_lanczos(dev, hub32):
    sb = hub32
    g = gpu_sb(sb)
    x0 = seeded_normal(0, sb.dim)
    e0, psi, infos, st = g.lanczos_ground(to_dev(x0[None]), tol=1e-6, max_iter=400, prec="bf16x3",
                                          refine="newton", refine_tol=1e-10)
    assert st == 0, infos
    ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), x0, tol=1e-12, max_iter=400)
    assert abs(e0[0] - ref.e0) <= 1e-8 * abs(ref.e0)
    p = psi.cpu().numpy()[0]
    assert min(np.linalg.norm(p - ref.psi), np.linalg.norm(p + ref.psi)) < 1e-5


def test_oracle_dmrg_superblock_fp64_lanczos(dev):
    model = dmrg.hubbard_chain(t=1.0, U=4.0, density=1.0)
    steps = dmrg.finite_dmrg(model, 12, m=48, n_sweeps=1, keep_superblocks=True)
    sb = steps[-1].superblock
    g = gpu_sb(sb)
    x0 = seeded_normal(1, sb.dim)
    e0, psi, infos, st = g.lanczos_ground(to_dev(x0[None]), tol=1e-12, max_iter=400)
    assert st == 0
    assert abs(e0[0] - steps[-1].energy) <= 1e-10 * abs(steps[-1].energy)


@pytest.mark.slow
def test_synthetic_64_sectors_full_size(dev):
    sb = random_sectored(seed=0)  # 64 sectors, 16..512, 760 pairs
    assert len(sb.pairs) == 760
    g = gpu_sb(sb)
    X = seeded_normal(9, sb.dim)[None]
    ref = osb.apply_H(sb, X[0])
    y = g.apply_H(to_dev(X)).cpu().numpy()[0]
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
    bound = osb.apply_H(abs_sb(sb), np.abs(X[0]))
    for prec in ("tf32", "bf16x3"):
        ym = g.apply_H(to_dev(X), prec=prec).cpu().numpy()[0]
        assert np.all(np.abs(ym - ref) <= GAMMA[prec] * bound), prec
    assert g.info["flops_per_matvec"] == pytest.approx(osb.matvec_flops(sb), rel=1e-12)


def _j1j2_superblock(L, J1, J2):
    model = dmrg.heisenberg_chain(J1, J2)
    S = dmrg.site_block(model)
    E = dmrg.site_block(model)
    for _ in range(L // 2 - 1):
        S = dmrg.grow(model, S, "left")
        E = dmrg.grow(model, E, "right")
    sb, _ = dmrg.make_superblock(model, S, E, L)
    return sb


@pytest.mark.parametrize("J2", [0.0, 0.25, 0.5])
def test_j1j2_gradients(dev, J2):
    L = 12
    sb0 = _j1j2_superblock(L, 1.0, 0.3)  # blocks are per coupling class: any J2 != 0 builds them
    sb = sb0.with_coeffs(sb0.coeffs_from_couplings([[1.0, J2]]))
    g = gpu_sb(sb)
    x0 = to_dev(seeded_normal(0, sb.dim)[None])

    def energy(J):
        g.set_coeffs(sb.coeffs_from_couplings([J]))
        e, _, _, st = g.lanczos_ground(x0, tol=1e-13, max_iter=500)
        assert st == 0
        return e[0]

    e0 = energy([1.0, J2])
    _, psi, _, _ = g.lanczos_ground(x0, tol=1e-13, max_iter=500)
    dEdc = g.energy_grad(psi).cpu().numpy()[0]
    grad = ograd.coupling_grad(sb, dEdc)  # classes (J1, J2)
    # Euler identity: H is homogeneous of degree one in the couplings
    assert e0 == pytest.approx(1.0 * grad[0] + J2 * grad[1], abs=1e-9)
    # central finite differences of GPU float64 energies
    h = 1e-5
    fd = [(energy([1.0 + h, J2]) - energy([1.0 - h, J2])) / (2 * h),
          (energy([1.0, J2 + h]) - energy([1.0, J2 - h])) / (2 * h)]
    assert np.allclose(grad, fd, rtol=1e-6, atol=1e-6)
    # the oracle's Hellmann-Feynman gradient on its own ground state
    ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), seeded_normal(0, sb.dim), tol=1e-13, max_iter=500)
    og = ograd.coupling_grad(sb, ograd.hf_grad(sb, ref.psi))
    assert np.allclose(grad, og, rtol=1e-8, atol=1e-9)
    if J2 == 0.5:
        assert e0 == pytest.approx(-3 * L / 8, abs=1e-9)
        assert grad[1] == pytest.approx(0.0, abs=1e-8)
        assert grad[0] == pytest.approx(-3 * L / 8, abs=1e-8)
