"""Local density of states on the device: c_i |psi> by the product of a
transition container (c_i (x) 1 between the N and N -/+ 1 targets), Lanczos
coefficients on the N -/+ 1 superblock (dmrg_lanczos_coeffs) and their
continued fractions (dmrg_continued_fraction), against the oracle.

Bars: the continued-fraction kernel against the oracle's evaluation to 1e-12
relative; an untruncated Hubbard chain (L = 6) against exact
diagonalisation to 1e-8 of the peak density; a truncated one (L = 12,
m = 48, two U values as batch members) against the oracle's Lanczos
coefficients (first 40, relative 1e-8; the Krylov spaces are the same up to
rounding) and its densities to 1e-7; BF16x3 products within 2 % of the peak.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dmrg, ldos
from oracle import lanczos as olz
from oracle import superblock as osb
from workloads.superblock import seeded_normal

OMEGA = np.linspace(-6.0, 6.0, 241)
ETA = 0.1


@pytest.fixture(scope="module")
def binding():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding as b
    b.load()
    return b


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def device_ldos(binding, inp, psi, e0, n_max, prec="fp64"):
    """(A_<, A_>) per member from the device path; psi [batch][D_N], e0 [batch]."""
    out = []
    for part in ("hole", "particle"):
        sb, tr = inp[part]
        gt = binding.GpuSuperblock(tr)
        n_out = tr.meta["dim_out"]
        x = np.zeros((psi.shape[0], tr.dim))
        x[:, n_out:] = psi
        y = gt.apply_H(to_dev(x))
        phi = y[:, :n_out].contiguous()
        g = binding.GpuSuperblock(sb)
        norm2, a, b, n = g.lanczos_coeffs(phi, n_max, prec=prec)
        sgn = -1.0 if part == "hole" else 1.0
        z = (e0[:, None] + sgn * OMEGA[None, :]) + 1j * ETA
        G = binding.continued_fraction(norm2, a, b, n, to_dev(z))
        out.append(-G.imag.cpu().numpy() / np.pi)
        out.append((norm2.cpu().numpy(), a.cpu().numpy(), b.cpu().numpy(), n))
    return out  # A_<, coeffs_<, A_>, coeffs_>


def test_continued_fraction_kernel(binding):
    rng = np.random.default_rng(5)
    batch, ld = 4, 12
    a = rng.standard_normal((batch, ld))
    b = np.abs(rng.standard_normal((batch, ld)))
    norm2 = rng.uniform(0.5, 2.0, batch)
    n = np.array([12, 5, 1, 0], dtype=np.int32)
    z = rng.uniform(-3, 3, (batch, 50)) + 1j * rng.uniform(0.01, 1.0, (batch, 50))
    G = binding.continued_fraction(to_dev(norm2), to_dev(a), to_dev(b), n, to_dev(z)).cpu().numpy()
    for k in range(batch):
        if n[k] == 0:
            assert np.all(G[k] == 0)
            continue
        ref = ldos.continued_fraction(norm2[k], a[k, :n[k]], b[k, :n[k] - 1], z[k])
        assert np.max(np.abs(G[k] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("spin", ["up", "dn"])
def test_untruncated_chain_against_ed(binding, spin):
    L, U = 6, 2.0
    model = dmrg.hubbard_chain(1.0, U, Lmax=L)
    steps, _, _ = dmrg.infinite_dmrg(model, L, m=1000, keep_superblocks=True)
    last = steps[-1]
    Sp, Ep = last.blocks
    i = Sp.n - 1
    h_ed, p_ed, e0 = ldos.hubbard_ldos_ed(L, i, spin, L // 2, L // 2, 1.0, U, OMEGA, ETA)
    inp = ldos.superblock_ldos_inputs(model, Sp, Ep, last.L, i, spin)
    # the ground state from the device solver (the density is quadratic in psi: its sign is free)
    g = binding.GpuSuperblock(last.superblock)
    e_dev, psi, _, st = g.lanczos_ground(to_dev(np.ones((1, last.superblock.dim))), tol=1e-12, max_iter=400)
    assert st == 0 and e_dev[0] == pytest.approx(e0, abs=1e-10)
    h, ch, p, cp = device_ldos(binding, inp, psi.cpu().numpy(), e_dev, n_max=400)
    assert ch[0][0] + cp[0][0] == pytest.approx(1.0, abs=1e-12)  # |c psi|^2 + |c^dag psi|^2
    peak = max(h_ed.max(), p_ed.max())
    assert np.max(np.abs(h[0] - h_ed)) <= 1e-8 * peak
    assert np.max(np.abs(p[0] - p_ed)) <= 1e-8 * peak


def test_truncated_chain_against_oracle(binding):
    L, m = 12, 48
    Us = [4.0, 6.0]
    model = dmrg.hubbard_chain(1.0, 4.0, Lmax=L)
    steps, _, _ = dmrg.infinite_dmrg(model, L, m=m, keep_superblocks=True)
    last = steps[-1]
    Sp, Ep = last.blocks
    i = Sp.n - 1
    inp = ldos.superblock_ldos_inputs(model, Sp, Ep, last.L, i, "up", couplings_batch=[[1.0, u] for u in Us])
    sbN = last.superblock.with_coeffs(last.superblock.coeffs_from_couplings([[1.0, u] for u in Us]))
    # ground states per U (oracle), then both paths from the same psi
    psis, e0s = [], []
    for b in range(len(Us)):
        r = olz.lanczos_ground(lambda v: osb.apply_H(sbN, v, b), seeded_normal(b, sbN.dim), tol=1e-12, max_iter=400)
        psis.append(r.psi)
        e0s.append(r.e0)
    psis, e0s = np.array(psis), np.array(e0s)
    n_max = 40
    h, ch, p, cp = device_ldos(binding, inp, psis, e0s, n_max)
    for part, A_dev, cf_dev in (("hole", h, ch), ("particle", p, cp)):
        sb, tr = inp[part]
        n_out = tr.meta["dim_out"]
        for b in range(len(Us)):
            y = osb.apply_H(tr, np.concatenate([np.zeros(n_out), psis[b]]), b)
            norm2, a, bb = ldos.lanczos_coefficients(lambda v: osb.apply_H(sb, v, b), y[:n_out], n_max)
            k = len(a)
            assert cf_dev[3][b] == k
            assert cf_dev[0][b] == pytest.approx(norm2, rel=1e-12)
            assert np.max(np.abs(cf_dev[1][b, :k] - a)) <= 1e-8 * np.max(np.abs(a))
            assert np.max(np.abs(cf_dev[2][b, :k - 1] - bb)) <= 1e-8 * np.max(np.abs(bb))
            z = (e0s[b] - OMEGA if part == "hole" else e0s[b] + OMEGA) + 1j * ETA
            ref = -ldos.continued_fraction(norm2, a, bb, z).imag / np.pi
            assert np.max(np.abs(A_dev[b] - ref)) <= 1e-7 * ref.max()
    # mixed-precision products: the same densities within 2 % of the peak
    hm, _, pm, _ = device_ldos(binding, inp, psis, e0s, n_max, prec="bf16x3")
    peak = max(h.max(), p.max())
    assert np.max(np.abs(hm - h)) <= 0.02 * peak and np.max(np.abs(pm - p)) <= 0.02 * peak


def test_zero_start_vector_member(binding):
    """A member whose start vector is zero (c on an empty site) gets no
    coefficients and G = 0; the other members are unaffected."""
    L, U = 6, 2.0
    model = dmrg.hubbard_chain(1.0, U, Lmax=L)
    steps, _, _ = dmrg.infinite_dmrg(model, L, m=1000, keep_superblocks=True)
    last = steps[-1]
    Sp, Ep = last.blocks
    inp = ldos.superblock_ldos_inputs(model, Sp, Ep, last.L, Sp.n - 1, "up", couplings_batch=[[1.0, U]] * 2)
    sb, tr = inp["hole"]
    n_out = tr.meta["dim_out"]
    phi1 = osb.apply_H(tr, np.concatenate([np.zeros(n_out), last.psi]))[:n_out]
    phi = np.stack([np.zeros(n_out), phi1])
    g = binding.GpuSuperblock(sb)
    norm2, a, b, n = g.lanczos_coeffs(to_dev(phi), 30)
    assert n[0] == 0 and n[1] == 30 and float(norm2[0]) == 0.0
    z = np.tile(last.energy - OMEGA + 1j * ETA, (2, 1))
    G = binding.continued_fraction(norm2, a, b, n, to_dev(z)).cpu().numpy()
    assert np.all(G[0] == 0)
    ref_n2, ra, rb = ldos.lanczos_coefficients(lambda v: osb.apply_H(sb, v, 1), phi1, 30)
    ref = ldos.continued_fraction(ref_n2, ra, rb, z[1])
    assert np.max(np.abs(G[1] - ref)) <= 1e-8 * np.max(np.abs(ref))
