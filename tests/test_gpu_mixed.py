"""GPU parity of the tensor-core (TF32, BF16x3) product and of the mixed
Lanczos with float64 refinement, through the C ABI, against the oracle.

Error model of a product y = c A Psi B^T computed with rounded operands,
a rounded intermediate and an FP32 accumulator: every output element obeys
|y - y_exact| <= gamma * (|c| |A| |Psi| |B|^T) summed over the pairs, with
gamma a few units of the operand precision u (TF32: u = 2^-11;
BF16 hi + lo: u = 2^-16 per split value) plus K * 2^-24 for the FP32 sums.
The tests use gamma = 8 u + 1e-5 (TF32) and 8 u + 2e-6 (BF16x3), checked
element by element against the oracle's |H| |psi|.
The mixed Lanczos followed by float64 refinement must reach the float64
oracle energy within |dE0| <= 1e-8 |E0|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lanczos as olz, superblock as osb
from workloads.grown import grown_hubbard_superblock, ladder_m1000
from workloads.superblock import Pair, Superblock, seeded_normal
from workloads.synthetic import ragged_small, random_sectored

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


def within_model(y, ref, bound, gamma):
    return np.all(np.abs(y - ref) <= gamma * bound + 1e-300)


CASES = {
    "ragged": lambda: ragged_small(seed=1, batch=3),
    "random_wide": lambda: random_sectored(seed=4, n_sectors=12, dmin=1, dmax=300, identity_terms=True, batch=2),
    "ladder_grown": lambda: grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0]),
    "chain_grown_b5": lambda: grown_hubbard_superblock(16, "chain", 8, 8, m=48, U_values=[1.0, 2.0, 3.0, 4.0, 6.0]),
}


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("name", list(CASES))
def test_apply_H_mixed(dev, name, prec):
    sb = CASES[name]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(10 + b, sb.dim) for b in range(sb.batch)])
    y = g.apply_H(to_dev(X), prec=prec).cpu().numpy()
    asb = abs_sb(sb)
    for b in range(sb.batch):
        ref = osb.apply_H(sb, X[b], b)
        bound = osb.apply_H(asb, np.abs(X[b]), b)
        err = np.abs(y[b] - ref)
        assert within_model(y[b], ref, bound, GAMMA[prec]), (name, prec, b, float((err / (bound + 1e-300)).max()))
    # accumulate
    y0 = np.stack([seeded_normal(50 + b, sb.dim) for b in range(sb.batch)])
    yt = to_dev(y0)
    g.apply_H(to_dev(X), y=yt, accumulate=True, prec=prec)
    yt = yt.cpu().numpy()
    for b in range(sb.batch):
        ref = y0[b] + osb.apply_H(sb, X[b], b)
        bound = osb.apply_H(asb, np.abs(X[b]), b)
        assert np.all(np.abs(yt[b] - ref) <= GAMMA[prec] * bound + 1e-12 * np.abs(ref))


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
@pytest.mark.parametrize("name", ["ragged", "random_wide"])
def test_transpose_mixed(dev, name, prec):
    sb = CASES[name]()
    g = gpu_sb(sb)
    G = np.stack([seeded_normal(30 + b, sb.dim) for b in range(sb.batch)])
    dpsi, _ = g.apply_H_backward(to_dev(G), to_dev(G), want_dc=False, prec=prec)
    dpsi = dpsi.cpu().numpy()
    asb = abs_sb(sb)
    for b in range(sb.batch):
        ref = osb.apply_HT(sb, G[b], b)
        bound = osb.apply_HT(asb, np.abs(G[b]), b)
        assert within_model(dpsi[b], ref, bound, GAMMA[prec])


def test_uncoupled_sector_zero_mixed(dev):
    sb = ragged_small(seed=3)
    g = gpu_sb(sb)
    off = sb.offsets()
    for prec in ("tf32", "bf16x3"):
        y = g.apply_H(to_dev(seeded_normal(0, sb.dim)[None]), prec=prec).cpu().numpy()[0]
        assert np.all(y[off[6]:off[7]] == 0.0)


@pytest.mark.parametrize("refine", ["newton", "lanczos", "newton_df64"])
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_mixed_lanczos_refined_matches_fp64(dev, prec, refine):
    sb = CASES["chain_grown_b5"]()
    g = gpu_sb(sb)
    P0 = np.stack([seeded_normal(b, sb.dim) for b in range(sb.batch)])
    e0, psi, infos, st = g.lanczos_ground(to_dev(P0), tol=1e-6, max_iter=300, prec=prec, refine=refine,
                                          refine_tol=1e-10)
    assert st == 0, infos
    psi = psi.cpu().numpy()
    for b in range(sb.batch):
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), P0[b], tol=1e-12, max_iter=300)
        assert abs(e0[b] - ref.e0) <= 1e-8 * abs(ref.e0), (b, e0[b], ref.e0)
        d = min(np.linalg.norm(psi[b] - ref.psi), np.linalg.norm(psi[b] + ref.psi))
        assert d < 1e-5
        assert infos[b]["mixed_matvecs"] > 0 and infos[b]["fp64_matvecs"] > 0
        assert infos[b]["residual"] <= 1e-10 * max(1.0, abs(e0[b]))
        if refine.startswith("newton"):
            assert infos[b]["fp64_matvecs"] <= 8


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_full_size_ladder_m1000_mixed(dev, prec):
    """2 x 32 ladder, m = 1000, 16 members in one launch: every element of two
    members within the error model."""
    sb = ladder_m1000(batch=16)
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(100 + b, sb.dim) for b in range(sb.batch)])
    y = g.apply_H(to_dev(X), prec=prec).cpu().numpy()
    asb = abs_sb(sb)
    for b in (0, 15):
        ref = osb.apply_H(sb, X[b], b)
        bound = osb.apply_H(asb, np.abs(X[b]), b)
        assert within_model(y[b], ref, bound, GAMMA[prec])


def test_folded_uniform_terms_follow_set_coeffs(dev):
    """Identity terms whose coefficient is the same for every member are
    folded into the tensor-core operator panels; the BF16x3 product stays
    within its error model after coefficient changes that keep a term
    uniform with a new value, that make it member-dependent, and that make it
    uniform again, and a Lanczos graph captured before the change is not
    reused with stale panels."""
    from paper_0902_3185_gb300 import binding
    sb0 = grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0, 6.0])
    g = gpu_sb(sb0)
    X = np.stack([seeded_normal(80 + b, sb0.dim) for b in range(sb0.batch)])
    x = to_dev(X)
    try:
        g.apply_H(x, prec="bf16x3")
    except binding.DmrgError as e:
        if e.status == 8:
            pytest.skip("tensor-core path not available")
        raise
    it = sb0.class_names.index("t")
    e_first, _, _, st = g.lanczos_ground(x, tol=1e-4, max_iter=200, prec="bf16x3", refine="newton_df64",
                                         refine_tol=1e-11)
    assert st == 0
    for tvals in ([1.3, 1.3, 1.3], [1.0, 0.8, 1.2], [0.9, 0.9, 0.9]):
        cp = sb0.couplings.copy()
        cp[:, it] = tvals
        sb = sb0.with_coeffs(sb0.coeffs_from_couplings(cp))
        g.set_coeffs(sb.coeffs)
        y = g.apply_H(x, prec="bf16x3").cpu().numpy()
        for b in range(sb.batch):
            ref = osb.apply_H(sb, X[b], b)
            assert within_model(y[b], ref, osb.apply_H(abs_sb(sb), np.abs(X[b]), b), GAMMA["bf16x3"]), tvals
        e0, _, _, st = g.lanczos_ground(x, tol=1e-4, max_iter=200, prec="bf16x3", refine="newton_df64",
                                        refine_tol=1e-11)
        assert st == 0
        for b in range(sb.batch):
            ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), X[b], tol=1e-12, max_iter=300)
            assert abs(e0[b] - ref.e0) <= 1e-8 * abs(ref.e0), (tvals, b)
