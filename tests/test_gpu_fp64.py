"""GPU parity of the float64 path against the CPU oracle, through the C ABI.

Tolerances (float64 products, different summation order than NumPy; the
double-float product, 48 significant bits, about 2^-46 relative per
multiply-add, meets the same bar):
element-wise |y_gpu - y_oracle| <= 1e-12 * max|y_oracle| for the product,
its transpose and the term dots; |dE0| <= 1e-10 * |E0| for Lanczos
(the paper's solver tolerance is the residual; the energy error is its
square over the gap), and psi within 1e-7 up to sign.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dmrg, grad as ograd, lanczos as olz, superblock as osb
from workloads.grown import grown_hubbard_superblock, ladder_m1000
from workloads.superblock import seeded_normal
from workloads.synthetic import ragged_small, random_sectored


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


def close(a, b, rel=1e-12):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = max(1.0, float(np.abs(b).max()) if b.size else 1.0)
    return float(np.abs(a - b).max() if a.size else 0.0) <= rel * scale


def heis16_superblock():
    model = dmrg.heisenberg_chain()
    steps, _, _ = dmrg.infinite_dmrg(model, 16, m=32, keep_superblocks=True)
    return steps[-1].superblock


CASES = {
    "ragged": lambda: ragged_small(seed=1, batch=3),
    "random16": lambda: random_sectored(seed=4, n_sectors=16, dmin=1, dmax=200, identity_terms=True, batch=2),
    "heis16_m32": heis16_superblock,
    "hub_ladder_grown": lambda: grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_apply_H_fp64(dev, name):
    sb = CASES[name]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(10 + b, sb.dim) for b in range(sb.batch)])
    y = g.apply_H(to_dev(X)).cpu().numpy()
    for b in range(sb.batch):
        assert close(y[b], osb.apply_H(sb, X[b], b)), (name, b)
    # accumulate mode: y += H psi
    y0 = np.stack([seeded_normal(50 + b, sb.dim) for b in range(sb.batch)])
    yt = to_dev(y0)
    g.apply_H(to_dev(X), y=yt, accumulate=True)
    yt = yt.cpu().numpy()
    for b in range(sb.batch):
        assert close(yt[b], y0[b] + osb.apply_H(sb, X[b], b))


@pytest.mark.parametrize("name", list(CASES))
def test_apply_H_df64(dev, name):
    """The double-float product against the float64 oracle, every element,
    plain and accumulating."""
    sb = CASES[name]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(10 + b, sb.dim) for b in range(sb.batch)])
    y = g.apply_H(to_dev(X), prec="df64").cpu().numpy()
    y0 = np.stack([seeded_normal(50 + b, sb.dim) for b in range(sb.batch)])
    yt = to_dev(y0)
    g.apply_H(to_dev(X), y=yt, accumulate=True, prec="df64")
    yt = yt.cpu().numpy()
    for b in range(sb.batch):
        ref = osb.apply_H(sb, X[b], b)
        assert close(y[b], ref), (name, b)
        assert close(yt[b], y0[b] + ref)


def test_df64_split_edge_values(dev):
    """Inputs outside the double-float range of the split (zeros, values
    below 2^-74 whose low part is dropped, signs) still give the product to
    the float64 bar in the max norm."""
    sb = CASES["ragged"]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(70 + b, sb.dim) for b in range(sb.batch)])
    X[:, ::7] = 0.0
    X[:, 1::11] *= 1e-30
    X[:, 2::13] *= -1.0
    y = g.apply_H(to_dev(X), prec="df64").cpu().numpy()
    for b in range(sb.batch):
        assert close(y[b], osb.apply_H(sb, X[b], b))


@pytest.mark.parametrize("name", ["ragged", "random16", "hub_ladder_grown"])
def test_backward_and_term_dots_fp64(dev, name):
    sb = CASES[name]()
    g = gpu_sb(sb)
    P = np.stack([seeded_normal(20 + b, sb.dim) for b in range(sb.batch)])
    G = np.stack([seeded_normal(30 + b, sb.dim) for b in range(sb.batch)])
    dpsi, dc = g.apply_H_backward(to_dev(P), to_dev(G))
    dpsi, dc = dpsi.cpu().numpy(), dc.cpu().numpy()
    for b in range(sb.batch):
        assert close(dpsi[b], osb.apply_HT(sb, G[b], b))
        assert close(dc[b], osb.term_products(sb, G[b], P[b]))


def test_empty_and_uncoupled_sectors(dev):
    sb = ragged_small(seed=3)
    g = gpu_sb(sb)
    y = g.apply_H(to_dev(seeded_normal(0, sb.dim)[None])).cpu().numpy()[0]
    off = sb.offsets()
    assert np.all(y[off[6]:off[7]] == 0.0)


def test_energy_grad_fp64(dev):
    sb = CASES["hub_ladder_grown"]()
    g = gpu_sb(sb)
    P = np.stack([seeded_normal(7 + b, sb.dim) for b in range(sb.batch)])
    out = g.energy_grad(to_dev(P)).cpu().numpy()
    for b in range(sb.batch):
        assert close(out[b], ograd.hf_grad(sb.with_coeffs(sb.coeffs[b:b + 1]), P[b]))


@pytest.mark.parametrize("name", ["heis16_m32", "hub_ladder_grown"])
def test_lanczos_fp64_matches_oracle(dev, name):
    sb = CASES[name]()
    g = gpu_sb(sb)
    P0 = np.stack([seeded_normal(b, sb.dim) for b in range(sb.batch)])
    e0, psi, infos, st = g.lanczos_ground(to_dev(P0), tol=1e-12, max_iter=300, prec="fp64")
    assert st == 0, infos
    psi = psi.cpu().numpy()
    for b in range(sb.batch):
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), P0[b], tol=1e-12, max_iter=300)
        assert abs(e0[b] - ref.e0) <= 1e-10 * abs(ref.e0), (b, e0[b], ref.e0)
        d = min(np.linalg.norm(psi[b] - ref.psi), np.linalg.norm(psi[b] + ref.psi))
        assert d < 1e-7
        th, res = olz.rayleigh(lambda v: osb.apply_H(sb, v, b), psi[b])
        assert res < 1e-9 * max(1.0, abs(th))


def test_lanczos_fp64_heis16_against_exact(dev):
    # last infinite-DMRG superblock of the L = 16, m = 32 chain: variational,
    # within the truncation error of the exact energy -6.911737145575
    sb = CASES["heis16_m32"]()
    g = gpu_sb(sb)
    e0, _, _, st = g.lanczos_ground(to_dev(seeded_normal(0, sb.dim)[None]), tol=1e-12)
    assert st == 0
    assert -6.911737145575 - 1e-10 <= e0[0] < -6.911737145575 + 1e-3


def test_lanczos_cap_reports_noconv(dev):
    sb = CASES["hub_ladder_grown"]()
    g = gpu_sb(sb)
    e0, psi, infos, st = g.lanczos_ground(to_dev(seeded_normal(0, sb.dim)[None].repeat(sb.batch, 0)),
                                          tol=1e-14, max_iter=3)
    assert st == 4 and all(i["status"] == 4 and i["iters"] == 3 for i in infos)


@pytest.mark.parametrize("check_every", [1, 3])
def test_lanczos_members_stop_apart(dev, check_every):
    """Members converge at different iterations and stop apart: status 0,
    the reported residual within tol, the true residual |H psi - E psi| of
    the returned state within a few tol, energies equal to the oracle's.  At
    tol = 1e-10, below what the float32 estimate resolves, members are tested
    in float64 at each check near convergence, so they stop at a check point
    no later than the oracle's own stopping iteration (tolerance 1e-12), not
    at the cap."""
    sb = CASES["hub_ladder_grown"]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(40 + b, sb.dim) for b in range(sb.batch)])
    tol = 1e-10
    e0, psi, infos, st = g.lanczos_ground(to_dev(X), tol=tol, max_iter=400, check_every=check_every)
    assert st == 0, infos
    P = psi.cpu().numpy()
    for b in range(sb.batch):
        scale = max(1.0, abs(e0[b]))
        assert infos[b]["status"] == 0 and infos[b]["residual"] <= tol * scale
        assert infos[b]["iters"] % check_every == 0
        r = osb.apply_H(sb, P[b], b) - e0[b] * P[b]
        assert np.linalg.norm(r) <= 10 * tol * scale
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), X[b], tol=1e-12, max_iter=400)
        assert ref.converged and infos[b]["iters"] <= ref.iters + check_every, (b, infos[b]["iters"], ref.iters)
        assert abs(e0[b] - ref.e0) <= 1e-10 * abs(ref.e0)


def test_lanczos_breakdown_exact(dev):
    # a start vector inside a small invariant subspace: the Krylov space closes
    sb = ragged_small(seed=1)
    g = gpu_sb(sb)
    off = sb.offsets()
    x = np.zeros(sb.dim)
    x[off[0]:off[1]] = 1.0  # 1x1 sector 0: H maps it into sectors it couples to
    e0, psi, infos, st = g.lanczos_ground(to_dev(x[None]), tol=1e-13, max_iter=400)
    ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v), x, tol=1e-13, max_iter=400)
    assert abs(e0[0] - ref.e0) <= 1e-9 * max(1, abs(ref.e0))


def test_set_coeffs_and_autograd(dev):
    from paper_0902_3185_gb300.binding import apply_H
    sb = ragged_small(seed=2, tiny=True)
    g = gpu_sb(sb)
    psi = torch.from_numpy(seeded_normal(0, sb.dim)[None]).cuda().requires_grad_(True)
    c = torch.from_numpy(sb.coeffs.copy()).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda p, cc: apply_H(p, cc, g), (psi, c), eps=1e-6, atol=1e-7)
    c2 = sb.coeffs * 1.7
    g.set_coeffs(c2)
    y = g.apply_H(psi.detach()).cpu().numpy()[0]
    assert close(y, osb.apply_H(sb.with_coeffs(c2), psi.detach().cpu().numpy()[0]))


@pytest.mark.slow
def test_full_size_ladder_m1000_sampled(dev):
    """The 2 x 32 ladder at m = 1000, 16 members: float64 and double-float
    products of two members against the oracle, every element."""
    sb = ladder_m1000(batch=16)
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(100 + b, sb.dim) for b in range(sb.batch)])
    y = g.apply_H(to_dev(X)).cpu().numpy()
    yd = g.apply_H(to_dev(X), prec="df64").cpu().numpy()
    for b in (0, 15):
        ref = osb.apply_H(sb, X[b], b)
        assert close(y[b], ref)
        assert close(yd[b], ref)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("name", list(CASES))
def test_apply_H_term_dots(dev, name, prec):
    """One pass gives H psi (as the float64 product) and the per-term dots
    <psi, (A_k x B_k) psi> (as the oracle's term products), in float64 or
    double-float arithmetic."""
    sb = CASES[name]()
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(30 + b, sb.dim) for b in range(sb.batch)])
    y, dots = g.apply_H_term_dots(to_dev(X), prec=prec)
    y, dots = y.cpu().numpy(), dots.cpu().numpy()
    for b in range(sb.batch):
        assert close(y[b], osb.apply_H(sb, X[b], b))
        assert close(dots[b], osb.term_products(sb, X[b], X[b]))
        # and H psi = sum_k c_k (A_k x B_k) psi, dotted with psi
        assert float(X[b] @ y[b]) == pytest.approx(float(sb.coeffs[b] @ dots[b]), rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("prec,refine", [("bf16x3", "newton"), ("tf32", "newton"), ("fp64", "none"),
                                         ("bf16x3", "lanczos"), ("bf16x3", "newton_df64")])
def test_lanczos_ground_grad(dev, prec, refine):
    """The gradient returned with the solve (from the refinement's last float64
    product, or computed after it) equals dmrg_energy_grad of the returned
    state and the oracle's Hellmann-Feynman gradient."""
    sb = grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0])
    g = gpu_sb(sb)
    x0 = to_dev(np.stack([seeded_normal(3 + b, sb.dim) for b in range(sb.batch)]))
    tol = 1e-12 if prec == "fp64" else 1e-5
    e0, psi, infos, st, dE = g.lanczos_ground(x0, tol=tol, max_iter=400, prec=prec, refine=refine,
                                              refine_tol=1e-11, grad=True)
    assert st == 0, infos
    ref = g.energy_grad(psi).cpu().numpy()
    dE = dE.cpu().numpy()
    assert close(dE, ref, rel=1e-12)
    P = psi.cpu().numpy()
    for b in range(sb.batch):
        assert close(dE[b], ograd.hf_grad(sb, P[b]), rel=1e-11)
        # E0 = sum_k c_k dE0/dc_k (H is linear in the coefficients)
        assert float(sb.coeffs[b] @ dE[b]) == pytest.approx(e0[b], rel=1e-10)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_lanczos_resumes_after_a_false_float32_pass(dev, prec):
    """A member whose float32 residual estimate passes although the float64
    test after the loop fails is restarted from its Ritz vector and converges
    (status 0) instead of reporting non-convergence with iterations left.
    The testing hook makes the float32 test pass at the first check of every
    member (a one-vector Krylov space: the float64 test must fail there), at
    the tight tolerance 1e-13."""
    from paper_0902_3185_gb300 import binding
    sb = grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0])
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(30 + b, sb.dim) for b in range(sb.batch)])
    assert g.lib.dmrg_test_inject(g.h, 2) == 0
    try:
        if prec == "fp64":
            e0, psi, infos, st = g.lanczos_ground(to_dev(X), tol=1e-13, max_iter=400)
        else:
            e0, psi, infos, st = g.lanczos_ground(to_dev(X), tol=1e-4, max_iter=400, prec=prec,
                                                  refine="newton_df64", refine_tol=1e-11)
    except binding.DmrgError as e:
        if e.status == 8:
            pytest.skip("tensor-core path not available")
        raise
    assert st == 0, infos
    for b in range(sb.batch):
        assert infos[b]["restarts"] >= 1 and infos[b]["status"] == 0
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), X[b], tol=1e-13, max_iter=400)
        assert abs(e0[b] - ref.e0) <= 1e-10 * abs(ref.e0), (b, e0[b], ref.e0)
    # the hook applies to one solve: the next runs without a restart
    e1, _, infos, st = g.lanczos_ground(to_dev(X), tol=1e-13, max_iter=400)
    assert st == 0 and all(i["restarts"] == 0 for i in infos)


def test_set_coeffs_is_ordered_on_the_callers_stream(dev):
    """dmrg_set_coeffs writes the coefficient table on the given stream, after
    the products already queued there: products queued before it on a side
    stream use the old coefficients, products after it the new ones."""
    sb = grown_hubbard_superblock(16, "chain", 8, 8, m=48, U_values=[1.0, 2.0, 3.0, 4.0, 6.0])
    g = gpu_sb(sb)
    X = np.stack([seeded_normal(40 + b, sb.dim) for b in range(sb.batch)])
    x = to_dev(X)
    c_new = sb.coeffs * 1.3 + 0.1
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        ys = [g.apply_H(x, stream=side) for _ in range(8)]  # queued, not yet run
        g.set_coeffs(c_new, stream=side)
        y_new = g.apply_H(x, stream=side)
    side.synchronize()
    sb_new = sb.with_coeffs(c_new)
    for b in range(sb.batch):
        ref_old = osb.apply_H(sb, X[b], b)
        ref_new = osb.apply_H(sb_new, X[b], b)
        for y in ys:
            assert close(y.cpu().numpy()[b], ref_old)
        assert close(y_new.cpu().numpy()[b], ref_new)


def test_time_reorth_hook(dev):
    """The Gram-Schmidt timing hook: positive time, the documented byte count,
    bad arguments rejected; a solve afterwards is unaffected."""
    from paper_0902_3185_gb300 import binding
    sb = grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0])
    g = gpu_sb(sb)
    for prec in ("fp64", "bf16x3"):
        ms, nbytes = g.time_reorth(10, prec=prec, reps=3)
        assert ms > 0 and nbytes == (2 * 11 + 3) * sb.dim * sb.batch * 8
    with pytest.raises(binding.DmrgError):
        g.time_reorth(-1)
    X = np.stack([seeded_normal(50 + b, sb.dim) for b in range(sb.batch)])
    e0, _, _, st = g.lanczos_ground(to_dev(X), tol=1e-12, max_iter=300)
    assert st == 0
    for b in range(sb.batch):
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), X[b], tol=1e-12, max_iter=300)
        assert abs(e0[b] - ref.e0) <= 1e-10 * abs(ref.e0)
