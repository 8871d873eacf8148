"""The autotuner: it times every candidate tiling, keeps the fastest, reports
the per-block-launch baseline, and the product stays within the error model
(and Lanczos, whose graphs it invalidates, still converges) afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import lanczos as olz, superblock as osb
from workloads.grown import grown_hubbard_superblock
from workloads.superblock import Pair, Superblock, seeded_normal

GAMMA = {"tf32": 8 * 2.0 ** -11 + 1e-5, "bf16x3": 8 * 2.0 ** -16 + 2e-6}


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    return binding


@pytest.mark.parametrize("prec", ["tf32", "bf16x3"])
def test_autotune_then_products_and_lanczos(gpu, prec):
    sb = grown_hubbard_superblock(16, "chain", 8, 8, m=48, U_values=[1.0, 3.0, 6.0])
    g = gpu.GpuSuperblock(sb)
    X = np.stack([seeded_normal(b, sb.dim) for b in range(sb.batch)])
    x = torch.from_numpy(X).cuda()
    g.lanczos_ground(x, tol=1e-6, prec=prec)  # captures graphs before tuning
    rep = g.autotune(prec=prec, reps=3)
    assert rep["candidates"] == 12
    assert rep["best_tile_n"] in (64, 128, 256) and rep["heavy_first"] in (0, 1) and rep["pieces"] in (0, 1)
    assert 0 < rep["best_ms"] <= rep["default_ms"] * 1.0001 or rep["best_ms"] <= rep["default_ms"]
    assert rep["per_block_ms"] > 0
    y = g.apply_H(x, prec=prec).cpu().numpy()
    asb = Superblock(sb.r, sb.c, np.abs(sb.coeffs),
                     [Pair(p.term, p.s_out, p.s_in, None if p.A is None else np.abs(p.A),
                           None if p.B is None else np.abs(p.B)) for p in sb.pairs])
    for b in range(sb.batch):
        ref = osb.apply_H(sb, X[b], b)
        assert np.all(np.abs(y[b] - ref) <= GAMMA[prec] * osb.apply_H(asb, np.abs(X[b]), b))
    e0, _, infos, st = g.lanczos_ground(x, tol=1e-6, prec=prec, refine="newton", refine_tol=1e-10)
    assert st == 0
    for b in range(sb.batch):
        ref = olz.lanczos_ground(lambda v: osb.apply_H(sb, v, b), X[b], tol=1e-12, max_iter=300)
        assert abs(e0[b] - ref.e0) <= 1e-8 * abs(ref.e0)
