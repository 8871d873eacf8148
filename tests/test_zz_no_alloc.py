"""The allocation-free float64 product (dmrg_apply_H_static_scratch).

Some callers cannot allocate device memory when they apply H -- processes
whose device memory is managed by another framework's pool, real-time loops
in which an allocation (which can synchronise the device) is not allowed.
This entry point keeps
its intermediate workspace in a static device buffer of the library.  The
test calls it through the C ABI twice in a row (the buffer keeps the first
call's contents) and compares with dmrg_apply_H in float64 within the
product tolerance of the other float64 tests, |dy| <= 1e-12 max|y|; it also
checks the size limit is enforced.  This file is collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from workloads.grown import grown_hubbard_superblock
from workloads.superblock import seeded_normal
from workloads.synthetic import random_sectored


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    return binding


def test_static_scratch_matches_apply_H_twice(gpu):
    sb = grown_hubbard_superblock(12, "ladder", 5, 5, m=60, cut=6, U_values=[4.0, 8.0])
    g = gpu.GpuSuperblock(sb)
    for call, seed in enumerate((11, 12)):
        X = np.stack([seeded_normal(seed + 10 * b, sb.dim) for b in range(sb.batch)])
        x = torch.from_numpy(X).cuda()
        ref = g.apply_H(x).cpu().numpy()
        y = g.apply_H_static_scratch(x).cpu().numpy()
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), call
        y0 = torch.from_numpy(np.stack([seeded_normal(99 + b, sb.dim) for b in range(sb.batch)])).cuda()
        y1 = y0.clone()
        g.apply_H_static_scratch(x, y=y1, accumulate=True)
        assert np.abs(y1.cpu().numpy() - (y0.cpu().numpy() + ref)).max() <= 1e-12 * np.abs(ref).max()


def test_static_scratch_rejects_oversized(gpu):
    sb = random_sectored(seed=3, n_sectors=8, dmin=400, dmax=512)
    g = gpu.GpuSuperblock(sb)
    x = torch.zeros(sb.batch, sb.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.DmrgError) as ei:
        g.apply_H_static_scratch(x)
    assert ei.value.status == 1 and "static buffer holds" in str(ei.value)
