"""Failure detection on the GPU without faulting it.

* A tensor-core product whose copy warp is told to issue nothing: every
  device-side wait of the kernel gives up after its time limit, the kernel
  releases its tensor memory and raises the error word, and the host reads
  DMRG_ETIMEOUT; the next product on the same context is correct.
* Device allocation failure injected on the host (DMRG_TEST_FAIL_ALLOC) is
  reported as DMRG_ENOMEM by dmrg_create_superblock (child process).
* Invalid Lanczos options are rejected with DMRG_EINVAL.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import superblock as osb
from workloads.synthetic import ragged_small
from workloads.superblock import seeded_normal

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0902_3185_gb300 import binding
    binding.load()
    return binding


def test_bounded_wait_times_out_and_context_survives(gpu):
    sb = ragged_small(seed=4, batch=2)
    g = gpu.GpuSuperblock(sb)
    X = np.stack([seeded_normal(b, sb.dim) for b in range(2)])
    x = torch.from_numpy(X).cuda()
    assert g.lib.dmrg_test_inject(g.h, 1) == 0
    g.apply_H(x, prec="bf16x3")
    with pytest.raises(gpu.DmrgError) as ei:
        g.sync_status()
    assert ei.value.status == 6  # DMRG_ETIMEOUT
    g.sync_status()  # cleared
    y = g.apply_H(x, prec="bf16x3").cpu().numpy()
    g.sync_status()
    for b in range(2):
        ref = osb.apply_H(sb, X[b], b)
        assert np.abs(y[b] - ref).max() <= 1e-3 * np.abs(ref).max()


def test_allocation_failure_reports_enomem(gpu):
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_0902_3185_gb300 import binding\n"
        "from workloads.synthetic import ragged_small\n"
        "try:\n"
        "    binding.GpuSuperblock(ragged_small())\n"
        "    print('created')\n"
        "except binding.DmrgError as e:\n"
        "    print('status', e.status)\n" % ROOT)
    env = dict(os.environ, DMRG_TEST_FAIL_ALLOC="3")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert "status 2" in out.stdout, out.stdout + out.stderr


def test_bad_lanczos_options(gpu):
    sb = ragged_small(seed=1)
    g = gpu.GpuSuperblock(sb)
    x = torch.from_numpy(seeded_normal(0, sb.dim)[None]).cuda()
    with pytest.raises(gpu.DmrgError) as ei:
        g.lanczos_ground(x, tol=-1.0)
    assert ei.value.status == 1
    with pytest.raises(gpu.DmrgError):
        g.lanczos_ground(x, prec=7)
