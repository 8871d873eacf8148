"""Failure handling that needs no GPU: the C ABI rejects inconsistent
descriptors with DMRG_EINVAL before touching the device (host-side checks),
and the multi-rank timing of bench.py (max over ranks, whole-job value) is
exercised with two gloo ranks on the CPU."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_0902_3185_gb300 import binding, build


def _lib():
    return C.CDLL(build.build())


def _create(desc, batch=1):
    lib = _lib()
    lib.dmrg_create_superblock.argtypes = [C.POINTER(binding._Desc), C.c_int32, C.POINTER(C.c_void_p)]
    lib.dmrg_create_superblock.restype = C.c_int
    h = C.c_void_p()
    st = lib.dmrg_create_superblock(C.byref(desc), batch, C.byref(h))
    return st, h


def _desc(r, c, pairs, n_terms=1, coeffs=None):
    r = np.ascontiguousarray(r, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.int32)
    coeffs = np.ones(n_terms) if coeffs is None else np.ascontiguousarray(coeffs, dtype=np.float64)
    arr = (binding._Pair * max(1, len(pairs)))(*pairs)
    keep = (r, c, coeffs, arr)
    d = binding._Desc(len(r), r.ctypes.data, c.ctypes.data, n_terms, coeffs.ctypes.data, len(pairs),
                      C.cast(arr, C.c_void_p), 0)
    return d, keep


A2 = np.eye(2)
B3 = np.ones((3, 3))


@pytest.mark.parametrize("case", ["neg_dim", "sector_range", "term_range", "id_a_shape", "both_id",
                                  "null_block", "small_ld", "empty"])
def test_descriptor_rejected(case):
    P = lambda term, so, si, flags, A, lda, B, ldb: binding._Pair(term, so, si, flags, A, lda, B, ldb)
    a, b = A2.ctypes.data, B3.ctypes.data
    r, c = [2, 2], [3, 3]
    pairs = [P(0, 0, 1, 0, a, 2, b, 3)]
    if case == "neg_dim":
        r = [2, -1]
    elif case == "sector_range":
        pairs = [P(0, 0, 5, 0, a, 2, b, 3)]
    elif case == "term_range":
        pairs = [P(3, 0, 1, 0, a, 2, b, 3)]
    elif case == "id_a_shape":
        r = [2, 4]
        pairs = [P(0, 0, 1, binding.ID_A, None, 0, b, 3)]
    elif case == "both_id":
        pairs = [P(0, 0, 0, binding.ID_A | binding.ID_B, None, 0, None, 0)]
    elif case == "null_block":
        pairs = [P(0, 0, 1, 0, None, 2, b, 3)]
    elif case == "small_ld":
        pairs = [P(0, 0, 1, 0, a, 1, b, 3)]
    elif case == "empty":
        r, c = [0, 2], [3, 0]
    d, keep = _desc(r, c, pairs)
    st, h = _create(d)
    assert st == 1 and not h.value  # DMRG_EINVAL, no handle


def test_batch_must_be_positive():
    d, keep = _desc([2], [3], [binding._Pair(0, 0, 0, 0, A2.ctypes.data, 2, B3.ctypes.data, 3)])
    st, h = _create(d, batch=0)
    assert st == 1


def _rank(rank, world, port, ms, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(ms[rank], dist, torch.device("cpu"))
    v = bench.job_value(world, products=10, flops=2e9, ms_total=t)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_bench_multi_rank_timing_gloo():
    import torch.multiprocessing as mp
    ms = [12.0, 15.5]
    port = 29500 + os.getpid() % 1000
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, ms, out), nprocs=2, join=True)
    for r in range(2):
        t, v = out[r]
        assert t == pytest.approx(15.5)            # the slowest rank defines the step
        assert v == pytest.approx(2 * 10 * 2e9 / 15.5e-3 / 1e12)  # whole-job TFLOP/s
