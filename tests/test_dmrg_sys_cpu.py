"""Host-side validation of the device DMRG driver's C ABI (include/dmrg_sys.h)
on the CPU: inconsistent models and options are rejected with DMRG_EINVAL
before any device work, a consistent model is accepted, the run calls
enforce their order, and the batched eigensolver rejects bad sizes.  No call
here reaches the GPU."""
import ctypes as C

import numpy as np
import pytest

from paper_0902_3185_gb300 import binding
from workloads import lattice_models as lm

EINVAL = 1


@pytest.fixture(scope="module")
def lib():
    return binding.load()


def make_desc(model, keep):
    d = model.d
    arrs = [np.ascontiguousarray(model.site_q, dtype=np.int64),
            np.ascontiguousarray(model.site_parity, dtype=np.int32),
            np.ascontiguousarray(model.ops, dtype=np.float64).reshape(-1, d, d),
            np.ascontiguousarray(model.op_fermion, dtype=np.int32),
            np.ascontiguousarray(model.couplings, dtype=np.float64),
            np.ascontiguousarray(model.onsite_class, dtype=np.int32),
            (np.ascontiguousarray(model.onsite, dtype=np.float64).reshape(-1, d, d) if len(model.onsite_class)
             else np.zeros((1, d, d))),
            np.ascontiguousarray(model.bond_rules, dtype=np.int32).reshape(-1, 4)]
    terms = (binding._BondTerm * max(1, len(model.bond_terms)))()
    for i, t in enumerate(model.bond_terms):
        terms[i] = binding._BondTerm(*t)
    keep += arrs + [terms]
    return binding._ModelDesc(d, arrs[0].ctypes.data, arrs[1].ctypes.data, len(model.op_names), arrs[2].ctypes.data,
                              arrs[3].ctypes.data, len(model.class_names), arrs[4].ctypes.data,
                              len(model.onsite_class), arrs[5].ctypes.data, arrs[6].ctypes.data, len(arrs[7]),
                              arrs[7].ctypes.data, len(model.bond_terms), C.cast(terms, C.c_void_p),
                              float(model.density), int(model.Q))


def opts(**kw):
    o = dict(tol=1e-12, max_iter=300, prec=0, refine=0, guess=0, mixed_tol=1e-6, tie_tol=1e-12, seed=0)
    o.update(kw)
    return binding.SysOpts(o["tol"], o["max_iter"], o["prec"], o["refine"], o["guess"], o["mixed_tol"],
                           o["tie_tol"], o["seed"])


def create(lib, model, L=8, m=16, **kw):
    keep = []
    desc = make_desc(model, keep)
    h = C.c_void_p()
    st = lib.dmrg_sys_create(C.byref(desc), L, m, C.byref(opts(**kw)), C.byref(h))
    return st, h


def test_consistent_models_are_accepted(lib):
    for model in (lm.heisenberg_chain(), lm.heisenberg_chain(1.0, 0.5), lm.hubbard_chain(), lm.hubbard_ladder()):
        st, h = create(lib, model)
        assert st == 0
        # run calls enforce their order, before any device work
        n = C.c_int32()
        steps = (binding.StepInfo * 10)()
        assert lib.dmrg_sys_sweeps(h, 1, steps, C.byref(n)) == EINVAL
        assert b"infinite" in lib.dmrg_sys_last_error(h)
        view = binding._SbView()
        assert lib.dmrg_sys_last_superblock(h, C.byref(view), None) == EINVAL
        lib.dmrg_sys_destroy(h)


@pytest.mark.parametrize("what", ["odd_L", "m0", "same_q", "delta0", "mixed_term", "bad_class", "neg_density",
                                  "mixed_tol", "tol"])
def test_inconsistent_inputs_are_rejected(lib, what):
    model = lm.hubbard_chain()
    L, m, kw = 8, 16, {}
    if what == "odd_L":
        L = 7
    elif what == "m0":
        m = 0
    elif what == "same_q":
        model.site_q = np.array([0, 1, 1, 2], dtype=np.int64)
    elif what == "delta0":
        model.bond_rules = np.array([[0, 0, 1, 0]], dtype=np.int32)
    elif what == "mixed_term":
        model.op_fermion = np.array([1, 0], dtype=np.int32)  # c_dn declared bosonic ...
        model.bond_terms = [(1.0, 0, 0, 1, 1)]               # ... and a term pairing c_up with c_dn
    elif what == "bad_class":
        model.onsite_class = np.array([7], dtype=np.int32)
    elif what == "neg_density":
        model.density = -1.0
    elif what == "mixed_tol":
        kw = dict(prec=2, mixed_tol=0.0)
    elif what == "tol":
        kw = dict(tol=0.0)
    st, h = create(lib, model, L, m, **kw)
    assert st == EINVAL and not h


def test_eigensolver_rejects_bad_sizes(lib):
    n = np.array([5000], dtype=np.int32)
    ptr = (C.c_void_p * 1)(1)
    assert lib.dmrg_sym_eig_batched(1, n.ctypes.data, ptr, ptr, ptr, None) == EINVAL
    n = np.array([-1], dtype=np.int32)
    assert lib.dmrg_sym_eig_batched(1, n.ctypes.data, ptr, ptr, ptr, None) == EINVAL
    assert lib.dmrg_sym_eig_batched(-1, None, None, None, None, None) == EINVAL
    assert lib.dmrg_sym_eig_batched(0, None, None, None, None, None) == 0
