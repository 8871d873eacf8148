"""The C ABI library builds, loads and exports every symbol that
include/dmrg_gb300.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_0902_3185_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dmrg_[a-z_A-Z0-9]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("dmrg_create_superblock", "dmrg_apply_H", "dmrg_lanczos_ground", "dmrg_energy_grad",
                 "dmrg_apply_H_backward", "dmrg_set_coeffs", "dmrg_destroy_superblock", "dmrg_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.SYMBOLS) <= set(declared_symbols())


def test_struct_layouts_match_header():
    # field sizes the C compiler would give the header's structs on LP64
    assert ctypes.sizeof(binding._Pair) == 4 * 4 + 8 * 4
    assert ctypes.sizeof(binding.LanczosOpts) == 8 + 4 * 3 + 4 + 8 + 4 * 2
    assert ctypes.sizeof(binding.LanczosInfo) == 8 * 2 + 4 * 8


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from workloads.synthetic import ragged_small
    with pytest.raises(RuntimeError):
        binding.GpuSuperblock(ragged_small())


def test_dmrg_sys_struct_layouts_match_header():
    # sizes of include/dmrg_sys.h's structs under the LP64 C layout rules
    assert ctypes.sizeof(binding._BondTerm) == 8 + 4 * 4
    assert ctypes.sizeof(binding._ModelDesc) == 136
    assert ctypes.sizeof(binding.SysOpts) == 8 + 4 * 4 + 8 + 8 + 8
    assert ctypes.sizeof(binding.StepInfo) == 4 * 4 + 8 + 8 * 5 + 4 * 4 + 8 + 8 * 4 + 4 * 2 + 8 * 3
    assert ctypes.sizeof(binding._SbView) == ctypes.sizeof(binding._Desc) + 8 * 3 + 4 * 2
