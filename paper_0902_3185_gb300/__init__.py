"""GB300 (sm_103a) superblock H*psi + Lanczos for DMRG.

The compute path is the CUDA library ``libdmrg_gb300.so`` built from
``csrc/`` (see ``build.py``); ``binding`` marshals arguments to its C ABI.
"""
from .binding import ApplyH, DmrgError, GpuSuperblock, apply_H, load

__all__ = ["ApplyH", "DmrgError", "GpuSuperblock", "apply_H", "load"]
