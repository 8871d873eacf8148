"""Thin ctypes binding of ``libdmrg_gb300.so`` (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module converts
a :class:`workloads.superblock.Superblock` into the C descriptor, passes
device pointers of torch tensors, and raises on any non-OK status.  There is
no CPU fallback: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdmrg_gb300.so")

FP64, TF32, BF16X3, DF64 = 0, 1, 2, 3
PREC = {"fp64": FP64, "tf32": TF32, "bf16x3": BF16X3, "df64": DF64}
ID_A, ID_B = 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "EBREAKDOWN",
          6: "ETIMEOUT", 7: "ENAN", 8: "EUNSUPPORTED"}

# exported symbols, as declared in include/dmrg_gb300.h
SYMBOLS = ["dmrg_create_superblock", "dmrg_destroy_superblock", "dmrg_last_error", "dmrg_query",
           "dmrg_set_coeffs", "dmrg_apply_H", "dmrg_apply_H_backward", "dmrg_lanczos_ground",
           "dmrg_energy_grad", "dmrg_apply_H_static_scratch", "dmrg_autotune", "dmrg_sync_status",
           "dmrg_test_inject", "dmrg_lanczos_ground_grad", "dmrg_apply_H_term_dots", "dmrg_lanczos_coeffs",
           "dmrg_continued_fraction", "dmrg_sys_create", "dmrg_sys_destroy", "dmrg_sys_last_error",
           "dmrg_sys_infinite", "dmrg_sys_sweeps", "dmrg_sys_last_superblock", "dmrg_sym_eig_batched",
           "dmrg_time_reorth"]


class DmrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Pair(C.Structure):
    _fields_ = [("term", C.c_int32), ("s_out", C.c_int32), ("s_in", C.c_int32), ("flags", C.c_int32),
                ("A", C.c_void_p), ("lda", C.c_int64), ("B", C.c_void_p), ("ldb", C.c_int64)]


class _Desc(C.Structure):
    _fields_ = [("n_sectors", C.c_int32), ("r", C.c_void_p), ("c", C.c_void_p), ("n_terms", C.c_int32),
                ("coeffs", C.c_void_p), ("n_pairs", C.c_int32), ("pairs", C.c_void_p),
                ("blocks_on_device", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("dim", C.c_int64), ("batch", C.c_int32), ("n_sectors", C.c_int32), ("n_terms", C.c_int32),
                ("n_pairs", C.c_int32), ("flops_per_matvec", C.c_double), ("op_bytes_f64", C.c_double),
                ("op_bytes_mixed", C.c_double)]


class TuneInfo(C.Structure):
    _fields_ = [("best_ms", C.c_double), ("default_ms", C.c_double), ("per_block_ms", C.c_double),
                ("best_tile_n", C.c_int32), ("heavy_first", C.c_int32), ("candidates", C.c_int32),
                ("pieces", C.c_int32)]


class LanczosOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("prec", C.c_int32), ("refine", C.c_int32),
                ("refine_tol", C.c_double), ("check_every", C.c_int32), ("graph_iters", C.c_int32)]


class LanczosInfo(C.Structure):
    _fields_ = [("e0", C.c_double), ("residual", C.c_double), ("iters", C.c_int32),
                ("refine_iters", C.c_int32), ("mixed_matvecs", C.c_int32), ("fp64_matvecs", C.c_int32),
                ("status", C.c_int32), ("breakdown", C.c_int32), ("kernel_launches", C.c_int32),
                ("restarts", C.c_int32)]


class _BondTerm(C.Structure):
    _fields_ = [("coef", C.c_double), ("op_a", C.c_int32), ("trans_a", C.c_int32), ("op_b", C.c_int32),
                ("trans_b", C.c_int32)]


class _ModelDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("site_q", C.c_void_p), ("site_parity", C.c_void_p), ("n_ops", C.c_int32),
                ("ops", C.c_void_p), ("op_fermion", C.c_void_p), ("n_classes", C.c_int32),
                ("couplings", C.c_void_p), ("n_onsite", C.c_int32), ("onsite_class", C.c_void_p),
                ("onsite", C.c_void_p), ("n_bond_rules", C.c_int32), ("bond_rules", C.c_void_p),
                ("n_bond_terms", C.c_int32), ("bond_terms", C.c_void_p), ("density", C.c_double),
                ("Q", C.c_int64)]


class SysOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("prec", C.c_int32), ("refine", C.c_int32),
                ("guess", C.c_int32), ("mixed_tol", C.c_double), ("tie_tol", C.c_double), ("seed", C.c_uint64)]


class StepInfo(C.Structure):
    _fields_ = [("L", C.c_int32), ("n_sys", C.c_int32), ("direction", C.c_int32), ("status", C.c_int32),
                ("dim", C.c_int64), ("energy", C.c_double), ("eps_S", C.c_double), ("eps_E", C.c_double),
                ("gap_S", C.c_double), ("gap_E", C.c_double), ("iters", C.c_int32), ("kept_S", C.c_int32),
                ("kept_E", C.c_int32), ("n_terms", C.c_int32), ("ms", C.c_double), ("ms_grow", C.c_double),
                ("ms_superblock", C.c_double), ("ms_solve", C.c_double), ("ms_truncate", C.c_double),
                ("max_sector", C.c_int32), ("guessed", C.c_int32), ("ms_eig", C.c_double),
                ("ms_select", C.c_double), ("ms_transform", C.c_double)]


class _SbView(C.Structure):
    _fields_ = [("desc", _Desc), ("term_class", C.c_void_p), ("term_mult", C.c_void_p), ("sector_q", C.c_void_p),
                ("n_sys", C.c_int32), ("L", C.c_int32)]


_lib = None


def library_path() -> str:
    return LIB_PATH


def load(build_if_missing: bool = True):
    """Load the library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH}")
    lib = C.CDLL(LIB_PATH)
    vp, i32, dp = C.c_void_p, C.c_int32, C.c_void_p
    lib.dmrg_create_superblock.argtypes = [C.POINTER(_Desc), i32, C.POINTER(vp)]
    lib.dmrg_destroy_superblock.argtypes = [vp]
    lib.dmrg_destroy_superblock.restype = None
    lib.dmrg_last_error.argtypes = [vp]
    lib.dmrg_last_error.restype = C.c_char_p
    lib.dmrg_query.argtypes = [vp, C.POINTER(_Info)]
    lib.dmrg_set_coeffs.argtypes = [vp, dp, vp]
    lib.dmrg_apply_H.argtypes = [vp, dp, dp, i32, i32, vp]
    lib.dmrg_apply_H_backward.argtypes = [vp, dp, dp, dp, dp, i32, vp]
    lib.dmrg_lanczos_ground.argtypes = [vp, dp, dp, dp, C.POINTER(LanczosOpts), C.POINTER(LanczosInfo), vp]
    lib.dmrg_energy_grad.argtypes = [vp, dp, dp, i32, vp]
    lib.dmrg_apply_H_static_scratch.argtypes = [vp, dp, dp, i32, vp]
    lib.dmrg_autotune.argtypes = [vp, i32, i32, vp, C.POINTER(TuneInfo)]
    lib.dmrg_sync_status.argtypes = [vp, vp]
    lib.dmrg_test_inject.argtypes = [vp, i32]
    lib.dmrg_lanczos_ground_grad.argtypes = [vp, dp, dp, dp, dp, C.POINTER(LanczosOpts), C.POINTER(LanczosInfo), vp]
    lib.dmrg_apply_H_term_dots.argtypes = [vp, dp, dp, dp, i32, vp]
    lib.dmrg_lanczos_coeffs.argtypes = [vp, dp, i32, i32, dp, dp, dp, dp, vp]
    lib.dmrg_continued_fraction.argtypes = [dp, dp, dp, dp, i32, i32, dp, dp, i32, dp, dp, vp]
    lib.dmrg_sys_create.argtypes = [C.POINTER(_ModelDesc), i32, i32, C.POINTER(SysOpts), C.POINTER(vp)]
    lib.dmrg_sys_destroy.argtypes = [vp]
    lib.dmrg_sys_destroy.restype = None
    lib.dmrg_sys_last_error.argtypes = [vp]
    lib.dmrg_sys_last_error.restype = C.c_char_p
    lib.dmrg_sys_infinite.argtypes = [vp, C.POINTER(StepInfo), C.POINTER(C.c_int32)]
    lib.dmrg_sys_sweeps.argtypes = [vp, i32, C.POINTER(StepInfo), C.POINTER(C.c_int32)]
    lib.dmrg_sys_last_superblock.argtypes = [vp, C.POINTER(_SbView), dp]
    lib.dmrg_sym_eig_batched.argtypes = [i32, vp, vp, vp, vp, vp]
    lib.dmrg_time_reorth.argtypes = [vp, i32, i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    for name in SYMBOLS:
        if name not in ("dmrg_destroy_superblock", "dmrg_last_error", "dmrg_sys_destroy", "dmrg_sys_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


class GpuSuperblock:
    """Device-resident superblock: operator blocks, task lists and workspace."""

    def __init__(self, sb, device=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.lib = load()
        self.device = torch.device(device or "cuda")
        self.sb = sb
        self.batch = sb.batch
        self.n_terms = sb.n_terms
        self.dim = sb.dim
        r = np.ascontiguousarray(sb.r, dtype=np.int32)
        c = np.ascontiguousarray(sb.c, dtype=np.int32)
        coeffs = np.ascontiguousarray(sb.coeffs, dtype=np.float64)
        keep = []
        pairs = (_Pair * max(1, len(sb.pairs)))()
        for i, p in enumerate(sb.pairs):
            flags = (ID_A if p.A is None else 0) | (ID_B if p.B is None else 0)
            A = None if p.A is None else np.ascontiguousarray(p.A, dtype=np.float64)
            B = None if p.B is None else np.ascontiguousarray(p.B, dtype=np.float64)
            keep += [A, B]
            pairs[i] = _Pair(p.term, p.s_out, p.s_in, flags,
                             None if A is None else A.ctypes.data, 0 if A is None else A.shape[1],
                             None if B is None else B.ctypes.data, 0 if B is None else B.shape[1])
        desc = _Desc(sb.n_sectors, r.ctypes.data, c.ctypes.data, sb.n_terms, coeffs.ctypes.data,
                     len(sb.pairs), C.cast(pairs, C.c_void_p), 0)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.dmrg_create_superblock(C.byref(desc), sb.batch, C.byref(h))
        if st != 0:
            raise DmrgError(st, "dmrg_create_superblock failed (see stderr)")
        self.h = h
        info = _Info()
        self._check(self.lib.dmrg_query(self.h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in _Info._fields_}

    def _check(self, st):
        if st != 0:
            msg = self.lib.dmrg_last_error(self.h) if getattr(self, "h", None) else b""
            raise DmrgError(st, (msg or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_destroy_superblock(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- calls
    def empty(self):
        return torch.empty(self.batch, self.dim, dtype=torch.float64, device=self.device)

    def set_coeffs(self, coeffs, stream=None):
        c = np.ascontiguousarray(np.broadcast_to(np.asarray(coeffs, dtype=np.float64),
                                                 (self.batch, self.n_terms)))
        self._check(self.lib.dmrg_set_coeffs(self.h, c.ctypes.data, _stream(stream)))

    def apply_H(self, psi, y=None, accumulate=False, prec="fp64", stream=None):
        if y is None:
            y = self.empty()
        self._check(self.lib.dmrg_apply_H(self.h, _ptr(psi), _ptr(y), int(accumulate), _prec(prec),
                                          _stream(stream)))
        return y

    def sync_status(self, stream=None):
        """Synchronise and raise DmrgError(ETIMEOUT) if a device-side wait gave up."""
        self._check(self.lib.dmrg_sync_status(self.h, _stream(stream)))

    def autotune(self, prec="bf16x3", reps=5, stream=None):
        """Pick the tensor-core tiling for this superblock by timing; returns the report."""
        info = TuneInfo()
        self._check(self.lib.dmrg_autotune(self.h, _prec(prec), reps, _stream(stream), C.byref(info)))
        return {k: getattr(info, k) for k, _ in TuneInfo._fields_ if k != "pad"}

    def apply_H_static_scratch(self, psi, y=None, accumulate=False, stream=None):
        """float64 product whose workspace is the library's static device
        buffer: for callers that must not allocate device memory while they
        apply H (the output tensor, when not given, is allocated here)."""
        if y is None:
            y = self.empty()
        self._check(self.lib.dmrg_apply_H_static_scratch(self.h, _ptr(psi), _ptr(y), int(accumulate),
                                                         _stream(stream)))
        return y

    def apply_H_backward(self, psi, g, want_dpsi=True, want_dc=True, prec="fp64", stream=None):
        dpsi = self.empty() if want_dpsi else None
        dc = torch.empty(self.batch, self.n_terms, dtype=torch.float64, device=self.device) if want_dc else None
        self._check(self.lib.dmrg_apply_H_backward(self.h, _ptr(psi), _ptr(g), _ptr(dpsi), _ptr(dc),
                                                   _prec(prec), _stream(stream)))
        return dpsi, dc

    def energy_grad(self, psi, prec="fp64", stream=None):
        out = torch.empty(self.batch, self.n_terms, dtype=torch.float64, device=self.device)
        self._check(self.lib.dmrg_energy_grad(self.h, _ptr(psi), _ptr(out), _prec(prec), _stream(stream)))
        return out

    REFINE = {None: 0, False: 0, "none": 0, "lanczos": 1, True: 2, "newton": 2, "newton_df64": 3}

    def lanczos_ground(self, psi0, tol=1e-12, max_iter=300, prec="fp64", refine="newton", refine_tol=1e-10,
                       check_every=1, graph_iters=8, psi_out=None, stream=None, grad=False):
        """Lowest eigenpair of every member.  With a mixed precision, refine =
        "newton" (float64 residual + mixed CG correction steps, default),
        "newton_df64" (the same with double-float residual products),
        "lanczos" (float64 Lanczos restarted from the mixed result) or "none".
        Returns (e0, psi, infos, status); with grad=True also the
        Hellmann-Feynman gradient [batch][n_terms] of psi, as a fifth value."""
        if psi_out is None:
            psi_out = self.empty()
        e0 = np.zeros(self.batch)
        info = (LanczosInfo * self.batch)()
        mode = refine if isinstance(refine, int) and not isinstance(refine, bool) else self.REFINE[refine]
        opts = LanczosOpts(tol, max_iter, _prec(prec), mode, refine_tol, check_every, graph_iters)
        if grad:
            dE = torch.empty(self.batch, self.n_terms, dtype=torch.float64, device=self.device)
            st = self.lib.dmrg_lanczos_ground_grad(self.h, _ptr(psi0), _ptr(psi_out), e0.ctypes.data, _ptr(dE),
                                                   C.byref(opts), info, _stream(stream))
        else:
            st = self.lib.dmrg_lanczos_ground(self.h, _ptr(psi0), _ptr(psi_out), e0.ctypes.data, C.byref(opts),
                                              info, _stream(stream))
        infos = [{k: getattr(info[b], k) for k, _ in LanczosInfo._fields_} for b in range(self.batch)]
        if st not in (0, 4):
            self._check(st)
        if grad:
            return e0, psi_out, infos, st, dE
        return e0, psi_out, infos, st

    def time_reorth(self, j, prec="bf16x3", reps=5, stream=None):
        """Event-timed full Gram-Schmidt pass at Krylov index j: (ms, bytes moved)."""
        ms, nbytes = C.c_double(), C.c_double()
        self._check(self.lib.dmrg_time_reorth(self.h, _prec(prec), int(j), int(reps), C.byref(ms), C.byref(nbytes),
                                              _stream(stream)))
        return ms.value, nbytes.value

    def apply_H_term_dots(self, psi, prec="fp64", stream=None):
        """y = H psi and dots[b][k] = <psi_b, (A_k (x) B_k) psi_b>, one pass
        (prec "fp64" or "df64")."""
        y = self.empty()
        dots = torch.empty(self.batch, self.n_terms, dtype=torch.float64, device=self.device)
        self._check(self.lib.dmrg_apply_H_term_dots(self.h, _ptr(psi), _ptr(y), _ptr(dots), _prec(prec),
                                                    _stream(stream)))
        return y, dots


    def lanczos_coeffs(self, phi0, n_max, prec="fp64", stream=None):
        """Lanczos coefficients from phi0 (no convergence test): returns
        (norm2 [batch], alpha [batch][n_max], beta [batch][n_max], n [batch]
        numpy int32); row b holds n[b] coefficients (beta[b][j] couples
        Krylov vectors j and j + 1)."""
        alpha = torch.empty(self.batch, n_max, dtype=torch.float64, device=self.device)
        beta = torch.empty_like(alpha)
        norm2 = torch.empty(self.batch, dtype=torch.float64, device=self.device)
        n = np.zeros(self.batch, dtype=np.int32)
        self._check(self.lib.dmrg_lanczos_coeffs(self.h, _ptr(phi0.contiguous()), int(n_max), _prec(prec),
                                                 _ptr(alpha), _ptr(beta), _ptr(norm2), n.ctypes.data,
                                                 _stream(stream)))
        return norm2, alpha, beta, n


def continued_fraction(norm2, alpha, beta, n, z, stream=None):
    """G_b(z) for complex z [batch][n_z] (device tensor) from Lanczos
    coefficients (as returned by GpuSuperblock.lanczos_coeffs); complex128."""
    lib = load()
    batch, ld = alpha.shape
    z = z.to(torch.complex128)
    zr, zi = z.real.contiguous(), z.imag.contiguous()
    gr, gi = torch.empty_like(zr), torch.empty_like(zi)
    nd = torch.as_tensor(np.asarray(n, dtype=np.int32), device=alpha.device)
    alpha, beta = alpha.contiguous(), beta.contiguous()
    st = lib.dmrg_continued_fraction(_ptr(norm2), _ptr(alpha), _ptr(beta), nd.data_ptr(),
                                     int(batch), int(ld), _ptr(zr), _ptr(zi), int(zr.shape[1]), _ptr(gr),
                                     _ptr(gi), _stream(stream))
    if st != 0:
        raise DmrgError(st, "continued_fraction")
    return torch.complex(gr, gi)


class ApplyH(torch.autograd.Function):
    """y = H(c) psi through the library; backward gives H^T g and <g, (A_k (x) B_k) psi>."""

    @staticmethod
    def forward(ctx, psi, coeffs, gsb: GpuSuperblock, prec="fp64"):
        c = coeffs.detach().cpu().numpy().copy()
        gsb.set_coeffs(c)
        ctx.gsb = gsb
        ctx.prec = prec
        ctx.coeffs = c  # the library holds one coefficient table: restore it for backward
        ctx.save_for_backward(psi)
        return gsb.apply_H(psi.contiguous(), prec=prec)

    @staticmethod
    def backward(ctx, g):
        (psi,) = ctx.saved_tensors
        need_psi, need_c = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        ctx.gsb.set_coeffs(ctx.coeffs)
        dpsi, dc = ctx.gsb.apply_H_backward(psi, g.contiguous(), want_dpsi=need_psi, want_dc=need_c,
                                            prec=ctx.prec)
        return dpsi, dc, None, None


def apply_H(psi, coeffs, gsb: GpuSuperblock, prec="fp64"):
    return ApplyH.apply(psi, coeffs, gsb, prec)


class GpuDmrg:
    """The infinite- and finite-system DMRG with every block operation on the
    device (dmrg_sys_*): growth, superblock, Lanczos, density matrices,
    truncation, change of basis.  `model` is a workloads.lattice_models.ModelDesc."""

    def __init__(self, model, L, m, tol=1e-12, max_iter=300, prec="fp64", refine="newton", mixed_tol=1e-6,
                 tie_tol=1e-12, seed=0, guess=False):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.lib = load()
        self.model = model
        self.L, self.m = int(L), int(m)
        d = model.d
        self._keep = [np.ascontiguousarray(model.site_q, dtype=np.int64),
                      np.ascontiguousarray(model.site_parity, dtype=np.int32),
                      np.ascontiguousarray(model.ops, dtype=np.float64).reshape(-1, d, d),
                      np.ascontiguousarray(model.op_fermion, dtype=np.int32),
                      np.ascontiguousarray(model.couplings, dtype=np.float64),
                      np.ascontiguousarray(model.onsite_class, dtype=np.int32),
                      np.ascontiguousarray(model.onsite, dtype=np.float64).reshape(-1, d, d) if len(model.onsite_class)
                      else np.zeros((1, d, d)),
                      np.ascontiguousarray(model.bond_rules, dtype=np.int32).reshape(-1, 4)]
        terms = (_BondTerm * max(1, len(model.bond_terms)))()
        for i, (c, a, ta, b, tb) in enumerate(model.bond_terms):
            terms[i] = _BondTerm(c, a, ta, b, tb)
        self._keep.append(terms)
        k = self._keep
        desc = _ModelDesc(d, k[0].ctypes.data, k[1].ctypes.data, len(model.op_names), k[2].ctypes.data,
                          k[3].ctypes.data, len(model.class_names), k[4].ctypes.data, len(model.onsite_class),
                          k[5].ctypes.data, k[6].ctypes.data, len(k[7]), k[7].ctypes.data, len(model.bond_terms),
                          C.cast(terms, C.c_void_p), float(model.density), int(model.Q))
        mode = refine if isinstance(refine, int) and not isinstance(refine, bool) else GpuSuperblock.REFINE[refine]
        opts = SysOpts(tol, max_iter, _prec(prec), mode, 1 if guess else 0, mixed_tol, tie_tol, seed)
        h = C.c_void_p()
        st = self.lib.dmrg_sys_create(C.byref(desc), self.L, self.m, C.byref(opts), C.byref(h))
        if st != 0:
            raise DmrgError(st, "dmrg_sys_create failed (see stderr)")
        self.h = h

    def _check(self, st, ok=(0,)):
        if st not in ok:
            raise DmrgError(st, (self.lib.dmrg_sys_last_error(self.h) or b"").decode())

    @staticmethod
    def _steps(arr, n):
        return [{k: getattr(arr[i], k) for k, _ in StepInfo._fields_} for i in range(n)]

    def infinite(self):
        """L/2 - 1 infinite-algorithm steps; one dict per step."""
        n_max = self.L // 2 - 1
        arr = (StepInfo * n_max)()
        n = C.c_int32()
        self._check(self.lib.dmrg_sys_infinite(self.h, arr, C.byref(n)), ok=(0, 4))
        return self._steps(arr, n.value)

    def sweeps(self, n_sweeps):
        """Finite-algorithm sweeps at fixed L (2 (L - 3) steps each)."""
        n_max = max(1, n_sweeps * 2 * (self.L - 3))
        arr = (StepInfo * n_max)()
        n = C.c_int32()
        self._check(self.lib.dmrg_sys_sweeps(self.h, int(n_sweeps), arr, C.byref(n)), ok=(0, 4))
        return self._steps(arr, n.value)

    def last_superblock(self):
        """The last step's superblock as a workloads Superblock (host copies)
        and its ground state (numpy [D])."""
        from workloads.superblock import Pair, Superblock
        v = _SbView()
        self._check(self.lib.dmrg_sys_last_superblock(self.h, C.byref(v), None))
        d = v.desc
        S, nt, npairs = d.n_sectors, d.n_terms, d.n_pairs
        r = np.ctypeslib.as_array(C.cast(d.r, C.POINTER(C.c_int32)), shape=(S,)).astype(np.int64)
        c = np.ctypeslib.as_array(C.cast(d.c, C.POINTER(C.c_int32)), shape=(S,)).astype(np.int64)
        coeffs = np.ctypeslib.as_array(C.cast(d.coeffs, C.POINTER(C.c_double)), shape=(nt,)).copy()
        pairs_c = C.cast(d.pairs, C.POINTER(_Pair))
        pairs = []
        for i in range(npairs):
            p = pairs_c[i]
            ro, ri, co, ci = r[p.s_out], r[p.s_in], c[p.s_out], c[p.s_in]
            A = B = None
            if not p.flags & ID_A:
                A = np.ctypeslib.as_array(C.cast(p.A, C.POINTER(C.c_double)), shape=(int(ro), int(p.lda)))[:, :ri].copy()
            if not p.flags & ID_B:
                B = np.ctypeslib.as_array(C.cast(p.B, C.POINTER(C.c_double)), shape=(int(co), int(p.ldb)))[:, :ci].copy()
            pairs.append(Pair(int(p.term), int(p.s_out), int(p.s_in), A, B))
        sb = Superblock(r, c, coeffs[None, :], pairs)
        sb.term_class = np.ctypeslib.as_array(C.cast(v.term_class, C.POINTER(C.c_int32)), shape=(nt,)).copy()
        sb.term_mult = np.ctypeslib.as_array(C.cast(v.term_mult, C.POINTER(C.c_double)), shape=(nt,)).copy()
        sb.q_labels = np.ctypeslib.as_array(C.cast(v.sector_q, C.POINTER(C.c_int64)), shape=(S,)).copy()
        sb.class_names = list(self.model.class_names)
        sb.couplings = np.asarray(self.model.couplings, dtype=np.float64)[None, :].copy()
        sb.meta.update(L=v.L, nS=v.n_sys)
        psi = np.zeros(sb.dim)
        self._check(self.lib.dmrg_sys_last_superblock(self.h, C.byref(v), psi.ctypes.data))
        return sb, psi

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_sys_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sym_eig_batched(mats, stream=None):
    """Eigen-decompositions of symmetric float64 CUDA matrices (list of
    [n, n] tensors): returns [(w decreasing, V with eigenvectors as columns)]."""
    lib = load()
    mats = [m.contiguous() for m in mats]
    ws = [torch.empty(m.shape[0], dtype=torch.float64, device=m.device) for m in mats]
    Vs = [torch.empty_like(m) for m in mats]
    cnt = len(mats)
    n = np.array([m.shape[0] for m in mats], dtype=np.int32)
    pa = (C.c_void_p * max(1, cnt))(*[_ptr(m) for m in mats])
    pv = (C.c_void_p * max(1, cnt))(*[_ptr(v) for v in Vs])
    pw = (C.c_void_p * max(1, cnt))(*[_ptr(w) for w in ws])
    st = lib.dmrg_sym_eig_batched(cnt, n.ctypes.data, C.cast(pa, C.c_void_p), C.cast(pv, C.c_void_p),
                                  C.cast(pw, C.c_void_p), _stream(stream))
    if st != 0:
        raise DmrgError(st, "sym_eig_batched")
    return list(zip(ws, Vs))
