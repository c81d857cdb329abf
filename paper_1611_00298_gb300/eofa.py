"""Thin ctypes binding of libeofa (include/eofa.h).

Argument marshalling only: every operator, solve, reduction and force runs
in the CUDA kernels of libeofa.  Host-buffer calls take numpy complex128
arrays in the canonical layouts; "_dev" calls take CUDA torch tensors
(complex128 or float64 views of the same layout) and use the current torch
stream.  There is no CPU fallback: if the library is not built or no GPU is
present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libeofa.so")

OK, EINVAL, ENOMEM, ENOTCONV, ENUMERIC, ETIMEOUT, EDEVICE = 0, -1, -2, -3, -4, -5, -6
PREC_F64, PREC_MIXED_F32, PREC_MIXED_F16 = 0, 1, 2
SYS_DWF, SYS_EOFA_L, SYS_EOFA_R = 0, 1, 2

# every symbol declared in include/eofa.h
EXPORTS = [
    "eofa_create", "eofa_destroy", "eofa_last_error", "eofa_gauge_load", "eofa_gauge_load_dev",
    "eofa_dwf_apply", "eofa_dwf_apply_dev", "eofa_eofa_apply", "eofa_eofa_apply_dev",
    "eofa_field_bytes", "eofa_hop_dev", "eofa_pack_dev", "eofa_unpack_dev",
    "eofa_solve", "eofa_solve_dev", "eofa_action", "eofa_action_dev", "eofa_force", "eofa_force_dev",
    "eofa_force_from_chi_dev", "eofa_grad_from_chi_dev", "eofa_coefficients", "eofa_link_update_dev",
    "eofa_solve_batched", "eofa_kernel_launches", "eofa_profile_start", "eofa_profile_stop",
    "eofa_dwf_apply_noalloc", "eofa_schur_hop_dev", "eofa_pseudofermion_solutions_dev",
    "eofa_set_reliable_delta", "eofa_leapfrog_dev", "eofa_rational_inv_sqrt", "eofa_heatbath_dev",
    "eofa_gauge_action_dev", "eofa_gauge_force_dev", "eofa_hmc_trajectory_dev", "eofa_force_parts_dev",
    "eofa_check_device", "eofa_hmc_dev", "eofa_probe_fp64_fma", "eofa_checkpoint_write", "eofa_checkpoint_read",
    "eofa_gauge_save", "eofa_gauge_restore", "eofa_set_cg_form", "eofa_get_cg_form",
]
CKPT_GAUGE, CKPT_MOMENTA = 0, 1
CG_FORM_AUTO, CG_FORM_FIVE, CG_FORM_SIX = -1, 0, 1
INT_LEAPFROG, INT_FG_PQPQP, INT_FG_QPQPQ = 0, 1, 2


class EOFAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libeofa error {code}: {msg}")
        self.code = code


class SolveParams(ctypes.Structure):
    _fields_ = [("Ls", ctypes.c_int), ("alpha", ctypes.c_double), ("M5", ctypes.c_double),
                ("system", ctypes.c_int), ("mf", ctypes.c_double), ("m1", ctypes.c_double),
                ("m2", ctypes.c_double), ("shift", ctypes.c_double), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("delta", ctypes.c_double),
                ("use_x0", ctypes.c_int)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * 6), ("ms", ctypes.c_double * 6), ("bytes", ctypes.c_double * 6)]


class MDParams(ctypes.Structure):
    _fields_ = [("Ls", ctypes.c_int), ("alpha", ctypes.c_double), ("M5", ctypes.c_double), ("m1", ctypes.c_double),
                ("m2", ctypes.c_double), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("beta", ctypes.c_double), ("integrator", ctypes.c_int), ("nsteps", ctypes.c_int),
                ("tau", ctypes.c_double), ("n_inner", ctypes.c_int), ("split_lr", ctypes.c_int),
                ("n_middle", ctypes.c_int)]


class MDInfo(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double), ("dH", ctypes.c_double), ("kinetic0", ctypes.c_double),
                ("kinetic1", ctypes.c_double), ("S_gauge0", ctypes.c_double), ("S_gauge1", ctypes.c_double),
                ("S_eofa0", ctypes.c_double), ("S_eofa1", ctypes.c_double), ("fermion_forces", ctypes.c_int),
                ("gauge_forces", ctypes.c_int), ("solver_iters", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HMCTrajInfo(ctypes.Structure):
    _fields_ = [("H0", ctypes.c_double), ("dH", ctypes.c_double), ("exp_minus_dH", ctypes.c_double),
                ("accepted", ctypes.c_int), ("plaquette", ctypes.c_double), ("S_eofa_start", ctypes.c_double),
                ("eta_norm2", ctypes.c_double), ("solver_iters", ctypes.c_int), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_resid", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int), ("low_updates", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libeofa.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1611_00298_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "eofa_create": (I, [ctypes.POINTER(P), ctypes.POINTER(I), I, I, I]),
        "eofa_destroy": (I, [P]),
        "eofa_last_error": (ctypes.c_char_p, [P]),
        "eofa_gauge_load": (I, [P, P]),
        "eofa_gauge_load_dev": (I, [P, P, P]),
        "eofa_dwf_apply": (I, [P, I, D, D, D, I, P, P]),
        "eofa_dwf_apply_dev": (I, [P, I, D, D, D, I, P, P, P]),
        "eofa_eofa_apply": (I, [P, I, D, D, D, P, P]),
        "eofa_eofa_apply_dev": (I, [P, I, D, D, D, P, P, P]),
        "eofa_field_bytes": (LL, [P, I]),
        "eofa_hop_dev": (I, [P, I, I, I, P, P, P]),
        "eofa_schur_hop_dev": (I, [P, I, I, I, I, D, D, D, P, P, P]),
        "eofa_pack_dev": (I, [P, I, P, P, P, P]),
        "eofa_unpack_dev": (I, [P, I, P, P, P, P]),
        "eofa_solve": (I, [P, ctypes.POINTER(SolveParams), P, P, ctypes.POINTER(SolveInfo)]),
        "eofa_solve_dev": (I, [P, ctypes.POINTER(SolveParams), P, P, ctypes.POINTER(SolveInfo), P]),
        "eofa_action": (I, [P, I, D, D, D, D, I, D, P, ctypes.POINTER(D), ctypes.POINTER(SolveInfo)]),
        "eofa_action_dev": (I, [P, I, D, D, D, D, I, D, P, ctypes.POINTER(D), ctypes.POINTER(SolveInfo), P]),
        "eofa_force": (I, [P, I, D, D, D, D, I, D, P, P, ctypes.POINTER(D), ctypes.POINTER(SolveInfo)]),
        "eofa_force_dev": (I, [P, I, D, D, D, D, I, D, P, P, ctypes.POINTER(D), ctypes.POINTER(SolveInfo), P]),
        "eofa_force_from_chi_dev": (I, [P, D, P, P, P, P]),
        "eofa_grad_from_chi_dev": (I, [P, D, P, P, P, P]),
        "eofa_coefficients": (I, [I, D, D, D, ctypes.POINTER(D), P, P]),
        "eofa_link_update_dev": (I, [P, D, P, P, P]),
        "eofa_solve_batched": (I, [ctypes.POINTER(P), I, ctypes.POINTER(SolveParams), ctypes.POINTER(P),
                                   ctypes.POINTER(P), ctypes.POINTER(SolveInfo)]),
        "eofa_kernel_launches": (LL, []),
        "eofa_dwf_apply_noalloc": (I, [P, I, D, D, D, I, P, P, P]),
        "eofa_pseudofermion_solutions_dev": (I, [P, I, D, D, D, D, I, D, P, P, P, ctypes.POINTER(D),
                                                 ctypes.POINTER(SolveInfo), P]),
        "eofa_set_reliable_delta": (I, [P, D]),
        "eofa_set_cg_form": (I, [P, I, I]),
        "eofa_get_cg_form": (I, [P, I, ctypes.POINTER(I)]),
        "eofa_gauge_action_dev": (I, [P, D, P, ctypes.POINTER(D), P]),
        "eofa_check_device": (I, [P, P]),
        "eofa_force_parts_dev": (I, [P, I, D, D, D, D, I, D, P, P, P, ctypes.POINTER(SolveInfo), P]),
        "eofa_gauge_force_dev": (I, [P, D, P, P, I, P]),
        "eofa_hmc_trajectory_dev": (I, [P, ctypes.POINTER(MDParams), P, P, P, ctypes.POINTER(MDInfo), P]),
        "eofa_rational_inv_sqrt": (I, [I, D, D, ctypes.POINTER(D), P, P, ctypes.POINTER(D)]),
        "eofa_heatbath_dev": (I, [P, I, D, D, D, D, I, D, I, D, P, P, P, P, I, ctypes.POINTER(SolveInfo), P]),
        "eofa_leapfrog_dev": (I, [P, I, D, D, D, D, I, D, I, D, P, P, P, ctypes.POINTER(D), ctypes.POINTER(D), P]),
        "eofa_hmc_dev": (I, [P, ctypes.POINTER(MDParams), I, D, I, P, P, P, P, P, P, ctypes.POINTER(HMCTrajInfo), P]),
        "eofa_probe_fp64_fma": (I, [ctypes.POINTER(D)]),
        "eofa_checkpoint_write": (I, [ctypes.c_char_p, I, ctypes.POINTER(I), LL, P]),
        "eofa_checkpoint_read": (I, [ctypes.c_char_p, I, ctypes.POINTER(I), ctypes.POINTER(LL), P]),
        "eofa_gauge_save": (I, [P, ctypes.c_char_p, LL]),
        "eofa_gauge_restore": (I, [P, ctypes.c_char_p, ctypes.POINTER(LL)]),
        "eofa_profile_start": (I, [P]),
        "eofa_profile_stop": (I, [P, ctypes.POINTER(Profile)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> int:
    """Address of a numpy array (C-contiguous) or a torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    assert a.is_contiguous(), "tensors must be contiguous"
    return a.data_ptr()


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def kernel_launches() -> int:
    """Number of CUDA kernels libeofa has launched since it was loaded."""
    return int(load_library().eofa_kernel_launches())


def probe_fp64_fma() -> float:
    """Measured FP64 FMA rate of the current GPU in TFLOP/s."""
    v = ctypes.c_double()
    rc = load_library().eofa_probe_fp64_fma(ctypes.byref(v))
    if rc != OK:
        raise EOFAError(rc, "eofa_probe_fp64_fma")
    return v.value


def checkpoint_write(path, kind, field, traj=0):
    """Write a gauge field or momenta (host canonical, shape (T, Z, Y, X, 4, 3, 3)) to a checkpoint."""
    f = np.ascontiguousarray(field, dtype=np.complex128)
    T, Z, Y, X = f.shape[:4]
    dims = (ctypes.c_int * 4)(X, Y, Z, T)
    rc = load_library().eofa_checkpoint_write(os.fsencode(path), kind, dims, int(traj), f.ctypes.data)
    if rc != OK:
        raise EOFAError(rc, f"eofa_checkpoint_write {path}")


def checkpoint_read(path, kind, dims):
    """Read a checkpoint of a lattice dims = (X, Y, Z, T); returns (field, trajectory number)."""
    X, Y, Z, T = dims
    f = np.empty((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    traj = ctypes.c_longlong()
    rc = load_library().eofa_checkpoint_read(os.fsencode(path), kind, (ctypes.c_int * 4)(*dims), ctypes.byref(traj),
                                             f.ctypes.data)
    if rc != OK:
        raise EOFAError(rc, f"eofa_checkpoint_read {path}")
    return f, traj.value


def rational_inv_sqrt(npoles, lmin, lmax):
    """(alpha0, alpha[], beta[], max relative error) of x^-1/2 ~ alpha0 + sum alpha/(x + beta) on [lmin, lmax]."""
    lib = load_library()
    a0 = ctypes.c_double()
    err = ctypes.c_double()
    al = np.zeros(npoles)
    be = np.zeros(npoles)
    rc = lib.eofa_rational_inv_sqrt(npoles, lmin, lmax, ctypes.byref(a0), al.ctypes.data, be.ctypes.data,
                                    ctypes.byref(err))
    if rc != OK:
        raise EOFAError(rc, "eofa_rational_inv_sqrt")
    return a0.value, al, be, err.value


def coefficients(Ls, alpha, m1, m2):
    """(k, Omega_+, Omega_-) of the EOFA rank-one factorisation (libeofa)."""
    lib = load_library()
    k = ctypes.c_double()
    Op = np.zeros(Ls)
    Om = np.zeros(Ls)
    rc = lib.eofa_coefficients(Ls, alpha, m1, m2, ctypes.byref(k), Op.ctypes.data, Om.ctypes.data)
    if rc != OK:
        raise EOFAError(rc, "eofa_coefficients")
    return k.value, Op, Om


@dataclass
class Params:
    alpha: float = 2.0
    M5: float = 1.8


class Lattice:
    """One lattice (dims = (X, Y, Z, T), Ls, time boundary phase) on the current GPU."""

    def __init__(self, dims, Ls, bc_t=-1):
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.bc_t = int(bc_t)
        X, Y, Z, T = self.dims
        self.V = X * Y * Z * T
        self.ctx = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        rc = self.lib.eofa_create(ctypes.byref(self.ctx), arr, self.Ls, self.bc_t, 0)
        if rc != OK:
            raise EOFAError(rc, "eofa_create failed (bad dims/Ls/bc or no CUDA device)")

    def close(self):
        if self.ctx:
            self.lib.eofa_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != OK:
            msg = self.lib.eofa_last_error(self.ctx)
            raise EOFAError(rc, f"{what}: {msg.decode() if msg else ''}")

    # -- shapes
    @property
    def shape5(self):
        X, Y, Z, T = self.dims
        return (self.Ls, T, Z, Y, X, 4, 3)

    @property
    def shape4(self):
        X, Y, Z, T = self.dims
        return (T, Z, Y, X, 4, 3)

    @property
    def shapeU(self):
        X, Y, Z, T = self.dims
        return (T, Z, Y, X, 4, 3, 3)

    # -- host-buffer calls
    def gauge_load(self, U):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        assert U.shape == self.shapeU
        self._check(self.lib.eofa_gauge_load(self.ctx, _ptr(U)), "gauge_load")

    def gauge_load_dev(self, U):
        self._check(self.lib.eofa_gauge_load_dev(self.ctx, _ptr(U), _stream()), "gauge_load_dev")

    def dwf_apply(self, psi, alpha, M5, mf, dagger=False):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(psi)
        self._check(self.lib.eofa_dwf_apply(self.ctx, self.Ls, alpha, M5, mf, int(dagger), _ptr(psi), _ptr(out)),
                     "dwf_apply")
        return out

    def eofa_apply(self, psi, alpha, M5, mf):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        out = np.empty_like(psi)
        self._check(self.lib.eofa_eofa_apply(self.ctx, self.Ls, alpha, M5, mf, _ptr(psi), _ptr(out)), "eofa_apply")
        return out

    def solve_params(self, system=SYS_DWF, alpha=2.0, M5=1.8, mf=0.0, m1=0.0, m2=0.0, shift=0.0,
                     precision=PREC_F64, tol=1e-10, maxiter=100000, delta=0.0, use_x0=False):
        return SolveParams(self.Ls, alpha, M5, system, mf, m1, m2, shift, precision, tol, maxiter, delta,
                           int(use_x0))

    def solve(self, b, x0=None, check=True, **kw):
        """Solve one system; with check=False a failure status is returned in info.status
        instead of raised."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        p = self.solve_params(use_x0=x0 is not None, **kw)
        x = np.zeros_like(b) if x0 is None else np.ascontiguousarray(x0, dtype=np.complex128).copy()
        info = SolveInfo()
        rc = self.lib.eofa_solve(self.ctx, ctypes.byref(p), _ptr(b), _ptr(x), ctypes.byref(info))
        if check:
            self._check(rc, "solve")
        else:
            info.status = rc
        return x, info

    def action(self, phi, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10):
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        S = ctypes.c_double()
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_action(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi), ctypes.byref(S),
                                  info)
        self._check(rc, "action")
        return S.value, info

    def force(self, phi, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10, out=None):
        phi = np.ascontiguousarray(phi, dtype=np.complex128)
        F = np.empty(self.shapeU, dtype=np.complex128) if out is None else out
        assert F.shape == self.shapeU and F.dtype == np.complex128 and F.flags["C_CONTIGUOUS"]
        S = ctypes.c_double()
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_force(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi), _ptr(F),
                                 ctypes.byref(S), info)
        self._check(rc, "force")
        return F, S.value, info

    # -- device calls (torch tensors)
    def field_bytes(self, precision):
        return int(self.lib.eofa_field_bytes(self.ctx, precision))

    def hop_dev(self, precision, out_parity, dagger, inp, out):
        self._check(self.lib.eofa_hop_dev(self.ctx, precision, out_parity, int(dagger), _ptr(inp), _ptr(out),
                                          _stream()), "hop_dev")

    def schur_hop_dev(self, precision, out_parity, dagger, inp, out, alpha, M5, mf):
        """out = G^-1 D_hop in (dagger: G^-T D_hop^+ in), one fused kernel."""
        self._check(self.lib.eofa_schur_hop_dev(self.ctx, precision, out_parity, int(dagger), self.Ls, alpha, M5, mf,
                                                _ptr(inp), _ptr(out), _stream()), "schur_hop_dev")

    def pack_dev(self, precision, canon, even, odd):
        self._check(self.lib.eofa_pack_dev(self.ctx, precision, _ptr(canon), _ptr(even), _ptr(odd), _stream()),
                    "pack_dev")

    def unpack_dev(self, precision, even, odd, canon):
        self._check(self.lib.eofa_unpack_dev(self.ctx, precision, _ptr(even), _ptr(odd), _ptr(canon), _stream()),
                    "unpack_dev")

    def dwf_apply_dev(self, psi, out, alpha, M5, mf, dagger=False):
        self._check(self.lib.eofa_dwf_apply_dev(self.ctx, self.Ls, alpha, M5, mf, int(dagger), _ptr(psi), _ptr(out),
                                                _stream()), "dwf_apply_dev")

    def dwf_apply_noalloc_dev(self, psi, out, alpha, M5, mf, dagger=False):
        """D_DWF (or D_DWF^+) without device allocation; see eofa_dwf_apply_noalloc in include/eofa.h."""
        self._check(self.lib.eofa_dwf_apply_noalloc(self.ctx, self.Ls, alpha, M5, mf, int(dagger), _ptr(psi),
                                                    _ptr(out), _stream()), "dwf_apply_noalloc")

    def solve_dev(self, b, x, use_x0=False, check=True, **kw):
        p = self.solve_params(use_x0=use_x0, **kw)
        info = SolveInfo()
        rc = self.lib.eofa_solve_dev(self.ctx, ctypes.byref(p), _ptr(b), _ptr(x), ctypes.byref(info), _stream())
        if check:
            self._check(rc, "solve_dev")
        else:
            info.status = rc
        return info

    def action_dev(self, phi, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10):
        S = ctypes.c_double()
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_action_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi),
                                      ctypes.byref(S), info, _stream())
        self._check(rc, "action_dev")
        return S.value, info

    def force_dev(self, phi, F, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10):
        S = ctypes.c_double()
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_force_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi), _ptr(F),
                                     ctypes.byref(S), info, _stream())
        self._check(rc, "force_dev")
        return S.value, info

    def force_from_chi_dev(self, k, chiL, chiR, F):
        self._check(self.lib.eofa_force_from_chi_dev(self.ctx, k, _ptr(chiL), _ptr(chiR), _ptr(F), _stream()),
                    "force_from_chi_dev")

    def grad_from_chi_dev(self, k, chiL, chiR, G):
        self._check(self.lib.eofa_grad_from_chi_dev(self.ctx, k, _ptr(chiL), _ptr(chiR), _ptr(G), _stream()),
                    "grad_from_chi_dev")

    def profile_start(self):
        self._check(self.lib.eofa_profile_start(self.ctx), "profile_start")

    def profile_stop(self):
        """Per-kind (hop FP64/FP32/FP16, 5D-local FP64/FP32/FP16) launch counts, milliseconds and
        algorithmic bytes."""
        pr = Profile()
        self._check(self.lib.eofa_profile_stop(self.ctx, ctypes.byref(pr)), "profile_stop")
        return list(pr.launches), list(pr.ms), list(pr.bytes)

    def pseudofermion_solutions_dev(self, phi, chiL, chiR, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10):
        """chi_L, chi_R of Eq. (5) / (7) into the given device tensors; returns (S, info)."""
        S = ctypes.c_double()
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_pseudofermion_solutions_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi),
                                                       _ptr(chiL), _ptr(chiR), ctypes.byref(S), info, _stream())
        self._check(rc, "pseudofermion_solutions_dev")
        return S.value, info

    def heatbath_dev(self, eta, phi, alpha, M5, m1, m2, alpha0, alphas, betas, precision=PREC_F64, tol=1e-10,
                     forecast=True):
        """phi = f(M_EOFA) eta (Eq. (6)); returns the 2 npoles solve records."""
        al = np.ascontiguousarray(alphas, dtype=np.float64)
        be = np.ascontiguousarray(betas, dtype=np.float64)
        info = (SolveInfo * (2 * len(al)))()
        rc = self.lib.eofa_heatbath_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, len(al), alpha0,
                                        al.ctypes.data, be.ctypes.data, _ptr(eta), _ptr(phi), int(forecast), info,
                                        _stream())
        self._check(rc, "heatbath_dev")
        return list(info)

    def set_reliable_delta(self, delta):
        self._check(self.lib.eofa_set_reliable_delta(self.ctx, delta), "set_reliable_delta")

    def set_cg_form(self, precision, form):
        """CG iteration form at one precision: CG_FORM_AUTO, CG_FORM_FIVE or CG_FORM_SIX."""
        self._check(self.lib.eofa_set_cg_form(self.ctx, precision, form), "set_cg_form")

    def cg_form(self, precision):
        """The form in use at one precision (CG_FORM_AUTO while undecided)."""
        f = ctypes.c_int()
        self._check(self.lib.eofa_get_cg_form(self.ctx, precision, ctypes.byref(f)), "get_cg_form")
        return f.value

    def leapfrog_dev(self, phi, P, U, alpha, M5, m1, m2, nsteps, dtau, precision=PREC_F64, tol=1e-10):
        """Leapfrog trajectory (P, U updated in place on the device); returns (dH, H0)."""
        dH = ctypes.c_double()
        H0 = ctypes.c_double()
        rc = self.lib.eofa_leapfrog_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, nsteps, dtau, _ptr(phi),
                                        _ptr(P), _ptr(U) if U is not None else None, ctypes.byref(dH),
                                        ctypes.byref(H0), _stream())
        self._check(rc, "leapfrog_dev")
        return dH.value, H0.value

    def force_parts_dev(self, phi, FL, FR, alpha, M5, m1, m2, precision=PREC_F64, tol=1e-10):
        """Forces of S_L and S_R separately (either output may be None); returns the two solve records."""
        info = (SolveInfo * 2)()
        rc = self.lib.eofa_force_parts_dev(self.ctx, self.Ls, alpha, M5, m1, m2, precision, tol, _ptr(phi),
                                           _ptr(FL) if FL is not None else None, _ptr(FR) if FR is not None else None,
                                           info, _stream())
        self._check(rc, "force_parts_dev")
        return [info[0].as_dict(), info[1].as_dict()]

    def check_device(self):
        """Raise EOFAError (ETIMEOUT) if a staged dslash launch's bounded wait ran out since the last check."""
        self._check(self.lib.eofa_check_device(self.ctx, _stream()), "check_device")

    def gauge_action_dev(self, beta, U=None):
        """Wilson plaquette action of U (device canonical) or of the context's links."""
        S = ctypes.c_double()
        self._check(self.lib.eofa_gauge_action_dev(self.ctx, beta, _ptr(U) if U is not None else None,
                                                   ctypes.byref(S), _stream()), "gauge_action_dev")
        return S.value

    def gauge_force_dev(self, beta, F, U=None, accumulate=False):
        self._check(self.lib.eofa_gauge_force_dev(self.ctx, beta, _ptr(U) if U is not None else None, _ptr(F),
                                                  int(accumulate), _stream()), "gauge_force_dev")

    def hmc_trajectory_dev(self, P, phi=None, U=None, *, alpha=2.0, M5=1.8, m1=0.04, m2=1.0, precision=PREC_F64,
                           tol=1e-10, beta=0.0, integrator=INT_FG_QPQPQ, nsteps=4, tau=1.0, n_inner=0,
                           split_lr=False, n_middle=0):
        """One MD trajectory (P and the context's links updated in place); returns the info dict."""
        prm = MDParams(self.Ls, alpha, M5, m1, m2, precision, tol, beta, integrator, nsteps, tau, n_inner,
                       int(split_lr), n_middle)  # split_lr: 0 / False, 1 / True (S_R outer), 2 (S_L outer)
        info = MDInfo()
        rc = self.lib.eofa_hmc_trajectory_dev(self.ctx, ctypes.byref(prm), _ptr(phi) if phi is not None else None,
                                              _ptr(P), _ptr(U) if U is not None else None, ctypes.byref(info),
                                              _stream())
        self._check(rc, "hmc_trajectory_dev")
        return info.as_dict()

    def hmc_dev(self, Ps, etas, us, U=None, *, alpha=2.0, M5=1.8, m1=0.04, m2=1.0, precision=PREC_F64, tol=1e-10,
                beta=0.0, integrator=INT_FG_QPQPQ, nsteps=4, tau=1.0, n_inner=0, split_lr=False, n_middle=0,
                rational=None):
        """HMC chain of len(us) trajectories: heatbath refresh of phi from etas[k] (rational =
        (alpha0, alphas, betas) of f ~ x^-1/2; None: pure gauge, no pseudofermion), momenta Ps[k],
        Metropolis with us[k].  Ps, etas: device tensors with the trajectories stacked on the first
        axis.  The context's links end at the chain's last state; returns the list of records."""
        prm = MDParams(self.Ls, alpha, M5, m1, m2, precision, tol, beta, integrator, nsteps, tau, n_inner,
                       int(split_lr), n_middle)
        u = np.ascontiguousarray(us, dtype=np.float64)
        n = len(u)
        if rational is None:
            a0, al, be, npoles = 0.0, np.zeros(1), np.zeros(1), 0
        else:
            a0 = float(rational[0])
            al = np.ascontiguousarray(rational[1], dtype=np.float64)
            be = np.ascontiguousarray(rational[2], dtype=np.float64)
            npoles = len(al)
        info = (HMCTrajInfo * max(1, n))()
        rc = self.lib.eofa_hmc_dev(self.ctx, ctypes.byref(prm), n, a0, npoles, al.ctypes.data, be.ctypes.data,
                                   _ptr(Ps), _ptr(etas) if etas is not None else None, u.ctypes.data,
                                   _ptr(U) if U is not None else None, info, _stream())
        self._check(rc, "hmc_dev")
        return [info[k].as_dict() for k in range(n)]

    def gauge_save(self, path, traj=0):
        """Write the context's current links to a gauge checkpoint."""
        self._check(self.lib.eofa_gauge_save(self.ctx, os.fsencode(path), int(traj)), "gauge_save")

    def gauge_restore(self, path):
        """Load the links of a gauge checkpoint of this lattice; returns its trajectory number."""
        traj = ctypes.c_longlong()
        self._check(self.lib.eofa_gauge_restore(self.ctx, os.fsencode(path), ctypes.byref(traj)), "gauge_restore")
        return traj.value

    def link_update_dev(self, eps, P, U=None):
        self._check(self.lib.eofa_link_update_dev(self.ctx, eps, _ptr(P), _ptr(U) if U is not None else None,
                                                  _stream()), "link_update_dev")


def solve_batched(lattices, params, bs, xs, check=True):
    """Solve len(lattices) systems; params: list of SolveParams; bs, xs: numpy arrays.
    With check=False a failure status is left in the info records instead of raised."""
    lib = load_library()
    n = len(lattices)
    ctxs = (ctypes.c_void_p * n)(*[lat.ctx.value for lat in lattices])
    prm = (SolveParams * n)(*params)
    bp = (ctypes.c_void_p * n)(*[_ptr(b) for b in bs])
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    info = (SolveInfo * n)()
    rc = lib.eofa_solve_batched(ctxs, n, prm, bp, xp, info)
    if check and rc != OK:
        raise EOFAError(rc, "solve_batched")
    return info
