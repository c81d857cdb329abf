"""ctypes loader of the C restatement of the oracle (oracle/c/dwf_oracle.c).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the same D_w,
D_DWF (Eq. (3)) and CGNR as dwf.py and solve.py, written as plain C loops
over sites (OpenMP over 4D sites) so that the host cores can be timed on
the benchmark's lattices.  Built with gcc on first use (or by
``__graft_entry__.build()``); shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "c", "dwf_oracle.c")
LIB = os.path.join(_HERE, "c", "_build", "libdwf_oracle.so")
_lib = None


def build() -> str:
    """Compile the C oracle (gcc, OpenMP) if its library is missing or older than the source."""
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"gcc failed for {SRC}:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.oracle_threads.restype = I
        lib.oracle_set_threads.argtypes = [I]
        lib.oracle_wilson.argtypes = [P, I, P, P, P, D, D, I]
        lib.oracle_dwf.argtypes = [P, I, P, P, P, D, D, D, D]
        lib.oracle_dwf_dag.argtypes = [P, I, P, P, P, D, D, D, D]
        lib.oracle_cgnr_dwf.argtypes = [P, I, P, P, P, D, D, D, D, D, I, ctypes.POINTER(D), ctypes.POINTER(D)]
        lib.oracle_cgnr_dwf.restype = I
        _lib = lib
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data


def _dims(U):
    T, Z, Y, X = U.shape[:4]
    return (ctypes.c_int * 4)(X, Y, Z, T)


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def wilson(U, psi, M5, bc_t, dagger=False):
    """D_w psi (or D_w^+ psi) on every s-slice, as dwf.wilson."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_wilson(_dims(U), psi.shape[0], pu, pp, out.ctypes.data, M5, float(bc_t), int(dagger))
    return out


def dwf(U, psi, alpha, M5, mf, bc_t):
    """D_DWF psi, as dwf.dwf."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_dwf(_dims(U), psi.shape[0], pu, pp, out.ctypes.data, alpha, M5, mf, float(bc_t))
    return out


def dwf_dag(U, psi, alpha, M5, mf, bc_t):
    """D_DWF^+ psi, as dwf.dwf_dag."""
    U, pu = _c(U)
    psi, pp = _c(psi)
    out = np.empty_like(psi)
    _load().oracle_dwf_dag(_dims(U), psi.shape[0], pu, pp, out.ctypes.data, alpha, M5, mf, float(bc_t))
    return out


def cgnr_dwf(U, b, alpha, M5, mf, bc_t, tol=1e-12, maxiter=20000, x0=None, timing=False):
    """At most maxiter CGNR iterations on D_DWF x = b; returns (x, iterations, recursive |r| / |b|)
    and, with timing=True, also the wall seconds of the iterations (set-up excluded)."""
    U, pu = _c(U)
    b, pb = _c(b)
    x = np.zeros_like(b) if x0 is None else np.ascontiguousarray(x0, dtype=np.complex128).copy()
    rel = ctypes.c_double()
    loop = ctypes.c_double()
    it = _load().oracle_cgnr_dwf(_dims(U), b.shape[0], pu, pb, x.ctypes.data, alpha, M5, mf, float(bc_t), tol,
                                 int(maxiter), ctypes.byref(rel), ctypes.byref(loop))
    if timing:
        return x, int(it), rel.value, loop.value
    return x, int(it), rel.value
