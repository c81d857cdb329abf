"""Plain conjugate gradient on the normal equations (oracle; test infrastructure).

Sec. 5.1 states that the cost of an HMC trajectory lies in repeated
inversions of the Dirac operator.  The oracle inverts any operator A by the
textbook CGNR / CGLS iteration (Hestenes-Stiefel CG applied to A^+ A x = A^+ b,
tracking the residual r = b - A x), with no preconditioning, and stops on the
recomputed true residual |b - A x| / |b|.
"""
from __future__ import annotations

import numpy as np


def vdot(a, b) -> complex:
    return complex(np.vdot(a, b))


def norm2(a) -> float:
    return float(np.vdot(a, a).real)


def cgnr(A, Adag, b, tol=1e-12, maxiter=20000, x0=None):
    """Solve A x = b; returns (x, iterations, true relative residual)."""
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else x0.copy()
    it = 0
    while True:
        r = b - A(x)
        true_res = np.sqrt(norm2(r)) / bnorm
        if true_res <= tol or it >= maxiter:
            return x, it, true_res
        z = Adag(r)
        p = z.copy()
        zz = norm2(z)
        while it < maxiter:
            w = A(p)
            a = zz / norm2(w)
            x += a * p
            r -= a * w
            it += 1
            if np.sqrt(norm2(r)) / bnorm <= 0.5 * tol:
                break
            z = Adag(r)
            zz_new = norm2(z)
            p = z + (zz_new / zz) * p
            zz = zz_new
