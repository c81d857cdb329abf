"""The C restatement of the oracle (oracle/c/dwf_oracle.c) against what fixes it.

It is timed as the CPU baseline, so it must compute the same operators as
the pinned numpy oracle: the free-field momentum-space closed form of D_w
directly (Sec. 2), agreement with dwf.wilson / dwf.dwf / dwf.dwf_dag on
random gauge fields (both time boundary conditions, odd and even Ls), and a
CGNR solution whose residual the numpy operator confirms.
"""
import numpy as np
import pytest

from oracle import c_oracle, dwf
from paper_1611_00298_gb300 import inputs


def test_free_field_plane_wave():
    """U = 1, periodic: D_w e^{ipx} u = [4 - M5 - sum cos p + i sum gamma_mu sin p_mu] e^{ipx} u."""
    X, Y, Z, T = 4, 6, 2, 8
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[..., :, :] = np.eye(3)
    rng = np.random.default_rng(5)
    n = (1, 2, 1, 3)
    p = [2 * np.pi * n[k] / d for k, d in enumerate((X, Y, Z, T))]
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
    psi = (ph[..., None, None] * u)[None]
    M5 = 1.8
    Dp = (4 - M5 - sum(np.cos(pk) for pk in p)) * np.eye(4) + 1j * sum(
        dwf.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    want = (ph[..., None, None] * (Dp @ u))[None]
    got = c_oracle.wilson(U, psi, M5, 1.0)
    assert np.abs(got - want).max() < 1e-13
    # the adjoint has -i sum gamma sin p
    Dd = (4 - M5 - sum(np.cos(pk) for pk in p)) * np.eye(4) - 1j * sum(
        dwf.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
    got = c_oracle.wilson(U, psi, M5, 1.0, dagger=True)
    assert np.abs(got - (ph[..., None, None] * (Dd @ u))[None]).max() < 1e-13


@pytest.mark.parametrize("bc", [-1, 1])
@pytest.mark.parametrize("Ls,alpha", [(5, 2.0), (4, 1.0)])
def test_operators_match_numpy_oracle(bc, Ls, alpha):
    dims = (4, 2, 2, 4)
    U = inputs.gauge_field(dims, 0.6, 3)
    psi = inputs.fermion5d(dims, Ls, 1, stream=3)
    for dag in (False, True):
        ref = dwf.wilson(U, psi, 1.8, bc, dag)
        assert np.abs(c_oracle.wilson(U, psi, 1.8, bc, dag) - ref).max() < 1e-13 * np.abs(ref).max()
    ref = dwf.dwf(U, psi, alpha, 1.8, 0.1, bc)
    assert np.abs(c_oracle.dwf(U, psi, alpha, 1.8, 0.1, bc) - ref).max() < 1e-13 * np.abs(ref).max()
    ref = dwf.dwf_dag(U, psi, alpha, 1.8, 0.1, bc)
    assert np.abs(c_oracle.dwf_dag(U, psi, alpha, 1.8, 0.1, bc) - ref).max() < 1e-13 * np.abs(ref).max()


def test_cgnr_solves_dwf():
    dims, Ls = (4, 2, 2, 4), 6
    U = inputs.gauge_field(dims, 0.5, 7)
    b = inputs.fermion5d(dims, Ls, 2, stream=8)
    x, it, rel = c_oracle.cgnr_dwf(U, b, 2.0, 1.8, 0.1, -1, tol=1e-12)
    assert 0 < it < 2000 and rel <= 1e-12
    res = np.linalg.norm(b - dwf.dwf(U, x, 2.0, 1.8, 0.1, -1)) / np.linalg.norm(b)
    assert res < 1e-11
    # a bounded run stops at maxiter
    _, it3, rel3 = c_oracle.cgnr_dwf(U, b, 2.0, 1.8, 0.1, -1, tol=1e-12, maxiter=3)
    assert it3 == 3 and rel3 > 1e-6


def test_threads_setting():
    n = c_oracle.threads()
    assert n >= 1
    c_oracle.set_threads(1)
    assert c_oracle.threads() == 1
    c_oracle.set_threads(n)
    assert c_oracle.threads() == n
