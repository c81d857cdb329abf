"""Pins of the oracle's Dirac operators against the paper and plain mathematics.

Sec. 2, Eq. (3) (factorisation), Eq. (4) (det D-tilde), Hermiticity of
H = gamma_5 R_5 D_EOFA, the adjoint, gauge covariance, and the free-field
spectrum in momentum space.
"""
import itertools

import numpy as np
import pytest

from oracle import dwf, eofa
from paper_1611_00298_gb300 import inputs
from tests._dense import dense

DIMS = (2, 2, 2, 2)


def _rand(dims, Ls, seed):
    return inputs.fermion5d(dims, Ls, seed, stream=11)


def test_gamma_matrices_clifford_and_chiral():
    g = dwf.GAMMA
    for m, n in itertools.product(range(4), repeat=2):
        assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
    assert np.allclose(dwf.GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("alpha,Ls,mf", [(2.0, 4, 0.04), (1.0, 3, 0.1), (4.0, 5, 0.3), (2.0, 1, 0.5)])
def test_factorisation_eq3(alpha, Ls, mf):
    U = inputs.gauge_field((2, 2, 2, 4), 0.5, 5)
    psi = _rand((2, 2, 2, 4), Ls, 1)
    lhs = dwf.dwf(U, psi, alpha, 1.8, mf, -1)
    rhs = dwf.deofa(U, dwf.dtilde(psi, alpha, mf), alpha, 1.8, mf, -1)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(lhs) < 1e-14


@pytest.mark.parametrize("alpha,Ls,mf", [(2.0, 4, 0.04), (2.0, 5, 0.04), (4.0, 3, 0.3), (1.0, 4, 0.2), (3.0, 6, 1.0)])
def test_det_dtilde_eq4(alpha, Ls, mf):
    # Eq. (4), with the sign of the c-d term written for any Ls:
    # det D-tilde = ((c+d)^Ls + m_f (d-c)^Ls)^(12 V); as printed it holds for even Ls.
    c, d = dwf.coefficients(alpha)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    M = dense(lambda v: dwf.dtilde(v, alpha, mf), shape)
    sign, logdet = np.linalg.slogdet(M)
    N = (c + d) ** Ls + mf * (d - c) ** Ls
    V = 16
    assert np.isclose(logdet, 12 * V * np.log(abs(N)), rtol=1e-13, atol=1e-10)
    assert np.isclose(sign, np.sign(N) ** (12 * V))
    if Ls % 2 == 0:
        printed = (c + d) ** Ls + mf * (c - d) ** Ls
        assert np.isclose(printed, N)


def test_adjoint():
    U = inputs.gauge_field((2, 4, 2, 2), 0.7, 6)
    for alpha, mf in ((2.0, 0.04), (1.0, 0.5)):
        psi, chi = _rand((2, 4, 2, 2), 4, 1), _rand((2, 4, 2, 2), 4, 2)
        lhs = np.vdot(chi, dwf.dwf(U, psi, alpha, 1.8, mf, -1))
        rhs = np.vdot(dwf.dwf_dag(U, chi, alpha, 1.8, mf, -1), psi)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)
        lhs = np.vdot(chi, dwf.wilson(U, psi, 1.8, -1))
        rhs = np.vdot(dwf.wilson(U, chi, 1.8, -1, dagger=True), psi)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_moebius_dwf_not_g5r5_hermitian_but_H_is():
    U = inputs.gauge_field(DIMS, 0.5, 7)
    psi, chi = _rand(DIMS, 4, 1), _rand(DIMS, 4, 2)
    g5r5 = lambda v: dwf.gamma5(dwf.R5(v))  # noqa: E731
    for mf in (0.04, 1.0):
        lhs = np.vdot(chi, dwf.hermitian_H(U, psi, 2.0, 1.8, mf, -1))
        rhs = np.vdot(dwf.hermitian_H(U, chi, 2.0, 1.8, mf, -1), psi)
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    lhs = np.vdot(chi, g5r5(dwf.dwf(U, psi, 2.0, 1.8, 0.04, -1)))
    rhs = np.vdot(g5r5(dwf.dwf(U, chi, 2.0, 1.8, 0.04, -1)), psi)
    assert abs(lhs - rhs) > 1e-3 * abs(lhs)
    # Shamir (alpha = 1) D_DWF is gamma_5 R_5 Hermitian.
    lhs = np.vdot(chi, g5r5(dwf.dwf(U, psi, 1.0, 1.8, 0.04, -1)))
    rhs = np.vdot(g5r5(dwf.dwf(U, chi, 1.0, 1.8, 0.04, -1)), psi)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_gauge_covariance():
    dims = (2, 2, 4, 2)
    U = inputs.gauge_field(dims, 0.6, 8)
    g = inputs.gauge_transform(dims, 8)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = dwf.shift_links(g, mu, +1)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    psi = _rand(dims, 4, 3)
    gpsi = lambda v: np.einsum("...ab,...sb->...sa", g, v)  # noqa: E731
    for op in (dwf.dwf, dwf.dwf_dag, dwf.deofa):
        lhs = op(Ug, gpsi(psi), 2.0, 1.8, 0.04, -1)
        rhs = gpsi(op(U, psi, 2.0, 1.8, 0.04, -1))
        assert np.linalg.norm(lhs - rhs) < 1e-13 * np.linalg.norm(rhs)


@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (2, 2, 2, 2)])
def test_free_field_momentum_space(dims):
    # U = 1, periodic: D_w e^{ipx} u = e^{ipx} [4 - M5 - sum cos p + i sum g_mu sin p] u.
    X, Y, Z, T = dims
    Ls, alpha, M5, mf = 4, 2.0, 1.8, 0.3
    c, d = dwf.coefficients(alpha)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (T, Z, Y, X, 4, 3, 3)).copy()
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    rng = np.random.default_rng(0)
    for n in [(0, 0, 0, 0), (1, 0, 1, 1), (1, 1, 0, 3)]:
        p = [2 * np.pi * n[i] / dims[i] for i in range(4)]
        wave = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        u = rng.standard_normal((Ls, 4, 3)) + 1j * rng.standard_normal((Ls, 4, 3))
        psi = wave[None, :, :, :, :, None, None] * u[:, None, None, None, None]
        Dw = (4 - M5 - sum(np.cos(p))) * np.eye(4) + 1j * sum(dwf.GAMMA[m] * np.sin(p[m]) for m in range(4))
        # 5D matrix in (s, spin): (c+d) Dw + 1 on the diagonal, ((c-d) Dw - 1) L.
        Lp = np.zeros((Ls, Ls))
        Lp[np.arange(1, Ls), np.arange(Ls - 1)] = 1
        Lp[0, Ls - 1] = -mf
        Pp, Pm = np.diag([1.0, 1, 0, 0]), np.diag([0.0, 0, 1, 1])
        Lfull = np.kron(Lp, Pp) + np.kron(Lp.T, Pm)
        Dfull = np.kron(np.eye(Ls), (c + d) * Dw + np.eye(4)) + np.kron(np.eye(Ls), (c - d) * Dw - np.eye(4)) @ Lfull
        expect_u = np.einsum("ij,jc->ic", Dfull, u.reshape(Ls * 4, 3)).reshape(Ls, 4, 3)
        expect = wave[None, :, :, :, :, None, None] * expect_u[:, None, None, None, None]
        got = dwf.dwf(U, psi, alpha, M5, mf, +1)
        assert np.linalg.norm(got - expect) < 1e-13 * np.linalg.norm(expect)
        if n == (0, 0, 0, 0):
            # closed form per chirality block at p = 0: det(B + C L) = B^Ls + m_f (-C)^Ls
            B, C = 1 - (c + d) * M5, -((c - d) * M5 + 1)
            det = np.linalg.det(Dfull)
            assert np.isclose(det, (B ** Ls + mf * (-C) ** Ls) ** 4, rtol=1e-12)


def test_antiperiodic_phase_only_on_t_boundary():
    dims = (2, 2, 2, 4)
    U = inputs.gauge_field(dims, 0.4, 9)
    psi = _rand(dims, 2, 4)
    a = dwf.wilson(U, psi, 1.8, -1)
    b = dwf.wilson(U, psi, 1.8, +1)
    diff = np.linalg.norm((a - b).reshape(2, 4, -1), axis=(0, 2))
    assert diff[1] < 1e-14 and diff[2] < 1e-14
    assert diff[0] > 1e-3 and diff[3] > 1e-3


def test_delta_rank_one_closed_form():
    for alpha, Ls, m1, m2 in ((2.0, 8, 0.04, 1.0), (1.0, 4, 0.1, 0.5), (4.0, 5, 0.0362, 1.0), (2.0, 24, 0.0362, 1.0)):
        Dp, Dm = eofa.delta_matrices(Ls, alpha, m1, m2)
        Op, Om = eofa.omega(Ls, alpha)
        k = eofa.k_coefficient(Ls, alpha, m1, m2)
        assert np.abs(Dp - k * np.outer(Op, Op)).max() < 1e-13 * max(1.0, np.abs(Dp).max())
        assert np.abs(Dm - k * np.outer(Om, Om)).max() < 1e-13 * max(1.0, np.abs(Dm).max())
        assert np.linalg.matrix_rank(Dp, tol=1e-10) == 1
        if alpha == 1.0:  # Shamir: Omega_+ = e_{Ls-1}, Omega_- = e_0, k = m2 - m1
            assert np.allclose(Op, np.eye(Ls)[Ls - 1]) and np.allclose(Om, np.eye(Ls)[0])
            assert np.isclose(k, m2 - m1)


def test_h_shift_identity():
    # H(m2) - Delta_+ P_+ = H(m1) - Delta_- P_-  (both sides act on 5D fields)
    U = inputs.gauge_field(DIMS, 0.5, 10)
    psi = _rand(DIMS, 6, 5)
    a = eofa.system_apply(U, psi, 2.0, 1.8, 0.04, 1.0, "R", -1.0, -1)
    b = eofa.system_apply(U, psi, 2.0, 1.8, 0.04, 1.0, "L", -1.0, -1)
    assert np.linalg.norm(a - b) < 1e-13 * np.linalg.norm(a)


def test_single_site_hop_matches_whole_field():
    dims = (4, 2, 2, 4)
    U = inputs.gauge_field(dims, 0.6, 12)
    psi = _rand(dims, 3, 9)
    for bc in (-1, 1):
        for dag in (False, True):
            full = dwf.wilson_hop(U, psi, bc, dagger=dag)
            for site in ((0, 0, 0, 0), (3, 1, 1, 3), (3, 0, 1, 2), (1, 1, 0, 0)):
                for s in range(3):
                    got = dwf.wilson_hop_at(U, psi, site, s, bc, dagger=dag)
                    assert np.abs(got - full[(s,) + site]).max() < 1e-14
