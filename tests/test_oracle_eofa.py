"""Pins of the oracle's EOFA pieces: Eq. (1), (2), (5), (7), (8) and the CG.

Dense linear algebra on a 2^4 x Ls=4 lattice (768 x 768 5D matrices).
"""
import numpy as np
import pytest

from oracle import dwf, eofa, solve
from oracle import eofa as oeofa
from paper_1611_00298_gb300 import inputs
from tests._dense import dense

DIMS = (2, 2, 2, 2)
LS = 4
SHAPE5 = (LS, 2, 2, 2, 2, 4, 3)
SHAPE4 = (2, 2, 2, 2, 4, 3)
ALPHA, M5, M1, M2, BC = 2.0, 1.8, 0.04, 1.0, -1


@pytest.fixture(scope="module")
def U():
    return inputs.gauge_field(DIMS, 0.8, 1)


def _eofa_matrices(U, alpha, m1, m2):
    """Dense M_L (on P_- phi) and M_R (on P_+ phi) as 4D 12V x 12V matrices (Eq. (5))."""
    k = eofa.k_coefficient(LS, alpha, m1, m2)
    Op, Om = eofa.omega(LS, alpha)
    H1 = dense(lambda v: dwf.hermitian_H(U, v, alpha, M5, m1, BC), SHAPE5)
    HR = dense(lambda v: eofa.system_apply(U, v, alpha, M5, m1, m2, "R", -1.0, BC), SHAPE5)
    E_m = dense(lambda v: eofa.embed(v, Om, -1), SHAPE4)
    E_p = dense(lambda v: eofa.embed(v, Op, +1), SHAPE4)
    ML = np.eye(192) - k * E_m.conj().T @ np.linalg.solve(H1, E_m)
    MR = np.eye(192) + k * E_p.conj().T @ np.linalg.solve(HR, E_p)
    return ML, MR, H1, HR


def _chiral_block(M, chirality):
    idx = np.arange(192).reshape(16, 4, 3)
    spins = [0, 1] if chirality > 0 else [2, 3]
    sel = idx[:, spins, :].reshape(-1)
    return M[np.ix_(sel, sel)]


def test_eofa_determinant_identity_eq1_and_eq2(U):
    ML, MR, _, _ = _eofa_matrices(U, ALPHA, M1, M2)
    MLb, MRb = _chiral_block(ML, -1), _chiral_block(MR, +1)
    # M_L, M_R Hermitian positive definite (Sec. 2), spectrum near 1 (Sec. 3.2)
    for M in (MLb, MRb):
        assert np.abs(M - M.conj().T).max() < 1e-12
        ev = np.linalg.eigvalsh(M)
        assert ev.min() > 0 and ev.max() < 2
    _, logML = np.linalg.slogdet(MLb)
    _, logMR = np.linalg.slogdet(MRb)
    DE1 = dense(lambda v: dwf.deofa(U, v, ALPHA, M5, M1, BC), SHAPE5)
    DE2 = dense(lambda v: dwf.deofa(U, v, ALPHA, M5, M2, BC), SHAPE5)
    s1, l1 = np.linalg.slogdet(DE1)
    s2, l2 = np.linalg.slogdet(DE2)
    # Eq. (1): det[D(m1)/D(m2)] = 1 / (det M_L det M_R), D = D_EOFA
    assert np.isclose(s1 / s2, 1.0, atol=1e-8)
    assert abs((l1 - l2) + (logML + logMR)) < 1e-10 * abs(l1 - l2)
    # Eq. (2) with Eq. (4): 1/2 logdet[D^+D(m1) / D^+D(m2)] for D = D_DWF equals the
    # EOFA ratio plus the gauge-independent normalisation 12 V log|N(m1)/N(m2)|.
    DD1 = dense(lambda v: dwf.dwf(U, v, ALPHA, M5, M1, BC), SHAPE5)
    DD2 = dense(lambda v: dwf.dwf(U, v, ALPHA, M5, M2, BC), SHAPE5)
    _, h1 = np.linalg.slogdet(DD1.conj().T @ DD1)
    _, h2 = np.linalg.slogdet(DD2.conj().T @ DD2)
    c, d = dwf.coefficients(ALPHA)
    N = lambda m: (c + d) ** LS + m * (d - c) ** LS  # noqa: E731
    rhmc = 0.5 * (h1 - h2)
    eofa_side = -(logML + logMR) + 12 * 16 * np.log(abs(N(M1) / N(M2)))
    assert abs(rhmc - eofa_side) < 1e-9 * abs(rhmc)


def test_action_matches_dense(U):
    ML, MR, _, _ = _eofa_matrices(U, ALPHA, M1, M2)
    phi = inputs.fermion4d(DIMS, 3)
    Pm = dwf.spin_mul(dwf.P_MINUS, phi).reshape(-1)
    Pp = dwf.spin_mul(dwf.P_PLUS, phi).reshape(-1)
    dense_S = (np.vdot(Pm, ML @ Pm) + np.vdot(Pp, MR @ Pp)).real
    S = eofa.action(U, phi, LS, ALPHA, M5, M1, M2, BC, tol=1e-13)
    assert abs(S - dense_S) < 1e-11 * abs(dense_S)
    # M_EOFA -> 1 when m1 = m2 (k = 0)
    assert np.isclose(eofa.action(U, phi, LS, ALPHA, M5, 0.3, 0.3, BC), solve.norm2(phi), rtol=1e-14)


def test_cg_matches_dense_lu(U):
    b = inputs.fermion5d(DIMS, LS, 4)
    D = dense(lambda v: dwf.dwf(U, v, ALPHA, M5, M1, BC), SHAPE5)
    exact = np.linalg.solve(D, b.reshape(-1)).reshape(SHAPE5)
    x, it, res = solve.cgnr(lambda v: dwf.dwf(U, v, ALPHA, M5, M1, BC),
                            lambda v: dwf.dwf_dag(U, v, ALPHA, M5, M1, BC), b, tol=1e-13)
    assert res <= 1e-13
    assert np.linalg.norm(x - exact) < 1e-10 * np.linalg.norm(exact)


def test_system_solve_matches_dense(U):
    rhs = inputs.fermion5d(DIMS, LS, 5)
    for which, a in (("L", 0.0), ("R", -1.0), ("L", -0.3), ("R", -0.7)):
        A = dense(lambda v: eofa.system_apply(U, v, ALPHA, M5, M1, M2, which, a, BC), SHAPE5)
        assert np.abs(A - A.conj().T).max() < 1e-12  # Eq. (8) operators are Hermitian
        exact = np.linalg.solve(A, rhs.reshape(-1)).reshape(SHAPE5)
        x, it, res = eofa.system_solve(U, rhs, ALPHA, M5, M1, M2, which, a, BC, tol=1e-13)
        assert np.linalg.norm(x - exact) < 1e-10 * np.linalg.norm(exact)


def _perturbed(U, site, mu, a, w):
    Up = U.copy()
    T = eofa.generators()[a]
    Up[site + (mu,)] = eofa.exp_i(w * T) @ U[site + (mu,)]
    return Up


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_force_matches_central_differences(U, alpha):
    phi = inputs.fermion4d(DIMS, 6)
    args = (LS, alpha, M5, M1, M2, BC)
    chiL, chiR, _ = eofa.pseudofermion_solutions(U, phi, *args, tol=1e-14)
    k = eofa.k_coefficient(LS, alpha, M1, M2)
    F, imag = eofa.force_from_chi(U, chiL, chiR, k, BC)
    assert imag < 1e-12
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() < 1e-14
    assert np.abs(np.einsum("...ii->...", F)).max() < 1e-14
    Fa = eofa.force_components(F)
    rng = np.random.default_rng(1)
    delta = 1e-5
    for _ in range(4):
        site = tuple(int(v) for v in rng.integers(0, 2, size=4))
        mu, a = int(rng.integers(4)), int(rng.integers(8))
        Sp = eofa.action(_perturbed(U, site, mu, a, +delta), phi, *args, tol=1e-14)
        Sm = eofa.action(_perturbed(U, site, mu, a, -delta), phi, *args, tol=1e-14)
        fd = (Sp - Sm) / (2 * delta)
        assert abs(fd - Fa[site + (mu, a)]) < 1e-6 * max(1.0, abs(fd))


def test_force_gauge_covariant(U):
    phi = inputs.fermion4d(DIMS, 7)
    g = inputs.gauge_transform(DIMS, 7)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(dwf.shift_links(g, mu, 1), -1, -2))
    phig = np.einsum("...ab,...sb->...sa", g, phi)
    args = (LS, ALPHA, M5, M1, M2, BC)
    S0 = eofa.action(U, phi, *args, tol=1e-13)
    S1 = eofa.action(Ug, phig, *args, tol=1e-13)
    assert abs(S0 - S1) < 1e-10 * abs(S0)
    F0 = eofa.force(U, phi, *args, tol=1e-13)
    F1 = eofa.force(Ug, phig, *args, tol=1e-13)
    gd = np.conj(np.swapaxes(g, -1, -2))
    expect = np.einsum("...ab,...mbc,...cd->...mad", g, F0, gd)
    assert np.abs(F1 - expect).max() < 1e-9 * np.abs(F0).max()


def test_exp_i_is_su3():
    P = inputs.momenta(DIMS, 1)
    E = eofa.exp_i(0.3 * P)
    assert np.abs(np.einsum("...ji,...jk->...ik", np.conj(E), E) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(E) - 1).max() < 1e-13
    # small argument: exp(iQ) = 1 + iQ - Q^2/2 + O(Q^3)
    Q = 1e-4 * P
    E = eofa.exp_i(Q)
    approx = np.eye(3) + 1j * Q - 0.5 * np.einsum("...ij,...jk->...ik", Q, Q)
    assert np.abs(E - approx).max() < 1e-11


@pytest.mark.slow
def test_leapfrog_dH_scales_as_dtau_squared_and_reversible(U):
    phi = inputs.fermion4d(DIMS, 8)
    P = inputs.momenta(DIMS, 8)
    args = (LS, ALPHA, M5, M1, M2, BC)
    tau = 0.5
    _, _, dH1 = eofa.leapfrog(U, P, phi, *args, nsteps=2, dtau=tau / 2, tol=1e-13)
    _, _, dH2 = eofa.leapfrog(U, P, phi, *args, nsteps=4, dtau=tau / 4, tol=1e-13)
    ratio = dH1 / dH2
    assert 3.0 < ratio < 5.3, (dH1, dH2)
    U1, P1, _ = eofa.leapfrog(U, P, phi, *args, nsteps=3, dtau=0.1, tol=1e-14)
    U2, P2, dHb = eofa.leapfrog(U1, -P1, phi, *args, nsteps=3, dtau=0.1, tol=1e-14)
    assert np.abs(U2 - U).max() < 1e-10
    assert np.abs(P2 + P).max() < 1e-10


def test_heatbath_eq6_equals_dense_rational_function(U):
    """Eq. (6) with arbitrary positive poles equals f(M_EOFA) eta by eigendecomposition."""
    ML, MR, _, _ = _eofa_matrices(U, ALPHA, M1, M2)
    M = np.zeros((192, 192), dtype=np.complex128)
    idx = np.arange(192).reshape(16, 4, 3)
    sm = idx[:, [2, 3], :].reshape(-1)
    sp = idx[:, [0, 1], :].reshape(-1)
    M[np.ix_(sm, sm)] = ML[np.ix_(sm, sm)]
    M[np.ix_(sp, sp)] = MR[np.ix_(sp, sp)]
    lam, vec = np.linalg.eigh(M)
    assert lam.min() > 0
    eta = inputs.fermion4d(DIMS, 9)
    a0, al, be = 0.3, np.array([0.7, 0.2, 1.3]), np.array([0.05, 0.9, 4.0])
    f = a0 + (al[None, :] / (lam[:, None] + be[None, :])).sum(1)
    exact = (vec @ (f * (vec.conj().T @ eta.reshape(-1)))).reshape(eta.shape)
    phi = oeofa.heatbath(U, eta, LS, ALPHA, M5, M1, M2, BC, a0, al, be, tol=1e-13)
    assert np.linalg.norm(phi - exact) < 1e-10 * np.linalg.norm(exact)


def test_force_parts_match_partial_action_differences(U):
    """Eq. (7) term by term: the chi_L part of the force is the derivative of
    S_L = phi_-^+ M_L phi_-, the chi_R part that of S_R; S_L + S_R = S."""
    phi = inputs.fermion4d(DIMS, 5)
    args = (LS, ALPHA, M5, M1, M2, BC)
    SL, SR = oeofa.partial_actions(U, phi, *args, tol=1e-13)
    assert SL + SR == pytest.approx(oeofa.action(U, phi, *args, tol=1e-13), rel=1e-11)
    T = oeofa.generators()
    rng = np.random.default_rng(4)
    d = 1e-4
    for part, idx in (("L", 0), ("R", 1)):
        Fa = oeofa.force_components(oeofa.force_part(U, phi, *args, part, tol=1e-13))
        for _ in range(2):
            site = tuple(int(rng.integers(n)) for n in U.shape[:4])
            mu, a = int(rng.integers(4)), int(rng.integers(8))
            vals = []
            for w in (d, -d):
                Up = U.copy()
                Up[site + (mu,)] = oeofa.exp_i(w * T[a]) @ U[site + (mu,)]
                vals.append(oeofa.partial_actions(Up, phi, *args, tol=1e-13)[idx])
            fd = (vals[0] - vals[1]) / (2 * d)
            assert abs(fd - Fa[site + (mu, a)]) < 1e-6 * max(1.0, abs(fd)), (part, fd, Fa[site + (mu, a)])
