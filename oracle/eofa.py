"""EOFA action, linear systems, force and MD update (oracle; test infrastructure).

Paper: D. Murphy, Lattice 2016, Sec. 2 (Eq. (5)), Sec. 3.3 (Eq. (7)) and
Sec. 5.1 (Eq. (8)).

Readings (pinned by tests):
  * Delta_pm = R_5 (D^perp_pm(m2) - D^perp_pm(m1)) is taken straight from its
    definition in Sec. 2.  The paper states Delta_pm = k Omega Omega^+ but does
    not print k or Omega; the closed forms used for them are, with
    b = c + d, c5 = c - d, beta = -c5 / b:
        Omega_+[s] = beta^(Ls-1-s) / b,   Omega_-[s] = beta^s / b,
        k = alpha (m2 - m1) / ((1 + m1 beta^Ls) (1 + m2 beta^Ls)).
    Only the product k Omega Omega^T is fixed; a test checks it against the
    dense Delta.
  * phi is a 4D field; (Omega P phi)(x, s) = Omega[s] (P phi)(x) and
    (Omega^+ P psi)(x) = P sum_s Omega[s] psi(x, s).
  * Force convention: U_mu(x) -> exp(i w T^a) U_mu(x) with T^a = lambda^a / 2,
    F^a = dS/dw at w = 0, returned as the traceless Hermitian F = sum_a F^a T^a.
  * MD: P <- P - dtau F, U <- exp(i dtau P) U, kinetic term sum_a p_a^2 / 2 =
    sum tr P^2.
"""
from __future__ import annotations

import numpy as np

from . import dwf
from .solve import cgnr, norm2

_LAMBDA = None


def generators() -> np.ndarray:
    """T^a = lambda^a / 2 (Gell-Mann), shape (8, 3, 3)."""
    global _LAMBDA
    if _LAMBDA is None:
        lam = np.zeros((8, 3, 3), dtype=np.complex128)
        lam[0][0, 1] = lam[0][1, 0] = 1
        lam[1][0, 1], lam[1][1, 0] = -1j, 1j
        lam[2][0, 0], lam[2][1, 1] = 1, -1
        lam[3][0, 2] = lam[3][2, 0] = 1
        lam[4][0, 2], lam[4][2, 0] = -1j, 1j
        lam[5][1, 2] = lam[5][2, 1] = 1
        lam[6][1, 2], lam[6][2, 1] = -1j, 1j
        lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
        _LAMBDA = lam / 2
    return _LAMBDA


# ---------------------------------------------------------------- Sec. 2 pieces

def omega(Ls, alpha):
    """(Omega_+, Omega_-) closed forms (see module docstring)."""
    c, d = dwf.coefficients(alpha)
    b, c5 = c + d, c - d
    beta = -c5 / b
    s = np.arange(Ls)
    return beta ** (Ls - 1 - s) / b, beta ** s / b


def k_coefficient(Ls, alpha, m1, m2):
    c, d = dwf.coefficients(alpha)
    beta = -(c - d) / (c + d)
    return alpha * (m2 - m1) / ((1 + m1 * beta ** Ls) * (1 + m2 * beta ** Ls))


def delta_matrices(Ls, alpha, m1, m2):
    """Delta_pm = R_5 (D^perp_pm(m2) - D^perp_pm(m1)) as Ls x Ls matrices (Sec. 2)."""
    P2p, P2m = dwf.dperp_matrices(Ls, alpha, m2)
    P1p, P1m = dwf.dperp_matrices(Ls, alpha, m1)
    R = np.eye(Ls)[::-1]
    return R @ (P2p - P1p), R @ (P2m - P1m)


def embed(phi, Om, chirality):
    """Omega P_chi phi: 4D -> 5D, (Omega P phi)(x, s) = Omega[s] P phi(x)."""
    P = dwf.P_PLUS if chirality > 0 else dwf.P_MINUS
    return Om[:, None, None, None, None, None, None] * dwf.spin_mul(P, phi)[None]


def contract(psi, Om, chirality):
    """P_chi Omega^+ psi: 5D -> 4D."""
    P = dwf.P_PLUS if chirality > 0 else dwf.P_MINUS
    return dwf.spin_mul(P, np.tensordot(Om, psi, axes=(0, 0)))


# ---------------------------------------------------------------- Eq. (8)

def system_apply(U, psi, alpha, M5, m1, m2, which, a, bc_t):
    """(H(m) + a Delta_chi P_chi) psi, the general EOFA system of Eq. (8).

    which = 'L': m = m1 and the Delta_- P_- term; which = 'R': m = m2 and the
    Delta_+ P_+ term.  The action's chi_L uses ('L', a = 0) and chi_R uses
    ('R', a = -1), as in Eq. (5).
    """
    Ls = psi.shape[0]
    m = m1 if which == "L" else m2
    out = dwf.hermitian_H(U, psi, alpha, M5, m, bc_t)
    if a != 0.0:
        Dp, Dm = delta_matrices(Ls, alpha, m1, m2)
        if which == "L":
            out = out + a * dwf.apply_s(np.zeros((Ls, Ls)), Dm, psi)
        else:
            out = out + a * dwf.apply_s(Dp, np.zeros((Ls, Ls)), psi)
    return out


def system_apply_at(U, psi, alpha, M5, m1, m2, which, a, bc_t, site):
    """(H(m) + a Delta_chi P_chi) psi at one 4D site for every s, shape (Ls, 4, 3).

    The same definition as system_apply: H = gamma_5 R_5 (D_w + D^perp) with
    D_w evaluated from the site's eight neighbours (dwf.wilson_at) and the
    5D-local D^perp and Delta terms, which act on the s index of the site
    alone; for checking solutions on lattices too large for whole-field numpy.
    """
    Ls = psi.shape[0]
    m = m1 if which == "L" else m2
    slab = dwf._site_slab(psi, site)
    Pp, Pm = dwf.dperp_matrices(Ls, alpha, m)
    deo = dwf.wilson_at(U, psi, M5, site, bc_t) + dwf.apply_s(Pp, Pm, slab)[:, 0, 0, 0, 0]
    out = dwf.gamma5(dwf.R5(deo))
    if a != 0.0:
        Dp, Dm = delta_matrices(Ls, alpha, m1, m2)
        zero = np.zeros((Ls, Ls))
        term = dwf.apply_s(zero, Dm, slab) if which == "L" else dwf.apply_s(Dp, zero, slab)
        out = out + a * term[:, 0, 0, 0, 0]
    return out


def system_solve(U, rhs, alpha, M5, m1, m2, which, a, bc_t, tol=1e-12, maxiter=20000):
    """Solve (H(m) + a Delta P) psi = rhs (Hermitian system) by CGNR."""
    A = lambda v: system_apply(U, v, alpha, M5, m1, m2, which, a, bc_t)  # noqa: E731
    return cgnr(A, A, rhs, tol=tol, maxiter=maxiter)


# ---------------------------------------------------------------- Eq. (5)

def pseudofermion_solutions(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol=1e-12):
    """chi_L = H(m1)^{-1} Omega_- P_- phi, chi_R = [H(m2) - Delta_+ P_+]^{-1} Omega_+ P_+ phi."""
    Op, Om = omega(Ls, alpha)
    chiL, itL, resL = system_solve(U, embed(phi, Om, -1), alpha, M5, m1, m2, "L", 0.0, bc_t, tol)
    chiR, itR, resR = system_solve(U, embed(phi, Op, +1), alpha, M5, m1, m2, "R", -1.0, bc_t, tol)
    return chiL, chiR, (itL, resL, itR, resR)


def action(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol=1e-12, chis=None):
    """S_f = phi^+ M_EOFA phi with M_EOFA of Eq. (5)."""
    Op, Om = omega(Ls, alpha)
    k = k_coefficient(Ls, alpha, m1, m2)
    if chis is None:
        chiL, chiR, _ = pseudofermion_solutions(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    else:
        chiL, chiR = chis
    S = norm2(phi)
    S -= k * complex(np.vdot(embed(phi, Om, -1), chiL)).real
    S += k * complex(np.vdot(embed(phi, Op, +1), chiR)).real
    return S


def partial_actions(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol=1e-12):
    """(S_L, S_R), the two terms of Eq. (5): S_L = phi_-^+ M_L phi_- (P_- part,
    through chi_L) and S_R = phi_+^+ M_R phi_+ (P_+ part, through chi_R)."""
    Op, Om = omega(Ls, alpha)
    k = k_coefficient(Ls, alpha, m1, m2)
    chiL, chiR, _ = pseudofermion_solutions(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    pm, pp = dwf.spin_mul(dwf.P_MINUS, phi), dwf.spin_mul(dwf.P_PLUS, phi)
    SL = norm2(pm) - k * complex(np.vdot(embed(phi, Om, -1), chiL)).real
    SR = norm2(pp) + k * complex(np.vdot(embed(phi, Op, +1), chiR)).real
    return SL, SR


# ---------------------------------------------------------------- Eq. (7)

def force_from_chi(U, chiL, chiR, k, bc_t):
    """F_mu(x) = sum_a F^a T^a with F^a of Eq. (7):
    F^a = k chi_L^+ g5 R5 (d^a D_w) chi_L - k chi_R^+ g5 R5 (d^a D_w) chi_R.

    d^a D_w is the derivative of D_w under U_mu(x) -> exp(i w T^a) U_mu(x);
    it touches the forward hop at x and the backward hop at x + mu.  Returns
    (F, imag) where imag is the largest imaginary part met (zero in exact
    arithmetic).
    """
    T = generators()
    one = np.eye(4)
    F = np.zeros(U.shape, dtype=np.complex128)
    worst_imag = 0.0
    for chi, sign in ((chiL, +1.0), (chiR, -1.0)):
        zeta = dwf.gamma5(dwf.R5(chi))  # (g5 R5 chi); chi^+ g5 R5 X = zeta^+ X
        for mu in range(4):
            Um = U[..., mu, :, :]
            chi_f = dwf.shift(chi, mu, +1, bc_t)
            zeta_f = dwf.shift(zeta, mu, +1, bc_t)
            for a in range(8):
                dU = 1j * T[a] @ Um                       # d/dw of U_mu(x)
                dUd = dwf.dagger3(dU)                     # d/dw of U_mu(x)^+
                t1 = dwf.spin_mul(one - dwf.GAMMA[mu], dwf.colour_mul(dU, chi_f))
                t2 = dwf.spin_mul(one + dwf.GAMMA[mu], dwf.colour_mul(dUd, chi))
                val = -0.5 * (np.einsum("s...,s...->...", np.conj(zeta), t1).sum(axis=(-2, -1))
                              + np.einsum("s...,s...->...", np.conj(zeta_f), t2).sum(axis=(-2, -1)))
                # val has shape (T, Z, Y, X) after summing s, spin, colour
                worst_imag = max(worst_imag, float(np.max(np.abs(val.imag))))
                F[..., mu, :, :] += sign * k * val.real[..., None, None] * T[a]
    return F, worst_imag


def force(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol=1e-12):
    chiL, chiR, _ = pseudofermion_solutions(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    k = k_coefficient(Ls, alpha, m1, m2)
    return force_from_chi(U, chiL, chiR, k, bc_t)[0]


def force_part(U, phi, Ls, alpha, M5, m1, m2, bc_t, part, tol=1e-12):
    """The force of S_L (part 'L', one solve for chi_L) or of S_R (part 'R',
    one solve for chi_R): the two terms of Eq. (7) separately."""
    Op, Om = omega(Ls, alpha)
    k = k_coefficient(Ls, alpha, m1, m2)
    if part == "L":
        chi, _, _ = system_solve(U, embed(phi, Om, -1), alpha, M5, m1, m2, "L", 0.0, bc_t, tol)
        return force_from_chi(U, chi, np.zeros_like(chi), k, bc_t)[0]
    chi, _, _ = system_solve(U, embed(phi, Op, +1), alpha, M5, m1, m2, "R", -1.0, bc_t, tol)
    return force_from_chi(U, np.zeros_like(chi), chi, k, bc_t)[0]


def force_components(F):
    """F^a = 2 tr(T^a F) for a traceless Hermitian F = sum_a F^a T^a."""
    return 2.0 * np.einsum("aij,...ji->...a", generators(), F).real


# ---------------------------------------------------------------- molecular dynamics

def exp_i(Q):
    """exp(i Q) for Hermitian 3x3 Q, by eigendecomposition."""
    w, v = np.linalg.eigh(Q)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def kinetic(P):
    """sum_links sum_a p_a^2 / 2 = sum tr(P^2) for P = sum_a p_a T^a."""
    return float(np.einsum("...ij,...ji->...", P, P).real.sum())


def leapfrog(U, P, phi, Ls, alpha, M5, m1, m2, bc_t, nsteps, dtau, tol=1e-12):
    """Leapfrog MD for H = sum tr P^2 + S_EOFA; returns (U', P', dH)."""
    H0 = kinetic(P) + action(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    U = U.copy()
    P = P - 0.5 * dtau * force(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    for step in range(nsteps):
        U = np.einsum("...ij,...jk->...ik", exp_i(dtau * P), U)
        f = force(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
        P = P - (dtau if step < nsteps - 1 else 0.5 * dtau) * f
    H1 = kinetic(P) + action(U, phi, Ls, alpha, M5, m1, m2, bc_t, tol)
    return U, P, H1 - H0


def force_at_link(U, chiL, chiR, k, bc_t, site, mu):
    """F_mu(x) of Eq. (7) at one link (t, z, y, x) = site, from its definition.

    Only chi at x and x + mu enter.  Plain loops over a = 1..8 and s; used to
    check the force at sampled links of lattices too large for force_from_chi.
    """
    T = generators()
    one = np.eye(4)
    dims = U.shape[:4]
    axis = {0: 3, 1: 2, 2: 1, 3: 0}[mu]  # position of mu in (t, z, y, x)
    fwd = list(site)
    fwd[axis] += 1
    phase = 1.0
    if fwd[axis] == dims[axis]:
        fwd[axis] = 0
        if mu == 3:
            phase = bc_t
    fwd = tuple(fwd)
    Ls = chiL.shape[0]
    Um = U[site + (mu,)]
    F = np.zeros((3, 3), dtype=np.complex128)
    for chi, sign in ((chiL, +1.0), (chiR, -1.0)):
        for a in range(8):
            dU = 1j * T[a] @ Um
            val = 0.0j
            for s in range(Ls):
                zeta_x = dwf.GAMMA5 @ chi[Ls - 1 - s][site]          # (g5 R5 chi)(x, s)
                zeta_f = dwf.GAMMA5 @ chi[Ls - 1 - s][fwd] * phase   # (g5 R5 chi)(x + mu, s), boundary phase
                chi_f = chi[s][fwd] * phase
                t1 = (one - dwf.GAMMA[mu]) @ (chi_f @ dU.T)           # (1 - g) dU chi(x + mu)
                t2 = (one + dwf.GAMMA[mu]) @ (chi[s][site] @ np.conj(dU))  # (1 + g) dU^+ chi(x)
                val += -0.5 * (np.vdot(zeta_x, t1) + np.vdot(zeta_f, t2))
            F += sign * k * val.real * T[a]
    return F


# ---------------------------------------------------------------- heatbath (Sec. 3.2)

def heatbath(U, eta, Ls, alpha, M5, m1, m2, bc_t, alpha0, alphas, betas, tol=1e-12):
    """phi = f(M_EOFA) eta for f(x) = alpha0 + sum_l alphas[l] / (x + betas[l]), Eq. (6).

    With gamma_l = 1 / (1 + beta_l), each pole needs one solve of Eq. (8) for
    the P_- part (H(m1) - gamma_l Delta_- P_-) and one for the P_+ part
    (H(m2) - gamma_l beta_l Delta_+ P_+).
    """
    Op, Om = omega(Ls, alpha)
    k = k_coefficient(Ls, alpha, m1, m2)
    bL, bR = embed(eta, Om, -1), embed(eta, Op, +1)
    phi = alpha0 * eta
    for al, be in zip(alphas, betas):
        g = 1.0 / (1.0 + be)
        psiL, _, _ = system_solve(U, bL, alpha, M5, m1, m2, "L", -g, bc_t, tol)
        psiR, _, _ = system_solve(U, bR, alpha, M5, m1, m2, "R", -g * be, bc_t, tol)
        phi = phi + al * g * (eta + k * g * contract(psiL, Om, -1) - k * g * contract(psiR, Op, +1))
    return phi
