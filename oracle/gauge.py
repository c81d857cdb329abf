"""Gauge action, gauge force and the force-gradient HMC integrators (oracle;
test infrastructure: imported by tests/ and bench.py's CPU baseline only).

Sec. 5 of the paper runs its ensemble with a nested force-gradient QPQPQ
integrator and the fermion (strange quark, EOFA) force on the outermost time
scale, on top of a gauge action.  Readings (pinned by tests):

  * Gauge action: Wilson plaquette action
        S_g = (beta / 3) sum_{x, mu < nu} Re tr (1 - U_mu,nu(x)),
        U_mu,nu(x) = U_mu(x) U_nu(x + mu) U_mu(x + nu)^+ U_nu(x)^+,
    periodic links (the fermion t-phase is not part of the gauge field).
    The paper's Iwasaki / DSDR gauge actions are not reproduced.
  * Force convention as for the fermion force: U_mu(x) -> exp(i w T^a) U_mu(x),
    F^a = dS/dw, F = sum_a F^a T^a.  With A_mu(x) the sum of the six staples
    (Re tr U_mu(x) A_mu(x) is the sum of the plaquettes holding U_mu(x)),
    F^a = (beta / 3) Im tr (T^a U_mu(x) A_mu(x)).
  * Integrators for H = sum tr P^2 + S (U <- exp(i h P) U, P <- P - h F).
    The paper names the integrator without coefficients; the fourth-order
    force-gradient forms are
      PQPQP:  P(h/6) Q(h/2) P~(2h/3) Q(h/2) P(h/6),
      QPQPQ:  Q(lam h) P~(h/2) Q((1 - 2 lam) h) P~(h/2) Q(lam h), lam = 1/2 - sqrt(3)/6,
    where P~(c) kicks with the force taken at the displaced field
    U' = exp(-i z F(U)) U, z = h^2 / 24 (PQPQP) or (2 - sqrt 3) h^2 / 12
    (QPQPQ): to first order in z this adds the force-gradient term that
    cancels the [S, [T, S]] error of the splitting, while lam cancels
    [T, [T, S]].  Nesting: each Q(t) of the outer (fermion) level is n_inner
    steps of the same integrator for the gauge action with step t / n_inner;
    the outer displacement uses the outer force only (the two forces
    commute).  Pinned by dH ~ h^4.
"""
from __future__ import annotations

import numpy as np

from . import dwf
from . import eofa as oeofa

LAMBDA_QPQPQ = 0.5 - np.sqrt(3.0) / 6.0
Z_QPQPQ = (2.0 - np.sqrt(3.0)) / 12.0
Z_PQPQP = 1.0 / 24.0


def _mm(a, b):
    return np.einsum("...ij,...jk->...ik", a, b)


def plaquette(U, mu, nu):
    """U_mu,nu(x) for every site, shape (T,Z,Y,X,3,3)."""
    Umu, Unu = U[..., mu, :, :], U[..., nu, :, :]
    return _mm(_mm(Umu, dwf.shift_links(Unu, mu, +1)),
               _mm(dwf.dagger3(dwf.shift_links(Umu, nu, +1)), dwf.dagger3(Unu)))


def action(U, beta):
    """Wilson plaquette action (beta / 3) sum_{x, mu < nu} Re tr (1 - U_mu,nu)."""
    S = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            S += (3.0 - np.einsum("...ii->...", plaquette(U, mu, nu)).real).sum()
    return beta / 3.0 * S


def staples(U, mu):
    """A_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
                                + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)]."""
    Umu = U[..., mu, :, :]
    A = np.zeros_like(Umu)
    for nu in range(4):
        if nu == mu:
            continue
        Unu = U[..., nu, :, :]
        A += _mm(_mm(dwf.shift_links(Unu, mu, +1), dwf.dagger3(dwf.shift_links(Umu, nu, +1))), dwf.dagger3(Unu))
        Unu_m = dwf.shift_links(Unu, nu, -1)  # U_nu(x - nu)
        Unu_pm = dwf.shift_links(Unu_m, mu, +1)  # U_nu(x + mu - nu)
        A += _mm(_mm(dwf.dagger3(Unu_pm), dwf.dagger3(dwf.shift_links(Umu, nu, -1))), Unu_m)
    return A


def force(U, beta):
    """Gauge force F = sum_a T^a (beta / 3) Im tr (T^a U_mu A_mu), shape (T,Z,Y,X,4,3,3)."""
    T = oeofa.generators()
    F = np.zeros_like(U)
    for mu in range(4):
        X = _mm(U[..., mu, :, :], staples(U, mu))
        Fa = beta / 3.0 * np.einsum("aij,...ji->...a", T, X).imag
        F[..., mu, :, :] = np.einsum("...a,aij->...ij", Fa, T)
    return F


def link_update(U, Q):
    """U <- exp(i Q) U for Hermitian Q on every link."""
    return _mm(oeofa.exp_i(Q), U)


class Forces:
    """The two time scales: the fermion (EOFA) force and the gauge force.

    ``fermion`` is None for a pure-gauge system (then the gauge force sits on
    the outer level).  Counters record the force evaluations for comparison
    with the device integrator.
    """

    def __init__(self, beta, fermion=None):
        self.beta = beta
        self.fermion = fermion  # dict(phi, Ls, alpha, M5, m1, m2, bc_t, tol) or None
        self.n_fermion = 0

    def outer(self, U):
        if self.fermion is None:
            return force(U, self.beta)
        self.n_fermion += 1
        f = self.fermion
        return oeofa.force(U, f["phi"], f["Ls"], f["alpha"], f["M5"], f["m1"], f["m2"], f["bc_t"], f["tol"])

    def inner(self, U):
        return force(U, self.beta)

    def energy(self, U, P):
        S = action(U, self.beta) if self.beta != 0 else 0.0
        if self.fermion is not None:
            f = self.fermion
            S += oeofa.action(U, f["phi"], f["Ls"], f["alpha"], f["M5"], f["m1"], f["m2"], f["bc_t"], f["tol"])
        return oeofa.kinetic(P) + S


def _kick(U, P, c, z, force_fn):
    """P <- P - c F(U'), U' = exp(-i z F(U)) U (z = 0: plain kick)."""
    if z == 0.0:
        return P - c * force_fn(U)
    return P - c * force_fn(link_update(U, -z * force_fn(U)))


def _level_steps(U, P, t, levels, scheme):
    """levels[0] = (force, n): n steps of length t / n of the scheme with that
    force; each drift is the next level's integration (a link update at the
    innermost level)."""
    force_fn, n = levels[0]
    rest = levels[1:]

    def drift(U_, P_, dt):
        if rest:
            return _level_steps(U_, P_, dt, rest, scheme)
        return link_update(U_, dt * P_), P_

    h = t / n
    for _ in range(n):
        if scheme == "pqpqp":
            P = _kick(U, P, h / 6, 0.0, force_fn)
            U, P = drift(U, P, h / 2)
            P = _kick(U, P, 2 * h / 3, Z_PQPQP * h * h, force_fn)
            U, P = drift(U, P, h / 2)
            P = _kick(U, P, h / 6, 0.0, force_fn)
        elif scheme == "qpqpq":
            lam = LAMBDA_QPQPQ
            U, P = drift(U, P, lam * h)
            P = _kick(U, P, h / 2, Z_QPQPQ * h * h, force_fn)
            U, P = drift(U, P, (1 - 2 * lam) * h)
            P = _kick(U, P, h / 2, Z_QPQPQ * h * h, force_fn)
            U, P = drift(U, P, lam * h)
        elif scheme == "leapfrog":
            P = _kick(U, P, h / 2, 0.0, force_fn)
            U, P = drift(U, P, h)
            P = _kick(U, P, h / 2, 0.0, force_fn)
        else:
            raise ValueError(scheme)
    return U, P


def trajectory_levels(U, P, levels, energy, tau, scheme="qpqpq"):
    """Multi-time-scale trajectory: levels = [(force_fn, n), ...], outermost
    first (n = outer steps, then steps per drift of the level above);
    energy(U, P) = H.  Returns (U', P', dH)."""
    H0 = energy(U, P)
    U1, P1 = _level_steps(U, P, tau, levels, scheme)
    return U1, P1, energy(U1, P1) - H0


def trajectory(U, P, forces, tau, nsteps, scheme="qpqpq", n_inner=0):
    """Integrate H = sum tr P^2 + S_g + S_EOFA over time tau; returns (U', P', dH).

    n_inner = 0 puts both forces on one level; n_inner > 0 nests the gauge
    force: every drift of the outer (fermion) level is n_inner steps of the
    same scheme for the gauge action alone.
    """
    if n_inner == 0:
        def both(U_):
            return forces.outer(U_) + (forces.inner(U_) if forces.fermion is not None else 0.0)
        levels = [(both, nsteps)]
    else:
        levels = [(forces.outer, nsteps), (forces.inner, n_inner)]
    return trajectory_levels(U, P, levels, forces.energy, tau, scheme)


def split_lr_trajectory(U, P, beta, fermion, tau, nsteps, n_middle, n_inner, scheme="qpqpq", outer="R"):
    """Asymmetric EOFA integration (Sexton-Weingarten over the two terms of
    Eq. (5)): one term's force (outer = 'R': S_R, 'L': S_L) on the outer
    level, the other in the middle, the gauge force innermost (omitted when
    beta = 0)."""
    f = fermion
    args = (f["phi"], f["Ls"], f["alpha"], f["M5"], f["m1"], f["m2"], f["bc_t"])
    inner_part = "L" if outer == "R" else "R"
    levels = [(lambda U_: oeofa.force_part(U_, *args, outer, f["tol"]), nsteps),
              (lambda U_: oeofa.force_part(U_, *args, inner_part, f["tol"]), n_middle)]
    if beta != 0.0:
        levels.append((lambda U_: force(U_, beta), n_inner))
    forces = Forces(beta, fermion)
    return trajectory_levels(U, P, levels, forces.energy, tau, scheme)


# ---------------------------------------------------------------- HMC chain (Sec. 3, Sec. 5)

def metropolis(dH, u):
    """The HMC accept test: accept with probability min(1, exp(-dH)), decided
    by a uniform u in [0, 1): accept when u < exp(-dH).  A NaN dH is rejected."""
    return bool(np.isfinite(dH) and u < np.exp(-dH))


def hmc_chain(U, Ps, us, beta, tau, nsteps, scheme="qpqpq", n_inner=0, fermion=None, etas=None, rational=None):
    """HMC Markov chain of len(us) trajectories.

    Trajectory k: when ``fermion`` is given (dict(Ls, alpha, M5, m1, m2, bc_t,
    tol)), a fresh pseudofermion phi = f(M_EOFA) eta_k (eta_k with density
    exp(-eta^+ eta): real and imaginary parts N(0, 1/2)) from the heatbath of
    Eq. (6) with f(x) = alpha0 + sum_l alphas[l] / (x + betas[l]) (rational =
    (alpha0, alphas, betas)); the MD trajectory of H = sum tr P^2 + S_g +
    S_EOFA(phi) from momenta Ps[k] (``trajectory``); the Metropolis step with
    us[k].  A rejected trajectory keeps the links it started from.  Returns
    (U, records) with records[k] = (dH, accepted, S_EOFA(phi) at the start).
    """
    recs = []
    for k, (P, u) in enumerate(zip(Ps, us)):
        f = None
        S_start = 0.0
        if fermion is not None:
            a0, al, be = rational
            fp = fermion
            phi = oeofa.heatbath(U, etas[k], fp["Ls"], fp["alpha"], fp["M5"], fp["m1"], fp["m2"], fp["bc_t"], a0,
                                 al, be, fp["tol"])
            f = dict(fermion, phi=phi)
            S_start = oeofa.action(U, phi, fp["Ls"], fp["alpha"], fp["M5"], fp["m1"], fp["m2"], fp["bc_t"], fp["tol"])
        forces = Forces(beta, f)
        U1, _, dH = trajectory(U, P, forces, tau, nsteps, scheme, n_inner)
        acc = metropolis(dH, u)
        if acc:
            U = U1
        recs.append((dH, acc, S_start))
    return U, recs
