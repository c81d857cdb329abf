"""Pins of the oracle's gauge action, gauge force and force-gradient integrators.

Closed forms (cold links, one rotated link), finite differences of the
action, gauge covariance, and the orders of the integrators (dH ~ h^4 for
the force-gradient forms, h^2 for leapfrog), none of which reuse the
formula under test.
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from oracle import gauge
from paper_1611_00298_gb300 import inputs

DIMS = (2, 2, 2, 2)
BETA = 5.7


def _cold(dims):
    X, Y, Z, T = dims
    U = np.zeros((T, Z, Y, X, 4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def test_cold_links_have_zero_action_and_force():
    U = _cold(DIMS)
    assert gauge.action(U, BETA) == pytest.approx(0.0, abs=1e-12)
    assert np.abs(gauge.force(U, BETA)).max() < 1e-13


@pytest.mark.parametrize("theta", [0.3, 1.1, 2.5])
def test_single_rotated_link_closed_form(theta):
    """One link exp(i theta lambda_3) on cold links: it sits in 6 plaquettes, each
    contributing Re tr (1 - U) = 2 - 2 cos theta, so S = 4 beta (1 - cos theta);
    rotating it by exp(i w T^3) shifts theta by w / 2, so F^3 = 2 beta sin theta."""
    U = _cold((4, 4, 4, 4))
    site, mu = (1, 2, 0, 3), 2
    U[site + (mu,)] = np.diag(np.exp(1j * theta * np.array([1.0, -1.0, 0.0])))
    assert gauge.action(U, BETA) == pytest.approx(4 * BETA * (1 - np.cos(theta)), rel=1e-12)
    Fa = oeofa.force_components(gauge.force(U, BETA)[site + (mu,)])
    expect = np.zeros(8)
    expect[2] = 2 * BETA * np.sin(theta)
    assert np.abs(Fa - expect).max() < 1e-12 * BETA


def test_force_matches_central_differences():
    U = inputs.gauge_field((4, 2, 2, 2), 0.6, 3)
    F = gauge.force(U, BETA)
    Fa = oeofa.force_components(F)
    T = oeofa.generators()
    rng = np.random.default_rng(2)
    d = 1e-3
    for _ in range(12):
        site = tuple(int(rng.integers(n)) for n in U.shape[:4])
        mu, a = int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for w in (2 * d, d, -d, -2 * d):
            Up = U.copy()
            Up[site + (mu,)] = oeofa.exp_i(w * T[a]) @ U[site + (mu,)]
            vals.append(gauge.action(Up, BETA))
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * d)  # error O(d^4)
        assert abs(fd - Fa[site + (mu, a)]) < 1e-9 * max(1.0, abs(fd))
    # traceless Hermitian
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() < 1e-13
    assert np.abs(np.einsum("...ii->...", F)).max() < 1e-13


def test_gauge_invariance_and_covariance():
    U = inputs.gauge_field(DIMS, 0.7, 4)
    g = inputs.gauge_field(DIMS, 1.0, 9)[..., 0, :, :]
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = np.roll(g, -1, axis=3 - mu)  # g(x + mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(gp, -1, -2))
    assert gauge.action(Ug, BETA) == pytest.approx(gauge.action(U, BETA), rel=1e-12)
    F, Fg = gauge.force(U, BETA), gauge.force(Ug, BETA)
    gd = np.conj(np.swapaxes(g, -1, -2))
    for mu in range(4):
        assert np.abs(Fg[..., mu, :, :] - g @ F[..., mu, :, :] @ gd).max() < 1e-12 * BETA


def _dH(scheme, nsteps, forces, U, P, tau=0.5, n_inner=0):
    return gauge.trajectory(U, P, forces, tau, nsteps, scheme, n_inner)[2]


@pytest.mark.parametrize("scheme,order", [("leapfrog", 2), ("pqpqp", 4), ("qpqpq", 4)])
def test_integrator_order(scheme, order):
    """dH(h) / dH(h / 2) -> 2^order."""
    U = inputs.gauge_field(DIMS, 0.4, 5)
    P = inputs.momenta(DIMS, 6)
    f = gauge.Forces(BETA)
    d1, d2 = _dH(scheme, 4, f, U, P), _dH(scheme, 8, f, U, P)
    assert abs(d1 / d2) == pytest.approx(2 ** order, rel=0.15), (d1, d2)


class _TwoScales(gauge.Forces):
    """H = T + S_g(beta_out) + S_g(beta_in) split over the two levels."""

    def __init__(self, beta_out, beta_in):
        super().__init__(beta_in)
        self.beta_out = beta_out

    def outer(self, U):
        return gauge.force(U, self.beta_out)

    def energy(self, U, P):
        return oeofa.kinetic(P) + gauge.action(U, self.beta) + gauge.action(U, self.beta_out)


def test_nested_integrator_order_and_reversibility():
    U = inputs.gauge_field(DIMS, 0.4, 7)
    P = inputs.momenta(DIMS, 8)
    f = _TwoScales(1.5, BETA)
    d1 = _dH("qpqpq", 3, f, U, P, n_inner=2)
    d2 = _dH("qpqpq", 6, f, U, P, n_inner=2)
    assert abs(d1 / d2) == pytest.approx(16, rel=0.2), (d1, d2)
    U1, P1, _ = gauge.trajectory(U, P, f, 0.5, 3, "qpqpq", 2)
    U2, P2, dH2 = gauge.trajectory(U1, -P1, f, 0.5, 3, "qpqpq", 2)
    assert np.abs(U2 - U).max() < 1e-11
    assert np.abs(P2 + P).max() < 1e-11


# ---------------------------------------------------------------- HMC chain (Sec. 3, Sec. 5)

def test_metropolis_accept_rule():
    """Accept with probability min(1, exp(-dH)): u < exp(-dH)."""
    assert gauge.metropolis(-0.5, 0.999999)          # dH <= 0 always accepted
    assert gauge.metropolis(0.0, 0.999999)
    assert gauge.metropolis(0.7, 0.49)               # exp(-0.7) = 0.4966
    assert not gauge.metropolis(0.7, 0.50)
    assert not gauge.metropolis(3.0, 0.05)           # exp(-3) = 0.0498
    assert gauge.metropolis(3.0, 0.049)
    assert not gauge.metropolis(float("nan"), 0.0)
    assert not gauge.metropolis(float("inf"), 0.0)


def _pure_gauge_chain(n, warm, nsteps=8, scheme="leapfrog", seed=200):
    dims = (2, 2, 2, 2)
    U = inputs.gauge_field(dims, 0.3, 1)
    Ps = [inputs.momenta(dims, seed, stream=10 + k) for k in range(n + warm)]
    us = inputs.uniform(inputs.stream_key(seed, 9), n + warm)
    U1, recs = gauge.hmc_chain(U, Ps, us, BETA, 1.0, nsteps, scheme)
    return U, Ps, us, U1, recs


def test_hmc_chain_keeps_the_links_of_a_rejected_trajectory():
    """Step by step: an accepted trajectory moves the links to the trajectory's
    end point, a rejected one leaves them bit for bit; the decision is the
    Metropolis rule on that trajectory's dH."""
    U, Ps, us, _, _ = _pure_gauge_chain(0, 12, nsteps=2)  # coarse steps: some rejections
    f = gauge.Forces(BETA)
    rejected = 0
    for k in range(12):
        Un, recs = gauge.hmc_chain(U, [Ps[k]], [us[k]], BETA, 1.0, 2, "leapfrog")
        U1, _, dH = gauge.trajectory(U, Ps[k], f, 1.0, 2, "leapfrog")
        assert recs[0][0] == dH
        assert recs[0][1] == (us[k] < np.exp(-dH))
        if recs[0][1]:
            assert np.array_equal(Un, U1)
        else:
            assert np.array_equal(Un, U)
            rejected += 1
        U = Un
    assert 0 < rejected < 12


def test_hmc_chain_creutz_equality_pure_gauge():
    """In equilibrium <exp(-dH)> = 1 (area preservation and reversibility of
    the integrator) and <dH> > 0; 300 trajectories after 60 of warm-up on 2^4
    at beta = 5.7 (8 leapfrog steps, acceptance about 0.9)."""
    _, _, _, _, recs = _pure_gauge_chain(300, 60)
    dH = np.array([r[0] for r in recs])[60:]
    e = np.exp(-dH)
    err = e.std() / np.sqrt(len(e))
    assert abs(e.mean() - 1.0) < 4 * err, (e.mean(), err)
    assert dH.mean() > 0, dH.mean()
