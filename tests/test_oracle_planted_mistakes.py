"""The oracle's pins are sharp: a plausible mistake planted in the oracle (on
the CPU, through monkeypatch) makes the pin that guards it fail.

Each case reruns the check of a pin test against a deliberately wrong
variant of one oracle function: a flipped sign, a dropped term, a transposed
operand, a wrong coefficient.  If a pin passed with the mistake in place it
would not be pinning that part of the oracle.
"""
import numpy as np
import pytest

from oracle import dwf
from oracle import eofa as oeofa
from oracle import gauge
from paper_1611_00298_gb300 import inputs

BETA = 5.7


def _gauge_fd_error(force_fn):
    """Largest |FD - F^a| over a few links for the Wilson gauge action (4-point stencil)."""
    U = inputs.gauge_field((4, 2, 2, 2), 0.6, 3)
    Fa = oeofa.force_components(force_fn(U, BETA))
    T = oeofa.generators()
    rng = np.random.default_rng(2)
    d, worst = 1e-3, 0.0
    for _ in range(6):
        site = tuple(int(rng.integers(n)) for n in U.shape[:4])
        mu, a = int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for w in (2 * d, d, -d, -2 * d):
            Up = U.copy()
            Up[site + (mu,)] = oeofa.exp_i(w * T[a]) @ U[site + (mu,)]
            vals.append(gauge.action(Up, BETA))
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * d)
        worst = max(worst, abs(fd - Fa[site + (mu, a)]))
    return worst


def test_gauge_force_pin_catches_transposed_staples():
    assert _gauge_fd_error(gauge.force) < 1e-8

    def transposed(U, beta):  # A^T instead of A in X = U A
        T = oeofa.generators()
        F = np.zeros_like(U)
        for mu in range(4):
            X = U[..., mu, :, :] @ np.swapaxes(gauge.staples(U, mu), -1, -2)
            Fa = beta / 3.0 * np.einsum("aij,...ji->...a", T, X).imag
            F[..., mu, :, :] = np.einsum("...a,aij->...ij", Fa, T)
        return F

    assert _gauge_fd_error(transposed) > 1e-3


def test_gauge_force_pin_catches_dropped_backward_staple(monkeypatch):
    def forward_only(U, mu):
        Umu = U[..., mu, :, :]
        A = np.zeros_like(Umu)
        for nu in range(4):
            if nu != mu:
                Unu = U[..., nu, :, :]
                A += (dwf.shift_links(Unu, mu, +1) @ dwf.dagger3(dwf.shift_links(Umu, nu, +1))) @ dwf.dagger3(Unu)
        return A

    monkeypatch.setattr(gauge, "staples", forward_only)
    assert _gauge_fd_error(gauge.force) > 1e-3


def _order_pin_holds(ratio, order=4):
    """The condition test_oracle_gauge.test_integrator_order asserts."""
    return abs(ratio - 2 ** order) <= 0.15 * 2 ** order


def _order_ratio(scheme):
    U = inputs.gauge_field((2, 2, 2, 2), 0.4, 5)
    P = inputs.momenta((2, 2, 2, 2), 6)
    f = gauge.Forces(BETA)
    d1 = gauge.trajectory(U, P, f, 0.5, 4, scheme)[2]
    d2 = gauge.trajectory(U, P, f, 0.5, 8, scheme)[2]
    return abs(d1 / d2)


def test_integrator_order_pin_catches_wrong_sign_of_the_force_gradient_shift(monkeypatch):
    assert _order_pin_holds(_order_ratio("qpqpq"))
    monkeypatch.setattr(gauge, "Z_QPQPQ", -gauge.Z_QPQPQ)  # displace uphill instead of downhill
    assert not _order_pin_holds(_order_ratio("qpqpq"))


def test_integrator_order_pin_catches_wrong_lambda(monkeypatch):
    monkeypatch.setattr(gauge, "LAMBDA_QPQPQ", 1.0 / 6.0)  # the PQPQP value in the QPQPQ slot
    assert not _order_pin_holds(_order_ratio("qpqpq"))


def test_closed_form_pin_catches_lambda_instead_of_half_lambda_generators(monkeypatch):
    """With T^a = lambda^a instead of lambda^a / 2 the rotated-link force doubles."""
    theta, site, mu = 1.1, (1, 2, 0, 3), 2
    U = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    U[site + (mu,)] = np.diag(np.exp(1j * theta * np.array([1.0, -1.0, 0.0])))
    good = oeofa.force_components(gauge.force(U, BETA)[site + (mu,)])[2]
    assert good == pytest.approx(2 * BETA * np.sin(theta), rel=1e-12)
    T2 = 2 * oeofa.generators()
    monkeypatch.setattr(oeofa, "generators", lambda: T2)
    bad = gauge.force(U, BETA)[site + (mu,)]
    Fa = 2.0 * np.einsum("aij,...ji->...a", T2 / 2, bad).real  # read back in the true normalisation
    assert abs(Fa[2] - 2 * BETA * np.sin(theta)) > 0.5 * BETA * np.sin(theta)


def test_heatbath_pin_catches_a_wrong_shift(monkeypatch):
    """Eq. (6) with the P_- system shifted by gamma_l beta_l instead of gamma_l
    no longer equals the dense rational function of M_EOFA."""
    import test_oracle_eofa as t
    U = inputs.gauge_field(t.DIMS, 0.8, 1)
    t.test_heatbath_eq6_equals_dense_rational_function(U)  # the pin holds for the oracle as written
    real_solve = oeofa.system_solve

    def wrong(U_, rhs, alpha, M5, m1, m2, which, a, bc_t, tol=1e-12, maxiter=20000):
        if which == "L" and a != 0.0:
            g = -a
            a = -g * (1.0 / g - 1.0)  # -gamma beta, the P_+ shift
        return real_solve(U_, rhs, alpha, M5, m1, m2, which, a, bc_t, tol, maxiter)

    monkeypatch.setattr(oeofa, "system_solve", wrong)
    with pytest.raises(AssertionError):
        t.test_heatbath_eq6_equals_dense_rational_function(U)


def test_force_part_pin_catches_a_swapped_sign(monkeypatch):
    """The S_R part of Eq. (7) enters with -k; flipping it breaks the finite-difference pin."""
    import test_oracle_eofa as t
    U = inputs.gauge_field(t.DIMS, 0.8, 1)
    real = oeofa.force_from_chi

    def flipped(U_, chiL, chiR, k, bc_t):
        F, im = real(U_, chiL, chiR, k, bc_t)
        if not np.any(chiL):  # the S_R-only call made by force_part
            return -F, im
        return F, im

    monkeypatch.setattr(oeofa, "force_from_chi", flipped)
    with pytest.raises(AssertionError):
        t.test_force_parts_match_partial_action_differences(U)


def test_creutz_pin_catches_a_flipped_metropolis_sign(monkeypatch):
    """Accepting with exp(+dH) drives the chain away from exp(-S): <dH> turns negative."""
    monkeypatch.setattr(gauge, "metropolis", lambda dH, u: bool(np.isfinite(dH) and u < np.exp(dH)))
    dims = (2, 2, 2, 2)
    U = inputs.gauge_field(dims, 0.3, 1)
    n, warm = 300, 60
    Ps = [inputs.momenta(dims, 200, stream=10 + k) for k in range(n + warm)]
    us = inputs.uniform(inputs.stream_key(200, 9), n + warm)
    _, recs = gauge.hmc_chain(U, Ps, us, BETA, 1.0, 8, "leapfrog")
    dH = np.array([r[0] for r in recs])[warm:]
    assert not dH.mean() > 0
