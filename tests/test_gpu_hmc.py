"""GPU gauge action / force and force-gradient HMC trajectories (Sec. 5)
against the oracle, plus the fourth-order dH scaling and reversibility of the
device integrator."""
import numpy as np
import pytest

from oracle import gauge
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

ALPHA, M5, M1, M2, BETA = 2.0, 1.8, 0.04, 1.0, 5.7


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_gauge_action_and_force_match_oracle(eofa):
    import torch
    dims = (4, 4, 2, 6)
    U = inputs.gauge_field(dims, 0.6, 3)
    lat = eofa.Lattice(dims, 4)
    lat.gauge_load(U)
    S = lat.gauge_action_dev(BETA)
    assert S == pytest.approx(gauge.action(U, BETA), rel=1e-13)
    F = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    lat.gauge_force_dev(BETA, F, U=_dev(U))
    Fo = gauge.force(U, BETA)
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-12 * np.abs(Fo).max()
    lat.gauge_force_dev(BETA, F, accumulate=True)
    torch.cuda.synchronize()
    assert np.abs(F.cpu().numpy() - 2 * Fo).max() < 1e-12 * np.abs(Fo).max()
    lat.close()


@pytest.mark.parametrize("integrator,scheme", [(0, "leapfrog"), (1, "pqpqp"), (2, "qpqpq")])
def test_pure_gauge_trajectory_matches_oracle(eofa, integrator, scheme):
    import torch
    dims = (4, 4, 2, 4)
    U = inputs.gauge_field(dims, 0.5, 5)
    P = inputs.momenta(dims, 6)
    lat = eofa.Lattice(dims, 4)
    lat.gauge_load(U)
    Pd = _dev(P)
    Ud = torch.empty_like(Pd)
    info = lat.hmc_trajectory_dev(Pd, None, Ud, beta=BETA, integrator=integrator, nsteps=3, tau=0.6)
    U1, P1, dH = gauge.trajectory(U, P, gauge.Forces(BETA), 0.6, 3, scheme)
    assert np.abs(Ud.cpu().numpy() - U1).max() < 1e-11
    assert np.abs(Pd.cpu().numpy() - P1).max() < 1e-10
    assert info["dH"] == pytest.approx(dH, abs=1e-9)
    lat.close()


def test_nested_eofa_trajectory_matches_oracle(eofa):
    """EOFA force on the outer level, gauge force nested (2 inner steps), QPQPQ."""
    import torch
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, 0.4, 7)
    P = inputs.momenta(dims, 8)
    phi = inputs.fermion4d(dims, 9)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    Pd, phid = _dev(P), _dev(phi)
    Ud = torch.empty_like(Pd)
    info = lat.hmc_trajectory_dev(Pd, phid, Ud, alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-13, beta=BETA,
                                  integrator=eofa.INT_FG_QPQPQ, nsteps=2, tau=0.5, n_inner=2)
    f = gauge.Forces(BETA, dict(phi=phi, Ls=Ls, alpha=ALPHA, M5=M5, m1=M1, m2=M2, bc_t=-1.0, tol=1e-13))
    U1, P1, dH = gauge.trajectory(U, P, f, 0.5, 2, "qpqpq", n_inner=2)
    assert info["fermion_forces"] == f.n_fermion == 8
    assert np.abs(Ud.cpu().numpy() - U1).max() < 1e-10
    assert np.abs(Pd.cpu().numpy() - P1).max() < 1e-9
    assert info["dH"] == pytest.approx(dH, abs=1e-8)
    lat.close()


def test_force_gradient_fourth_order_and_reversible(eofa):
    """dH(h) / dH(h/2) ~ 16 for the nested QPQPQ force-gradient trajectory with
    EOFA + gauge forces; integrating back with -P recovers U and P."""
    import torch
    dims, Ls = (4, 4, 4, 4), 8
    U = inputs.gauge_field(dims, 0.3, 11)
    P = inputs.momenta(dims, 12)
    phi = inputs.fermion4d(dims, 13)
    kw = dict(alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-13, beta=BETA, integrator=eofa.INT_FG_QPQPQ, tau=0.5,
              n_inner=2)
    lat = eofa.Lattice(dims, Ls)
    dHs = []
    for n in (2, 4):
        lat.gauge_load(U)
        Pd = _dev(P)
        dHs.append(lat.hmc_trajectory_dev(Pd, _dev(phi), None, nsteps=n, **kw)["dH"])
    assert abs(dHs[0] / dHs[1]) == pytest.approx(16, rel=0.3), dHs
    lat.gauge_load(U)
    Pd = _dev(P)
    Ud = torch.empty_like(Pd)
    lat.hmc_trajectory_dev(Pd, _dev(phi), Ud, nsteps=2, **kw)
    Pd.neg_()
    lat.hmc_trajectory_dev(Pd, _dev(phi), Ud, nsteps=2, **kw)
    assert np.abs(Ud.cpu().numpy() - U).max() < 1e-9
    assert np.abs(Pd.cpu().numpy() + P).max() < 1e-8
    lat.close()


def test_trajectory_rejects_bad_parameters(eofa):
    dims = (2, 2, 2, 2)
    lat = eofa.Lattice(dims, 4)
    lat.gauge_load(inputs.gauge_field(dims, 0.3, 1))
    Pd = _dev(inputs.momenta(dims, 2))
    with pytest.raises(eofa.EOFAError):
        lat.hmc_trajectory_dev(Pd, None, None, beta=0.0)  # nothing to integrate
    with pytest.raises(eofa.EOFAError):
        lat.hmc_trajectory_dev(Pd, None, None, beta=BETA, n_inner=2)  # nesting needs a fermion level
    lat.close()


def test_force_parts_match_oracle(eofa):
    """Eq. (7) term by term on the device: F_L + F_R = F, each part vs the oracle."""
    import torch
    from oracle import eofa as oeofa
    dims, Ls = (4, 4, 2, 4), 6
    U = inputs.gauge_field(dims, 0.5, 21)
    phi = inputs.fermion4d(dims, 22)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    shape = U.shape
    FL = torch.empty(shape, dtype=torch.complex128, device="cuda")
    FR = torch.empty_like(FL)
    info = lat.force_parts_dev(_dev(phi), FL, FR, ALPHA, M5, M1, M2, tol=1e-13)
    assert info[0]["iters"] > 0 and info[1]["iters"] > 0
    F, _, _ = lat.force(phi, ALPHA, M5, M1, M2, precision=0, tol=1e-13)
    fl, fr = FL.cpu().numpy(), FR.cpu().numpy()
    assert np.abs(fl + fr - F).max() < 1e-9 * np.abs(F).max()
    for part, got in (("L", fl), ("R", fr)):
        ref = oeofa.force_part(U, phi, Ls, ALPHA, M5, M1, M2, -1.0, part, tol=1e-13)
        assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max(), part
    only = torch.zeros_like(FL)
    info = lat.force_parts_dev(_dev(phi), None, only, ALPHA, M5, M1, M2, tol=1e-13)
    assert info[0]["iters"] == 0 and np.abs(only.cpu().numpy() - fr).max() < 1e-9 * np.abs(fr).max()
    lat.close()


@pytest.mark.parametrize("order,outer", [(1, "R"), (2, "L")])
def test_split_lr_trajectory_matches_oracle(eofa, order, outer):
    """Asymmetric integration: one EOFA term outermost, the other in the middle, gauge innermost."""
    import torch
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, 0.4, 23)
    P = inputs.momenta(dims, 24)
    phi = inputs.fermion4d(dims, 25)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    Pd = _dev(P)
    Ud = torch.empty_like(Pd)
    info = lat.hmc_trajectory_dev(Pd, _dev(phi), Ud, alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-13, beta=BETA,
                                  integrator=eofa.INT_FG_QPQPQ, nsteps=1, tau=0.4, n_inner=1, split_lr=order,
                                  n_middle=2)
    ferm = dict(phi=phi, Ls=Ls, alpha=ALPHA, M5=M5, m1=M1, m2=M2, bc_t=-1.0, tol=1e-13)
    U1, P1, dH = gauge.split_lr_trajectory(U, P, BETA, ferm, 0.4, 1, 2, 1, "qpqpq", outer=outer)
    # 4 outer forces (two displaced kicks) + 3 drifts x 2 steps x 4 middle forces
    assert info["fermion_forces"] == 28
    assert np.abs(Ud.cpu().numpy() - U1).max() < 1e-10
    assert np.abs(Pd.cpu().numpy() - P1).max() < 1e-9
    assert info["dH"] == pytest.approx(dH, abs=1e-8)
    lat.close()


def test_mixed_precision_trajectory_matches_fp64(eofa):
    """The trajectory with mixed FP32 solves (FP64 reliable updates, true
    residual 1e-11) ends where the all-FP64 one does, to the solver tolerance."""
    import torch
    dims, Ls = (4, 4, 4, 4), 8
    U = inputs.gauge_field(dims, 0.3, 31)
    P = inputs.momenta(dims, 32)
    phi = inputs.fermion4d(dims, 33)
    kw = dict(alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-11, beta=BETA, integrator=eofa.INT_FG_QPQPQ, tau=0.5,
              nsteps=2, n_inner=2)
    lat = eofa.Lattice(dims, Ls)
    ends = []
    for prec in (eofa.PREC_F64, eofa.PREC_MIXED_F32):
        lat.gauge_load(U)
        Pd = _dev(P)
        Ud = torch.empty_like(Pd)
        info = lat.hmc_trajectory_dev(Pd, _dev(phi), Ud, precision=prec, **kw)
        ends.append((Ud.cpu().numpy(), Pd.cpu().numpy(), info["dH"]))
    (U64, P64, dH64), (U32, P32, dH32) = ends
    assert np.abs(U32 - U64).max() < 1e-8
    assert np.abs(P32 - P64).max() < 1e-7
    assert abs(dH32 - dH64) < 1e-6 * max(1.0, abs(dH64))
    lat.close()


# ---------------------------------------------------------------- the HMC chain (Metropolis)

def _rational_fit(n, lmin, lmax):
    """Some rational f(x) = alpha0 + sum_l alpha_l / (x + beta_l) close to x^-1/2
    on [lmin, lmax] (least squares at fixed poles); the chain comparison only
    needs both sides to use the same f."""
    betas = np.geomspace(lmin, lmax, n)
    x = np.geomspace(lmin / 2, lmax * 2, 600)
    A = np.column_stack([np.ones_like(x)] + [1.0 / (x + b) for b in betas]) * np.sqrt(x)[:, None]
    c = np.linalg.lstsq(A, np.ones_like(x), rcond=None)[0]
    return c[0], c[1:], betas


def test_hmc_chain_matches_oracle_chain(eofa):
    """Four trajectories on 2^4 x Ls=4 from the same random numbers on both
    sides (momenta, heatbath noise, Metropolis uniforms): heatbath refresh of
    phi, nested QPQPQ trajectory with the EOFA and Wilson gauge forces,
    accept/reject.  The decisions, dH, the start action and the final links
    agree with the oracle chain; the chain has both outcomes."""
    import torch
    dims, Ls, ntraj = (2, 2, 2, 2), 4, 4
    U0 = inputs.gauge_field(dims, 0.4, 31)
    Ps = [inputs.momenta(dims, 32, stream=10 + k) for k in range(ntraj)]
    etas = [inputs.fermion4d(dims, 33, stream=20 + k) / np.sqrt(2.0) for k in range(ntraj)]  # density exp(-eta^+ eta)
    us = inputs.uniform(inputs.stream_key(34, 1), ntraj)
    rational = _rational_fit(10, 1e-2, 10.0)
    fermion = dict(Ls=Ls, alpha=ALPHA, M5=M5, m1=M1, m2=M2, bc_t=-1.0, tol=1e-13)
    Uo, recs = gauge.hmc_chain(U0, Ps, us, BETA, 1.0, 1, "qpqpq", n_inner=2, fermion=fermion, etas=etas,
                               rational=rational)
    assert {r[1] for r in recs} == {True, False}
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U0)
    Pd = _dev(np.stack(Ps))
    etad = _dev(np.stack(etas))
    Ud = torch.empty(U0.shape, dtype=torch.complex128, device="cuda")
    info = lat.hmc_dev(Pd, etad, us, Ud, alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-13, beta=BETA,
                       integrator=eofa.INT_FG_QPQPQ, nsteps=1, tau=1.0, n_inner=2, rational=rational)
    for k, (dH, acc, S0) in enumerate(recs):
        assert bool(info[k]["accepted"]) == acc, (k, info[k], recs[k])
        assert info[k]["dH"] == pytest.approx(dH, abs=1e-8 * max(1.0, abs(dH)))
        assert info[k]["S_eofa_start"] == pytest.approx(S0, rel=1e-10)
        assert info[k]["eta_norm2"] == pytest.approx(np.vdot(etas[k], etas[k]).real, rel=1e-12)
        assert info[k]["exp_minus_dH"] == pytest.approx(np.exp(-dH), rel=1e-7)
    assert np.abs(Ud.cpu().numpy() - Uo).max() < 1e-10
    # the context's links are the chain's state
    Ud2 = torch.empty_like(Ud)
    lat.hmc_dev(Pd[:1], etad[:1], [0.0], Ud2, alpha=ALPHA, M5=M5, m1=M1, m2=M2, tol=1e-13, beta=BETA,
                integrator=eofa.INT_FG_QPQPQ, nsteps=1, tau=1.0, n_inner=2, rational=rational)
    U5, _ = gauge.hmc_chain(Uo, Ps[:1], [0.0], BETA, 1.0, 1, "qpqpq", n_inner=2, fermion=fermion, etas=etas[:1],
                            rational=rational)
    assert np.abs(Ud2.cpu().numpy() - U5).max() < 1e-10
    lat.close()


def test_hmc_chain_pure_gauge_and_bad_arguments(eofa):
    """npoles = 0 runs a pure-gauge chain (same records as the oracle's); the
    uniforms must lie in [0, 1)."""
    import torch
    dims = (2, 2, 2, 2)
    U0 = inputs.gauge_field(dims, 0.3, 1)
    n = 12
    Ps = [inputs.momenta(dims, 200, stream=10 + k) for k in range(n)]
    us = inputs.uniform(inputs.stream_key(200, 9), n)
    Uo, recs = gauge.hmc_chain(U0, Ps, us, BETA, 1.0, 2, "leapfrog")
    lat = eofa.Lattice(dims, 4)
    lat.gauge_load(U0)
    Ud = torch.empty(U0.shape, dtype=torch.complex128, device="cuda")
    info = lat.hmc_dev(_dev(np.stack(Ps)), None, us, Ud, beta=BETA, integrator=eofa.INT_LEAPFROG, nsteps=2,
                       tau=1.0)
    assert [bool(i["accepted"]) for i in info] == [r[1] for r in recs]
    assert 0 < sum(r[1] for r in recs) < n
    for i, r in zip(info, recs):
        assert i["dH"] == pytest.approx(r[0], abs=1e-9)
    assert np.abs(Ud.cpu().numpy() - Uo).max() < 1e-11
    with pytest.raises(eofa.EOFAError):
        lat.hmc_dev(_dev(np.stack(Ps[:1])), None, [1.0], None, beta=BETA)
    with pytest.raises(eofa.EOFAError):
        lat.hmc_dev(_dev(np.stack(Ps[:1])), None, [0.5], None, beta=0.0)
    lat.close()


def test_checkpoint_resume_continues_the_chain(eofa, tmp_path):
    """Save the links after two trajectories, restore them into a new context and
    continue both: the next trajectory gives the same dH and links bit for bit,
    and the checkpoint holds the chain's links."""
    import torch
    dims = (4, 4, 4, 4)
    U0 = inputs.gauge_field(dims, 0.3, 5)
    Ps = [inputs.momenta(dims, 60, stream=10 + k) for k in range(3)]
    us = [0.0, 0.0, 0.0]  # accept everything: the links move every trajectory
    kw = dict(beta=BETA, integrator=eofa.INT_FG_QPQPQ, nsteps=2, tau=0.5)
    lat = eofa.Lattice(dims, 4)
    lat.gauge_load(U0)
    U2 = torch.empty(U0.shape, dtype=torch.complex128, device="cuda")
    lat.hmc_dev(_dev(np.stack(Ps[:2])), None, us[:2], U2, **kw)
    path = tmp_path / "chain.ckpt"
    lat.gauge_save(path, traj=2)
    saved, traj = eofa.checkpoint_read(path, eofa.CKPT_GAUGE, dims)
    assert traj == 2 and np.array_equal(saved, U2.cpu().numpy())
    lat2 = eofa.Lattice(dims, 4)
    assert lat2.gauge_restore(path) == 2
    Ua, Ub = torch.empty_like(U2), torch.empty_like(U2)
    ia = lat.hmc_dev(_dev(Ps[2][None]), None, us[2:], Ua, **kw)
    ib = lat2.hmc_dev(_dev(Ps[2][None]), None, us[2:], Ub, **kw)
    assert ia[0]["dH"] == ib[0]["dH"]
    assert torch.equal(Ua, Ub)
    lat.close()
    lat2.close()
