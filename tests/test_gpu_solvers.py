"""GPU solves, EOFA action and force against the FP64 oracle (through the C ABI).

Solves are judged by the FP64 true residual of the full system (<= tol) on
both sides; solutions are compared at a tolerance set by the residuals.
"""
import numpy as np
import pytest

from oracle import dwf, eofa as oeofa, solve as osolve
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

ALPHA, M5, M1, M2 = 2.0, 1.8, 0.04, 1.0


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


def _setup(eofa, dims, Ls, bc=-1, seed=1, eps=0.3):
    U = inputs.gauge_field(dims, eps, seed)
    lat = eofa.Lattice(dims, Ls, bc_t=bc)
    lat.gauge_load(U)
    return lat, U


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_dwf_solve_true_residual(eofa, prec, alpha):
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls)
    b = inputs.fermion5d(dims, Ls, 5)
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=alpha, M5=M5, mf=M1, precision=prec, tol=1e-10)
    res = np.linalg.norm(b - dwf.dwf(U, x, alpha, M5, M1, -1)) / np.linalg.norm(b)
    assert res <= 1.05e-10, res
    assert info.true_resid <= 1e-10
    assert abs(info.true_resid - res) < 1e-3 * res + 1e-14
    if prec > 0:
        assert info.reliable_updates >= 1


def test_dwf_solve_matches_oracle_solution(eofa):
    dims, Ls = (4, 4, 2, 4), 6
    lat, U = _setup(eofa, dims, Ls, eps=0.5)
    b = inputs.fermion5d(dims, Ls, 6)
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=0.1, tol=1e-13)
    xo, it, res = osolve.cgnr(lambda v: dwf.dwf(U, v, ALPHA, M5, 0.1, -1),
                              lambda v: dwf.dwf_dag(U, v, ALPHA, M5, 0.1, -1), b, tol=1e-13)
    assert _rel(x, xo) < 1e-10


@pytest.mark.parametrize("cfg", ["5,1,2", "2,1,3", "5,1,-2", "4,1,-3"])
def test_solves_with_staged_dslash(eofa, cfg, monkeypatch):
    """The staged (bulk-copy) and pipelined (cp.async) dslash kernels, forced
    for every launch including the solver's fused axpy form, give the
    oracle's D_DWF solution in FP64 and a converged mixed-precision EOFA
    solve (ragged last tile at NS = 5)."""
    monkeypatch.setenv("EOFA_DSLASH_CONFIG", cfg)
    dims, Ls = (4, 4, 2, 4), 8
    lat, U = _setup(eofa, dims, Ls, eps=0.5)
    b = inputs.fermion5d(dims, Ls, 6)
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=0.1, tol=1e-13)
    xo, it, res = osolve.cgnr(lambda v: dwf.dwf(U, v, ALPHA, M5, 0.1, -1),
                              lambda v: dwf.dwf_dag(U, v, ALPHA, M5, 0.1, -1), b, tol=1e-13)
    assert _rel(x, xo) < 1e-10
    x, info = lat.solve(b, system=1, alpha=ALPHA, M5=M5, m1=M1, m2=M2, shift=-0.3, precision=1, tol=1e-10)
    Ax = oeofa.system_apply(U, x, ALPHA, M5, M1, M2, "L", -0.3, -1)
    assert np.linalg.norm(b - Ax) / np.linalg.norm(b) < 2e-10
    assert info.reliable_updates >= 1


def test_dwf_solve_warm_start(eofa):
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls)
    b = inputs.fermion5d(dims, Ls, 7)
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=M1, tol=1e-8)
    x2, info2 = lat.solve(b, x0=x, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=M1, tol=1e-10)
    assert info2.true_resid <= 1e-10
    assert info2.iters < info.iters


@pytest.mark.parametrize("which,shift", [(1, 0.0), (2, -1.0), (1, -0.3), (2, -0.7)])
@pytest.mark.parametrize("prec", [0, 1])
def test_eofa_system_solve(eofa, which, shift, prec):
    """Eq. (8): (H(m) + a Delta P) psi = phi; residual checked with the oracle operator."""
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls, eps=0.4)
    rhs = inputs.fermion5d(dims, Ls, 8)
    x, info = lat.solve(rhs, system=which, alpha=ALPHA, M5=M5, m1=M1, m2=M2, shift=shift, precision=prec, tol=1e-10)
    wh = "L" if which == 1 else "R"
    Ax = oeofa.system_apply(U, x, ALPHA, M5, M1, M2, wh, shift, -1)
    res = np.linalg.norm(rhs - Ax) / np.linalg.norm(rhs)
    assert res <= 1.05e-10, res


def test_action_matches_oracle(eofa):
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls)
    phi = inputs.fermion4d(dims, 1)
    S_ref = oeofa.action(U, phi, Ls, ALPHA, M5, M1, M2, -1, tol=1e-13)
    for prec in (0, 1, 2):
        S, info = lat.action(phi, ALPHA, M5, M1, M2, precision=prec, tol=1e-11)
        assert abs(S - S_ref) < 1e-9 * abs(S_ref), (prec, S, S_ref)


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_force_matches_oracle(eofa, alpha):
    import torch
    dims, Ls = (4, 2, 2, 4), 6
    lat, U = _setup(eofa, dims, Ls, eps=0.6)
    phi = inputs.fermion4d(dims, 2)
    F, S, info = lat.force(phi, alpha, M5, M1, M2, precision=0, tol=1e-13)
    Fo = oeofa.force(U, phi, Ls, alpha, M5, M1, M2, -1, tol=1e-13)
    assert np.abs(F - Fo).max() < 1e-9 * np.abs(Fo).max()
    # force kernel alone, same chi on both sides: 1e-12
    chiL, chiR, _ = oeofa.pseudofermion_solutions(U, phi, Ls, alpha, M5, M1, M2, -1, tol=1e-12)
    k = oeofa.k_coefficient(Ls, alpha, M1, M2)
    Fo2, _ = oeofa.force_from_chi(U, chiL, chiR, k, -1)
    Fd = torch.empty(lat.shapeU, dtype=torch.complex128, device="cuda")
    lat.force_from_chi_dev(k, torch.from_numpy(chiL).cuda(), torch.from_numpy(chiR).cuda(), Fd)
    torch.cuda.synchronize()
    assert _rel(Fd.cpu().numpy(), Fo2) < 1e-12


# ---------------------------------------------------------------- failure statuses (host-side inputs only)

@pytest.mark.parametrize("prec", [0, 1])
def test_solve_maxiter_reports_not_converged(eofa, prec):
    """maxiter = 1 cannot reach 1e-10: EOFA_ENOTCONV, with info filled and x the current iterate."""
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls)
    b = inputs.fermion5d(dims, Ls, 7)
    x, info = lat.solve(b, check=False, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=M1, precision=prec, tol=1e-10,
                        maxiter=1)
    assert info.status == eofa.ENOTCONV
    assert info.iters == 1
    assert 1e-10 < info.true_resid < 1.0
    res = np.linalg.norm(b - dwf.dwf(U, x, ALPHA, M5, M1, -1)) / np.linalg.norm(b)
    assert abs(res - info.true_resid) < 1e-6 * res
    msg = lat.lib.eofa_last_error(lat.ctx).decode()
    assert "did not reach tol" in msg
    lat.close()


def test_solve_nan_source_reports_numeric(eofa):
    dims, Ls = (4, 4, 4, 4), 8
    lat, _ = _setup(eofa, dims, Ls)
    b = inputs.fermion5d(dims, Ls, 8)
    b.reshape(-1)[17] = np.nan
    _, info = lat.solve(b, check=False, system=eofa.SYS_EOFA_L, alpha=ALPHA, M5=M5, m1=M1, m2=M2, precision=1,
                        tol=1e-10)
    assert info.status == eofa.ENUMERIC
    with pytest.raises(eofa.EOFAError) as ei:
        lat.solve(b, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=M1, precision=0, tol=1e-10)
    assert ei.value.code == eofa.ENUMERIC
    # the context stays usable
    b2 = inputs.fermion5d(dims, Ls, 9)
    _, info2 = lat.solve(b2, system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=M1, precision=1, tol=1e-10)
    assert info2.status == eofa.OK and info2.true_resid <= 1e-10
    lat.close()


@pytest.mark.parametrize("system", [0, 1, 2])
def test_solve_zero_source_returns_zero(eofa, system):
    dims, Ls = (4, 4, 2, 4), 6
    lat, _ = _setup(eofa, dims, Ls)
    b = np.zeros(lat.shape5, dtype=np.complex128)
    x0 = inputs.fermion5d(dims, Ls, 10)  # overwritten: the solution of a zero source is zero
    x, info = lat.solve(b, x0=x0, system=system, alpha=ALPHA, M5=M5, mf=M1, m1=M1, m2=M2,
                        shift=-1.0 if system == 2 else 0.0, precision=1, tol=1e-10)
    assert info.status == eofa.OK
    assert info.iters == 0
    assert np.count_nonzero(x) == 0
    lat.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cg_forms_reach_the_oracle_residual(eofa, prec):
    """The five- and six-launch CG iterations, each forced, and the timed
    choice (which switches form between iterations while it times them) all
    reach the true residual of the oracle's EOFA system; in FP64 the forced
    forms agree with each other to the solve tolerance.  After a solve the
    timed choice is one of the two forms."""
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls, eps=0.5)
    b = inputs.fermion5d(dims, Ls, 7)
    assert lat.cg_form(prec) == eofa.CG_FORM_AUTO
    sols = {}
    for form in (eofa.CG_FORM_FIVE, eofa.CG_FORM_SIX, eofa.CG_FORM_AUTO):
        lat.set_cg_form(prec, form)
        assert lat.cg_form(prec) == form
        x, info = lat.solve(b, system=1, alpha=ALPHA, M5=M5, m1=M1, m2=M2, shift=-0.3, precision=prec,
                            tol=1e-10)
        Ax = oeofa.system_apply(U, x, ALPHA, M5, M1, M2, "L", -0.3, -1)
        res = np.linalg.norm(b - Ax) / np.linalg.norm(b)
        assert res <= 1.05e-10, (form, res)
        assert info.iters > 10
        sols[form] = x
    assert lat.cg_form(prec) in (eofa.CG_FORM_FIVE, eofa.CG_FORM_SIX)
    if prec == 0:
        assert _rel(sols[eofa.CG_FORM_FIVE], sols[eofa.CG_FORM_SIX]) < 1e-8


def test_cg_form_rejects_bad_arguments(eofa):
    lat, U = _setup(eofa, (4, 4, 2, 4), 4)
    with pytest.raises(eofa.EOFAError):
        lat.set_cg_form(3, eofa.CG_FORM_FIVE)
    with pytest.raises(eofa.EOFAError):
        lat.set_cg_form(1, 2)
    assert lat.cg_form(1) == eofa.CG_FORM_AUTO


def test_fp16_solve_recomputes_mostly_in_fp32(eofa):
    """FP16 inner storage: the residual is recomputed in FP32 at every ~0.1
    reduction (relative to the last FP64 residual) and in FP64 at every ~1e-4
    reduction; the solve still reaches the oracle's true residual.  FP32
    inner storage recomputes in FP64 only."""
    dims, Ls = (4, 4, 4, 4), 8
    lat, U = _setup(eofa, dims, Ls)
    b = inputs.fermion5d(dims, Ls, 5)
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=2.0, M5=M5, mf=M1, precision=2, tol=1e-10)
    res = np.linalg.norm(b - dwf.dwf(U, x, 2.0, M5, M1, -1)) / np.linalg.norm(b)
    assert res <= 1.05e-10, res
    assert 1 <= info.reliable_updates <= 4, info.reliable_updates
    assert info.low_updates >= 4 and info.low_updates > info.reliable_updates, info.low_updates
    x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=2.0, M5=M5, mf=M1, precision=1, tol=1e-10)
    assert info.low_updates == 0
