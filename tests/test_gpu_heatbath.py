"""GPU EOFA heatbath, Eq. (6): phi = f(M_EOFA) eta through 2 N_p solves of Eq. (8).

Compared with the FP64 oracle (whose Eq. (6) is pinned to the dense rational
function of M_EOFA on CPU) on the same coefficients and noise, at sizes the
oracle finishes in seconds; the chronological initial guesses must not change
the result and must cut the iteration count.
"""
import numpy as np
import pytest

from oracle import eofa as oeofa
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

M5, M1, M2 = 1.8, 0.04, 1.0


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


def _heatbath(lat, eta_np, alpha, coeffs, precision, tol, forecast):
    import torch
    a0, al, be = coeffs
    eta = torch.from_numpy(eta_np).cuda()
    phi = torch.empty_like(eta)
    info = lat.heatbath_dev(eta, phi, alpha, M5, M1, M2, a0, al, be, precision=precision, tol=tol,
                            forecast=forecast)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), info


@pytest.mark.parametrize("alpha,dims,forecast", [(1.0, (2, 2, 2, 2), False), (2.0, (2, 2, 2, 4), True)])
def test_heatbath_matches_oracle(eofa, alpha, dims, forecast):
    Ls = 4
    U = inputs.gauge_field(dims, 0.5, 11)
    eta = inputs.fermion4d(dims, 12)
    coeffs = eofa.rational_inv_sqrt(4, 0.02, 8.0)[:3]
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    phi, info = _heatbath(lat, eta, alpha, coeffs, eofa.PREC_F64, 1e-13, forecast)
    ref = oeofa.heatbath(U, eta, Ls, alpha, M5, M1, M2, -1.0, *coeffs, tol=1e-13)
    assert len(info) == 8 and all(i.status == 0 for i in info)
    assert np.linalg.norm(phi - ref) < 1e-11 * np.linalg.norm(ref)
    lat.close()


def test_heatbath_f_of_m_inverts_square_root(eofa):
    """With f ~ x^-1/2 on a range holding the spectrum, the action of the
    heatbath field, phi^+ M phi, reproduces |eta|^2 to the approximation
    error, which falls with the number of poles."""
    dims, Ls, alpha = (4, 4, 4, 4), 8, 2.0
    U = inputs.gauge_field(dims, 0.5, 3)
    eta = inputs.fermion4d(dims, 4)
    e2 = np.vdot(eta, eta).real
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    devs = []
    for n in (4, 8, 16):
        a0, al, be, err = eofa.rational_inv_sqrt(n, 1e-4, 100.0)
        phi, _ = _heatbath(lat, eta, alpha, (a0, al, be), eofa.PREC_F64, 1e-13, True)
        S = lat.action(phi, alpha, M5, M1, M2, precision=0, tol=1e-13)[0]
        devs.append(abs(S - e2) / e2)
        assert devs[-1] < 4 * err + 1e-10, (n, devs[-1], err)
    assert devs[2] < devs[1] < devs[0]
    lat.close()


def test_heatbath_forecast_saves_iterations_and_mixed_precision(eofa):
    dims, Ls, alpha = (8, 8, 8, 8), 12, 2.0
    U = inputs.gauge_field(dims, 0.4, 21)
    eta = inputs.fermion4d(dims, 22)
    coeffs = eofa.rational_inv_sqrt(10, 1e-3, 20.0)[:3]
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    phi0, info0 = _heatbath(lat, eta, alpha, coeffs, eofa.PREC_F64, 1e-11, False)
    phi1, info1 = _heatbath(lat, eta, alpha, coeffs, eofa.PREC_F64, 1e-11, True)
    phi2, info2 = _heatbath(lat, eta, alpha, coeffs, eofa.PREC_MIXED_F32, 1e-11, True)
    n0, n1 = sum(i.iters for i in info0), sum(i.iters for i in info1)
    per0 = [info0[2 * l].iters + info0[2 * l + 1].iters for l in range(10)]
    per1 = [info1[2 * l].iters + info1[2 * l + 1].iters for l in range(10)]
    # Sec. 5.2 reports the iteration count about halved by the tenth pole on
    # its ensemble.  Measured here (8^4 x 12, 10 poles, FP64 to 1e-11): 0.62
    # over all 20 solves (8747 -> 5417) and 0.64 at the tenth pole
    # (1014 -> 652); the bounds keep ~10% margin above those.
    assert n1 < 0.7 * n0, (n0, n1, per0, per1)
    assert per1[9] <= 0.7 * per0[9], (per0, per1)
    ref = np.linalg.norm(phi0)
    assert np.linalg.norm(phi1 - phi0) < 1e-9 * ref
    assert np.linalg.norm(phi2 - phi0) < 1e-9 * ref
    lat.close()


def test_heatbath_rejects_bad_poles(eofa):
    import torch
    dims, Ls = (4, 4, 2, 4), 6
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(inputs.gauge_field(dims, 0.5, 1))
    eta = torch.zeros(lat.shape4, dtype=torch.complex128, device="cuda")
    with pytest.raises(eofa.EOFAError):
        lat.heatbath_dev(eta, torch.empty_like(eta), 1.0, M5, M1, M2, 0.5, [1.0], [-0.1])
    with pytest.raises(eofa.EOFAError):
        lat.heatbath_dev(eta, torch.empty_like(eta), 1.0, M5, M2, M1, 0.5, [1.0], [0.1])
    lat.close()
