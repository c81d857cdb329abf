"""GPU force (Eq. (7)) through autograd and the adjoint kernel, molecular dynamics, batched solves.

Checks against the FP64 oracle and against finite differences of the
action computed by the library itself.
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


def _perturb(U, site, mu, a, w):
    Up = U.copy()
    Up[site + (mu,)] = oeofa.exp_i(w * oeofa.generators()[a]) @ U[site + (mu,)]
    return Up


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_autograd_gradient_matches_finite_differences(eofa, alpha):
    import torch
    from paper_1611_00298_gb300.autograd import eofa_action
    dims, Ls = (4, 4, 2, 4), 6
    U = inputs.gauge_field(dims, 0.5, 4)
    phi_np = inputs.fermion4d(dims, 4)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    phi = torch.from_numpy(phi_np).cuda()
    Ur = torch.view_as_real(torch.from_numpy(U).cuda()).clone().requires_grad_(True)
    S = eofa_action(Ur, phi, lat, alpha, M5, M1, M2, eofa.PREC_F64, 1e-13)
    S.backward()
    G = torch.view_as_complex(Ur.grad).cpu().numpy()
    # the force kernel's F^a equals the gradient projected on i T^a U
    F, S2, _ = lat.force(phi_np, alpha, M5, M1, M2, precision=0, tol=1e-13)
    assert abs(S2 - S.item()) < 1e-10 * abs(S2)
    T = oeofa.generators()
    Fa = oeofa.force_components(F)
    dirs = np.einsum("aij,...jk->...aik", 1j * T, U)  # i T^a U for every link
    Ga = np.einsum("...ij,...aij->...a", np.conj(G), dirs).real
    assert np.abs(Ga - Fa).max() < 1e-9 * np.abs(Fa).max()
    # central differences (4-point, delta = 1e-4) of the library's own action
    rng = np.random.default_rng(5)
    d = 1e-4
    for _ in range(8):
        site = tuple(int(rng.integers(n)) for n in U.shape[:4])
        mu, a = int(rng.integers(4)), int(rng.integers(8))
        vals = []
        for w in (2 * d, d, -d, -2 * d):
            lat.gauge_load(_perturb(U, site, mu, a, w))
            vals.append(lat.action(phi_np, alpha, M5, M1, M2, precision=0, tol=1e-14)[0])
        fd = (-vals[0] + 8 * vals[1] - 8 * vals[2] + vals[3]) / (12 * d)
        assert abs(fd - Ga[site + (mu, a)]) < 2e-6 * max(1.0, abs(fd)), (fd, Ga[site + (mu, a)])
    lat.close()


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_force_sampled_links_16I_shape(eofa, alpha):
    """16^3 x 32, Ls = 12: GPU force at 16 random links vs the oracle's single-link Eq. (7)."""
    import torch
    dims, Ls = (16, 16, 16, 32), 12
    U = inputs.gauge_field(dims, 0.5, 4)
    phi_np = inputs.fermion4d(dims, 4)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    phi = torch.from_numpy(phi_np).cuda()
    chiL = torch.empty(lat.shape5, dtype=torch.complex128, device="cuda")
    chiR = torch.empty_like(chiL)
    S, info = lat.pseudofermion_solutions_dev(phi, chiL, chiR, alpha, M5, M1, M2, eofa.PREC_MIXED_F32, 1e-10)
    assert info[0].true_resid <= 1e-10 and info[1].true_resid <= 1e-10
    k, _, _ = eofa.coefficients(Ls, alpha, M1, M2)
    F = torch.empty(lat.shapeU, dtype=torch.complex128, device="cuda")
    lat.force_from_chi_dev(k, chiL, chiR, F)
    torch.cuda.synchronize()
    Fh = F.cpu().numpy()
    cL, cR = chiL.cpu().numpy(), chiR.cpu().numpy()
    rng = np.random.default_rng(7)
    for _ in range(16):
        site = tuple(int(rng.integers(n)) for n in U.shape[:4])
        mu = int(rng.integers(4))
        ref = oeofa.force_at_link(U, cL, cR, k, -1, site, mu)
        assert np.abs(Fh[site + (mu,)] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    # the t-boundary links carry the antiperiodic phase
    ref = oeofa.force_at_link(U, cL, cR, k, -1, (31, 3, 5, 7), 3)
    assert np.abs(Fh[31, 3, 5, 7, 3] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert np.abs(Fh - np.conj(np.swapaxes(Fh, -1, -2))).max() < 1e-12
    lat.close()


@pytest.mark.parametrize("alpha", [1.0, 2.0])
def test_force_central_differences_16I_shape(eofa, alpha):
    """16^3 x 32, Ls = 12, Shamir (alpha = 1) and Moebius (alpha = 2): the GPU
    force F^a (Eq. (7)) at 16 (link, generator) pairs against central
    differences (delta = 1e-5) of the GPU action (Eq. (5)).  phi is Gaussian on
    one 2^4 block (at the time boundary) and zero elsewhere, so that S is of
    order ten and its change 2 delta F^a is resolved by solves to 1e-12
    (with phi Gaussian everywhere S ~ 3e6 would need 1e-14 accuracy); the
    solves still span the whole lattice.  The pairs sit on and next to the
    block, some on the antiperiodic t-boundary links."""
    dims, Ls = (16, 16, 16, 32), 12
    U = inputs.gauge_field(dims, 0.5, 4)
    full = inputs.fermion4d(dims, 4)
    phi = np.zeros_like(full)
    blk = (slice(30, 32), slice(6, 8), slice(6, 8), slice(6, 8))
    phi[blk] = full[blk]
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    kw = dict(alpha=alpha, M5=M5, m1=M1, m2=M2, precision=eofa.PREC_MIXED_F32, tol=1e-12)
    F, S0, info = lat.force(phi, **kw)
    assert info[0].true_resid <= 1e-12 and info[1].true_resid <= 1e-12
    Fa = oeofa.force_components(F)
    rng = np.random.default_rng(11)
    d = 1e-5
    worst = 0.0
    for n in range(16):
        site = (int(rng.integers(29, 32)), int(rng.integers(5, 9)), int(rng.integers(5, 9)), int(rng.integers(5, 9)))
        mu = 3 if n < 4 else int(rng.integers(4))  # the first four on t-links, some across the boundary
        a = int(rng.integers(8))
        vals = []
        for w in (d, -d):
            lat.gauge_load(_perturb(U, site, mu, a, w))
            vals.append(lat.action(phi, **kw)[0])
        fd = (vals[0] - vals[1]) / (2 * d)
        ref = Fa[site + (mu, a)]
        err = abs(fd - ref)
        worst = max(worst, err / max(1.0, abs(ref)))
        assert err < 1e-5 * max(1.0, abs(ref)) + 1e-6, (site, mu, a, fd, ref)
    assert np.abs(Fa).max() > 1e-2  # the sampled region carries a force
    lat.close()


def test_leapfrog_matches_oracle(eofa):
    import torch
    dims, Ls = (2, 2, 2, 2), 4
    U = inputs.gauge_field(dims, 0.8, 1)
    P = inputs.momenta(dims, 8)
    phi_np = inputs.fermion4d(dims, 8)
    U1o, P1o, dHo = oeofa.leapfrog(U, P, phi_np, Ls, 2.0, M5, M1, M2, -1, nsteps=3, dtau=0.1, tol=1e-14)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    Pd = torch.from_numpy(P.copy()).cuda()
    Ud = torch.from_numpy(U.copy()).cuda()
    phi = torch.from_numpy(phi_np).cuda()
    dH, H0 = lat.leapfrog_dev(phi, Pd, Ud, 2.0, M5, M1, M2, 3, 0.1, precision=0, tol=1e-14)
    torch.cuda.synchronize()
    assert abs(dH - dHo) < 1e-8 * max(1.0, abs(H0)), (dH, dHo)
    assert np.abs(Ud.cpu().numpy() - U1o).max() < 1e-11
    assert np.abs(Pd.cpu().numpy() - P1o).max() < 1e-10
    lat.close()


def test_leapfrog_16I_shape_reversible_and_dtau2(eofa):
    """10-step leapfrog, dtau = 0.1, on 16^3 x 32 x 12; forward then back returns to the start."""
    import torch
    dims, Ls = (16, 16, 16, 32), 12
    U = inputs.gauge_field(dims, 0.5, 4)
    P = inputs.momenta(dims, 4)
    phi_np = inputs.fermion4d(dims, 4)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    phi = torch.from_numpy(phi_np).cuda()
    Pd = torch.from_numpy(P.copy()).cuda()
    Ud = torch.from_numpy(U.copy()).cuda()
    dH1, H0 = lat.leapfrog_dev(phi, Pd, Ud, 2.0, M5, M1, M2, 10, 0.1, precision=eofa.PREC_MIXED_F32, tol=1e-12)
    Pd.neg_()
    dH2, _ = lat.leapfrog_dev(phi, Pd, Ud, 2.0, M5, M1, M2, 10, 0.1, precision=eofa.PREC_MIXED_F32, tol=1e-12)
    torch.cuda.synchronize()
    assert abs(dH1 + dH2) < 1e-6 * abs(H0)
    assert np.abs(Ud.cpu().numpy() - U).max() < 1e-8
    assert np.abs(Pd.cpu().numpy() + P).max() < 1e-8
    print(f"16^3x32x12 leapfrog 10 x 0.1: dH = {dH1:.6e}, H0 = {H0:.6e}")
    lat.close()


def test_batched_matches_single_solves(eofa):
    """Several lattices, L and R systems of Eq. (8) and D_DWF systems in one batched, graph-captured solve."""
    lats = []
    for dims, Ls, seed in (((4, 4, 4, 4), 8, 5), ((6, 4, 4, 6), 12, 6), ((4, 4, 2, 8), 16, 7)):
        lat = eofa.Lattice(dims, Ls)
        lat.gauge_load(inputs.gauge_field(dims, 0.5, seed))
        lats.append((lat, seed))
    ctxs, params, bs, xs, singles = [], [], [], [], []
    for lat, seed in lats:
        for (m1, m2) in ((0.04, 0.2), (0.2, 0.6)):
            for system, shift in ((eofa.SYS_EOFA_L, 0.0), (eofa.SYS_EOFA_R, -1.0)):
                b = inputs.fermion5d(lat.dims, lat.Ls, seed, stream=30 + system)
                kw = dict(system=system, alpha=2.0, M5=M5, m1=m1, m2=m2, shift=shift,
                          precision=eofa.PREC_MIXED_F32, tol=1e-10)
                ctxs.append(lat)
                params.append(lat.solve_params(**kw))
                bs.append(b)
                xs.append(np.zeros_like(b))
                singles.append(lat.solve(b, **kw)[0])
        b = inputs.fermion5d(lat.dims, lat.Ls, seed, stream=40)
        kw = dict(system=eofa.SYS_DWF, alpha=2.0, M5=M5, mf=0.04, precision=eofa.PREC_MIXED_F32, tol=1e-10)
        ctxs.append(lat)
        params.append(lat.solve_params(**kw))
        bs.append(b)
        xs.append(np.zeros_like(b))
        singles.append(lat.solve(b, **kw)[0])
    info = eofa.solve_batched(ctxs, params, bs, xs)
    for i in range(len(bs)):
        assert info[i].status == 0 and info[i].true_resid <= 1e-10
        rel = np.linalg.norm(xs[i] - singles[i]) / np.linalg.norm(singles[i])
        assert rel < 1e-8, (i, rel)
    for lat, _ in lats:
        lat.close()
