"""Full-size checks: the kernels in the launch configuration the benchmark times.

24^3 x 64, Ls = 24 (the benchmark lattice): the even-odd hop and the fused
G^{-1} D_hop kernel in every storage precision, compared at sampled output
sites with the oracle's single-site evaluation of the same definitions.
16^4 x 16: mixed-precision and FP64 D_DWF solves of four sources to a true
residual of 1e-10, one of them checked with the oracle operator.
"""
import numpy as np
import pytest

from oracle import dwf
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

DIMS, LS = (24, 24, 24, 64), 24
ALPHA, M5, MF = 2.0, 1.8, 0.0362


@pytest.fixture(scope="module")
def big():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa
    eofa.load_library()
    U = inputs.gauge_field(DIMS, 0.7, 3)
    lat = eofa.Lattice(DIMS, LS, bc_t=-1)
    lat.gauge_load(U)
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    psi = torch.randn(lat.V * LS * 12, dtype=torch.complex128, device="cuda", generator=g)
    return eofa, lat, U, psi, psi.cpu().numpy().reshape(lat.shape5)


def _samples(n, seed, parity):
    rng = np.random.default_rng(seed)
    X, Y, Z, T = DIMS
    out = []
    while len(out) < n:
        t, z, y, x = (int(rng.integers(T)), int(rng.integers(Z)), int(rng.integers(Y)), int(rng.integers(X)))
        if (x + y + z + t) % 2 == parity:
            out.append((t, z, y, x))
    # include the t boundary on both sides
    for t in (0, T - 1):
        for x in range(2):
            if (x + t) % 2 == parity:
                out.append((t, 0, 0, x))
    return out


def _run(eofa, lat, psi, prec, out_par, dag, schur):
    import torch
    nb = lat.field_bytes(prec)
    ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
    od = torch.empty_like(ev)
    out = torch.empty_like(ev)
    lat.pack_dev(prec, psi, ev, od)
    src = od if out_par == 0 else ev
    if schur:
        lat.schur_hop_dev(prec, out_par, dag, src, out, ALPHA, M5, MF)
    else:
        lat.hop_dev(prec, out_par, dag, src, out)
    res = torch.empty_like(psi)
    if out_par == 0:
        lat.unpack_dev(prec, out, od, res)
    else:
        lat.unpack_dev(prec, ev, out, res)
    torch.cuda.synchronize()
    return res.cpu().numpy().reshape(lat.shape5)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6), (2, 3e-3)])
def test_hop_full_size_sampled(big, prec, tol):
    eofa, lat, U, psi, psi_h = big
    for out_par, dag in ((0, 0), (1, 1)):
        got = _run(eofa, lat, psi, prec, out_par, dag, schur=False)
        rng = np.random.default_rng(prec)
        num = den = 0.0
        for site in _samples(24, 10 + out_par, out_par):
            s = int(rng.integers(LS))
            ref = dwf.wilson_hop_at(U, psi_h, site, s, -1, dagger=bool(dag))
            num += np.sum(np.abs(got[(s,) + site] - ref) ** 2)
            den += np.sum(np.abs(ref) ** 2)
        assert np.sqrt(num / den) < tol, (prec, out_par, dag, np.sqrt(num / den))


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6), (2, 3e-3)])
def test_schur_hop_full_size_sampled(big, prec, tol):
    eofa, lat, U, psi, psi_h = big
    Pp, Pm = dwf.dperp_matrices(LS, ALPHA, MF)
    one = np.eye(LS)
    Gp, Gm = np.linalg.inv((4 - M5) * one + Pp), np.linalg.inv((4 - M5) * one + Pm)
    for out_par, dag in ((0, 0), (1, 1)):
        got = _run(eofa, lat, psi, prec, out_par, dag, schur=True)
        num = den = 0.0
        for site in _samples(6, 20 + out_par, out_par):
            hop = np.stack([dwf.wilson_hop_at(U, psi_h, site, s, -1, dagger=bool(dag)) for s in range(LS)])
            Bp, Bm = (Gp.T, Gm.T) if dag else (Gp, Gm)
            ref = np.einsum("st,tc->sc", Bp, hop.reshape(LS, 12))
            refm = np.einsum("st,tc->sc", Bm, hop.reshape(LS, 12))
            ref[:, 6:] = refm[:, 6:]
            g = np.stack([got[(s,) + site].reshape(12) for s in range(LS)])
            num += np.sum(np.abs(g - ref) ** 2)
            den += np.sum(np.abs(ref) ** 2)
        assert np.sqrt(num / den) < tol, (prec, out_par, dag, np.sqrt(num / den))


def test_dwf_solves_16_4_x_16_four_sources():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa
    dims, Ls = (16, 16, 16, 16), 16
    U = inputs.gauge_field(dims, 0.6, 2)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    times = {}
    for src in range(4):
        b = inputs.fermion5d(dims, Ls, 2, stream=50 + src)
        for prec in (eofa.PREC_MIXED_F16, eofa.PREC_MIXED_F32, eofa.PREC_F64):
            x, info = lat.solve(b, system=eofa.SYS_DWF, alpha=2.0, M5=M5, mf=0.04, precision=prec, tol=1e-10)
            assert info.true_resid <= 1e-10
            times.setdefault(prec, []).append(info.seconds)
            if src == 0 and prec == eofa.PREC_MIXED_F16:
                res = np.linalg.norm(b - dwf.dwf(U, x, 2.0, M5, 0.04, -1)) / np.linalg.norm(b)
                assert res <= 1.05e-10
    print("16^4x16 D_DWF solves (s):", {k: np.round(v, 3).tolist() for k, v in times.items()})
    lat.close()
