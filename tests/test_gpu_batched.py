"""Batched solves against the oracle.

eofa_solve_batched iterates the systems of one lattice together (the
multi-system kernels share every link and neighbour load across them; the CG
loop runs on the device inside a CUDA graph).  Every returned solution is fed
to the oracle's operator: the Eq. (8) system (oracle.eofa.system_apply) or
D_DWF (oracle.dwf.dwf), whole-field where numpy is quick and at sampled sites
(system_apply_at / dwf_at) on the 16^3 x 32 x 16 lattice.

The main case is the batched workload: three lattices 8^4 x 8, 12^4 x 12 and
16^3 x 32 x 16 (links exp(i 0.5 H), seeds 5, 6, 7; alpha = 2, M5 = 1.8), the
mass pairs (0.04, 0.2), (0.2, 0.6), (0.6, 1.0) with the L (a = 0) and R
(a = -1) systems of Eq. (8), plus D_DWF at m_f = 0.04 and 0.2 per lattice:
24 solves to a true residual of 1e-10 in mixed precision.
"""
import numpy as np
import pytest

from oracle import dwf, eofa as oeofa
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

ALPHA, M5 = 2.0, 1.8
PAIRS = ((0.04, 0.2), (0.2, 0.6), (0.6, 1.0))


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


def _systems(eofa, lat, seed, first_stream, pairs=PAIRS, dwf_masses=(0.04, 0.2)):
    out = []
    for m1, m2 in pairs:
        for system, shift in ((eofa.SYS_EOFA_L, 0.0), (eofa.SYS_EOFA_R, -1.0)):
            out.append(dict(system=system, alpha=ALPHA, M5=M5, m1=m1, m2=m2, shift=shift))
    for mf in dwf_masses:
        out.append(dict(system=eofa.SYS_DWF, alpha=ALPHA, M5=M5, mf=mf))
    bs = [inputs.fermion5d(lat.dims, lat.Ls, seed, stream=first_stream + k) for k in range(len(out))]
    return out, bs


def _apply(eofa, U, kw, x):
    if kw["system"] == eofa.SYS_DWF:
        return dwf.dwf(U, x, kw["alpha"], kw["M5"], kw["mf"], -1)
    which = "L" if kw["system"] == eofa.SYS_EOFA_L else "R"
    return oeofa.system_apply(U, x, kw["alpha"], kw["M5"], kw["m1"], kw["m2"], which, kw["shift"], -1)


def _apply_at(eofa, U, kw, x, site, Lx):
    if kw["system"] == eofa.SYS_DWF:
        return dwf.dwf_at(U, x, kw["alpha"], kw["M5"], kw["mf"], -1, site, Lpsi=Lx)
    which = "L" if kw["system"] == eofa.SYS_EOFA_L else "R"
    return oeofa.system_apply_at(U, x, kw["alpha"], kw["M5"], kw["m1"], kw["m2"], which, kw["shift"], -1, site)


def _full_residual(eofa, U, kw, x, b):
    return np.linalg.norm(b - _apply(eofa, U, kw, x)) / np.linalg.norm(b)


def _sampled_residual(eofa, U, kw, x, b, nsites, seed):
    """|b - A x| / |b| estimated from the whole fifth dimension at nsites 4D sites."""
    rng = np.random.default_rng(seed)
    T, Z, Y, X = b.shape[1:5]
    Lx = dwf.L_apply(x, kw["mf"]) if kw["system"] == eofa.SYS_DWF else None
    sites = [(int(rng.integers(T)), int(rng.integers(Z)), int(rng.integers(Y)), int(rng.integers(X)))
             for _ in range(nsites)] + [(0, 0, 0, 0), (T - 1, 0, 0, 1)]
    r2 = b2 = 0.0
    for site in sites:
        bs = b[(slice(None),) + site]
        r2 += np.sum(np.abs(bs - _apply_at(eofa, U, kw, x, site, Lx)) ** 2)
        b2 += np.sum(np.abs(bs) ** 2)
    return np.sqrt(r2 / b2)


def test_batched_workload_three_lattices_24_solves_vs_oracle(eofa):
    lattices = (((8, 8, 8, 8), 8, 5), ((12, 12, 12, 12), 12, 6), ((16, 16, 16, 32), 16, 7))
    lats, Us, ctxs, kws, bs, xs = [], [], [], [], [], []
    for dims, Ls, seed in lattices:
        U = inputs.gauge_field(dims, 0.5, seed)
        lat = eofa.Lattice(dims, Ls)
        lat.gauge_load(U)
        lats.append(lat)
        Us.append(U)
        sy, b = _systems(eofa, lat, seed, 60)
        for kw, bb in zip(sy, b):
            ctxs.append(lat)
            kws.append((len(lats) - 1, kw))
            bs.append(bb)
            xs.append(np.zeros_like(bb))
    assert len(bs) == 24
    params = [ctxs[i].solve_params(precision=eofa.PREC_MIXED_F32, tol=1e-10, **kw) for i, (_, kw) in enumerate(kws)]
    info = eofa.solve_batched(ctxs, params, bs, xs)
    big_checked = 0
    for i, (li, kw) in enumerate(kws):
        assert info[i].status == eofa.OK and info[i].true_resid <= 1e-10, (i, info[i].as_dict())
        U = Us[li]
        if li < 2:
            res = _full_residual(eofa, U, kw, xs[i], bs[i])
            assert res <= 1.05e-10, (i, kw, res)
            assert abs(res - info[i].true_resid) <= 1e-3 * res + 1e-15
        else:
            est = _sampled_residual(eofa, U, kw, xs[i], bs[i], 24, seed=i)
            assert est <= 3e-10, (i, kw, est)
            hard = (kw["system"] == eofa.SYS_DWF and kw["mf"] == 0.04) or (
                kw["system"] == eofa.SYS_EOFA_L and kw["m1"] == 0.04)
            if hard:
                res = _full_residual(eofa, U, kw, xs[i], bs[i])
                assert res <= 1.05e-10, (i, kw, res)
                big_checked += 1
    assert big_checked == 2
    for lat in lats:
        lat.close()


def test_batched_groups_precisions_and_edge_cases(eofa):
    """More systems on one lattice than one group holds (two groups on one context
    at once), FP64, FP32 and FP16 groups side by side, a zero source, and a
    system that stops at maxiter with EOFA_ENOTCONV while the rest converge."""
    dims, Ls, seed = (4, 4, 4, 4), 8, 9
    U = inputs.gauge_field(dims, 0.5, seed)
    lat = eofa.Lattice(dims, Ls)
    lat.gauge_load(U)
    pairs = ((0.04, 0.2), (0.1, 0.3), (0.2, 0.6), (0.3, 0.5), (0.5, 0.8), (0.6, 1.0), (0.05, 0.9), (0.4, 0.45),
             (0.01, 0.02))
    sy, bs = _systems(eofa, lat, seed, 100, pairs=pairs, dwf_masses=(0.04, 0.1, 0.2))
    assert len(sy) == 21
    precs = [eofa.PREC_MIXED_F32] * 21
    precs[3] = precs[7] = eofa.PREC_F64
    precs[5] = precs[11] = eofa.PREC_MIXED_F16
    bs[4] = np.zeros_like(bs[4])
    maxiter = [100000] * 21
    maxiter[9] = 5
    params = [lat.solve_params(precision=p, tol=1e-10, maxiter=m, **kw) for p, m, kw in zip(precs, maxiter, sy)]
    xs = [np.zeros_like(b) for b in bs]
    info = eofa.solve_batched([lat] * 21, params, bs, xs, check=False)
    for i, kw in enumerate(sy):
        if i == 9:
            assert info[i].status == eofa.ENOTCONV
            assert 5 <= info[i].iters < 5 + 8
            assert info[i].true_resid > 1e-10
            res = _full_residual(eofa, U, kw, xs[i], bs[i])
            assert abs(res - info[i].true_resid) <= 1e-6 * res
            continue
        assert info[i].status == eofa.OK, (i, info[i].as_dict())
        if i == 4:
            assert np.count_nonzero(xs[i]) == 0 and info[i].iters == 0
            continue
        res = _full_residual(eofa, U, kw, xs[i], bs[i])
        assert res <= 1.05e-10, (i, precs[i], kw, res)
    lat.close()
