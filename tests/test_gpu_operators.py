"""GPU parity of the operator kernels against the FP64 oracle (through the C ABI).

Tolerance: 1e-12 relative L2 per output vector for FP64 operator applications.
"""
import numpy as np
import pytest

from oracle import dwf
from paper_1611_00298_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    # dims, Ls, alpha, M5, mf, bc
    ((4, 4, 4, 4), 8, 2.0, 1.8, 0.04, -1),
    ((2, 2, 2, 2), 4, 2.0, 1.8, 0.04, -1),    # L = 2: x+mu = x-mu
    ((4, 2, 6, 4), 5, 1.0, 1.8, 0.3, +1),     # Shamir, odd Ls, periodic
    ((2, 4, 2, 6), 1, 3.0, 1.4, 0.0, -1),     # Ls = 1, m_f = 0
    ((4, 4, 2, 2), 6, 4.0, 1.8, 1.0, -1),     # m_f = 1
    ((6, 4, 4, 8), 12, 2.0, 1.8, 0.0362, -1),  # several tiles, ragged tail
]


@pytest.fixture(scope="module")
def eofa():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1611_00298_gb300 import eofa as e
    e.load_library()
    return e


def _setup(eofa, dims, Ls, bc, seed=1, eps=0.5):
    U = inputs.gauge_field(dims, eps, seed)
    lat = eofa.Lattice(dims, Ls, bc_t=bc)
    lat.gauge_load(U)
    return lat, U


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES)
def test_dwf_apply_parity(eofa, case):
    dims, Ls, alpha, M5, mf, bc = case
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 2)
    out = lat.dwf_apply(psi, alpha, M5, mf)
    assert _rel(out, dwf.dwf(U, psi, alpha, M5, mf, bc)) < 1e-12
    out = lat.dwf_apply(psi, alpha, M5, mf, dagger=True)
    assert _rel(out, dwf.dwf_dag(U, psi, alpha, M5, mf, bc)) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_eofa_apply_parity(eofa, case):
    dims, Ls, alpha, M5, mf, bc = case
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 3)
    out = lat.eofa_apply(psi, alpha, M5, mf)
    assert _rel(out, dwf.deofa(U, psi, alpha, M5, mf, bc)) < 1e-12


def test_gauge_load_rejects_non_unitary(eofa):
    dims = (2, 2, 2, 2)
    U = inputs.gauge_field(dims, 0.5, 1)
    U[0, 0, 0, 1, 2] *= 1.001
    lat = eofa.Lattice(dims, 4)
    with pytest.raises(eofa.EOFAError) as ei:
        lat.gauge_load(U)
    assert ei.value.code == eofa.EINVAL
    U[0, 0, 0, 1, 2] = np.nan
    with pytest.raises(eofa.EOFAError):
        lat.gauge_load(U)


def test_bad_arguments(eofa):
    with pytest.raises(eofa.EOFAError):
        eofa.Lattice((3, 4, 4, 4), 8)
    with pytest.raises(eofa.EOFAError):
        eofa.Lattice((4, 4, 4, 4), 0)
    lat = eofa.Lattice((2, 2, 2, 2), 4)
    with pytest.raises(eofa.EOFAError):  # no gauge loaded
        lat.dwf_apply(np.zeros(lat.shape5, complex), 2.0, 1.8, 0.1)
    lat.gauge_load(inputs.gauge_field((2, 2, 2, 2), 0.3, 1))
    p = lat.solve_params(system=eofa.SYS_EOFA_L, m1=0.5, m2=0.2)
    with pytest.raises(eofa.EOFAError):
        lat.solve(np.ones(lat.shape5, complex), system=eofa.SYS_EOFA_L, m1=0.5, m2=0.2)
    del p


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 2e-6), (2, 2e-3)])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[5]])
def test_hop_kernel_each_precision(eofa, case, prec, tol):
    """Even-odd hop in FP64 / FP32 / FP16 storage against the oracle hop."""
    import torch
    dims, Ls, alpha, M5, mf, bc = case
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 4)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    par = (x + y + z + t) % 2
    for out_par in (0, 1):
        for dag in (0, 1):
            src = psi * (par == 1 - out_par)[None, :, :, :, :, None, None]
            ref = dwf.wilson_hop(U, src, bc, dagger=bool(dag)) * (par == out_par)[None, :, :, :, :, None, None]
            dev = torch.from_numpy(src.copy()).cuda()
            nb = lat.field_bytes(prec)
            ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
            od = torch.empty(nb, dtype=torch.uint8, device="cuda")
            oe = torch.zeros(nb, dtype=torch.uint8, device="cuda")
            oo = torch.zeros(nb, dtype=torch.uint8, device="cuda")
            lat.pack_dev(prec, dev, ev, od)
            if out_par == 0:
                lat.hop_dev(prec, 0, dag, od, oe)
                lat.pack_dev(prec, torch.zeros_like(dev), ev, oo)
            else:
                lat.hop_dev(prec, 1, dag, ev, oo)
                lat.pack_dev(prec, torch.zeros_like(dev), oe, od)
            res = torch.empty_like(dev)
            lat.unpack_dev(prec, oe, oo, res)
            torch.cuda.synchronize()
            got = res.cpu().numpy()
            assert _rel(got, ref) < tol, (out_par, dag, _rel(got, ref))


def _ginv_blocks(Ls, alpha, M5, mf):
    """Dense per-chirality G^{-1} with G = (4 - M5) + D^perp, the 5D-local block of D_EOFA (Eq. (3))."""
    Pp, Pm = dwf.dperp_matrices(Ls, alpha, mf)
    one = np.eye(Ls)
    return np.linalg.inv((4 - M5) * one + Pp), np.linalg.inv((4 - M5) * one + Pm)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6), (2, 3e-3)])
@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3], CASES[5], ((4, 4, 2, 2), 16, 2.0, 1.8, 0.1, -1),
                                  ((2, 2, 2, 4), 24, 4.0, 1.8, 0.0362, -1)])
def test_schur_hop_parity(eofa, case, prec, tol):
    """Fused G^{-1} D_hop (and G^{-T} D_hop^+) against the oracle hop and dense 5D blocks."""
    import torch
    dims, Ls, alpha, M5, mf, bc = case
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 6)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    par = (x + y + z + t) % 2
    Gp, Gm = _ginv_blocks(Ls, alpha, M5, mf)
    nb = lat.field_bytes(prec)
    for out_par in (0, 1):
        for dag in (0, 1):
            src = psi * (par == 1 - out_par)[None, :, :, :, :, None, None]
            hop = dwf.wilson_hop(U, src, bc, dagger=bool(dag))
            if dag:
                ref = dwf.apply_s(Gp.T, Gm.T, hop)
            else:
                ref = dwf.apply_s(Gp, Gm, hop)
            ref = ref * (par == out_par)[None, :, :, :, :, None, None]
            dev = torch.from_numpy(src.copy()).cuda()
            ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
            od = torch.empty_like(ev)
            out = torch.empty_like(ev)
            zero = torch.zeros_like(ev)
            lat.pack_dev(prec, dev, ev, od)
            lat.pack_dev(prec, torch.zeros_like(dev), zero, zero)
            lat.schur_hop_dev(prec, out_par, dag, od if out_par == 0 else ev, out, alpha, M5, mf)
            res = torch.empty_like(dev)
            if out_par == 0:
                lat.unpack_dev(prec, out, zero, res)
            else:
                lat.unpack_dev(prec, zero, out, res)
            torch.cuda.synchronize()
            got = res.cpu().numpy()
            assert _rel(got, ref) < tol, (out_par, dag, _rel(got, ref))


@pytest.mark.parametrize("cfg", ["2,1", "4,1", "8,1", "8,1,2", "5,1,3", "2,1,4", "10,1,3", "4,1,-2", "5,1,-3",
                                 "2,1,-2"])
def test_forced_dslash_configurations(eofa, cfg, monkeypatch):
    """Every configuration the autotuner may pick gives the same fused kernel
    result: direct kernel "NS,SPT", staged bulk-copy kernel "NS,SPT,depth",
    pipelined cp.async kernel "NS,SPT,-slots"; Vh = 96 leaves a ragged last
    tile for NS = 5 and 10."""
    import torch
    monkeypatch.setenv("EOFA_DSLASH_CONFIG", cfg)
    dims, Ls, alpha, M5, mf, bc = (4, 4, 2, 6), 24, 2.0, 1.8, 0.0362, -1
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 7)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    par = (x + y + z + t) % 2
    Gp, Gm = _ginv_blocks(Ls, alpha, M5, mf)
    for prec, tol in ((0, 1e-12), (1, 2e-6), (2, 3e-3)):
        nb = lat.field_bytes(prec)
        for schur in (False, True):
            src = psi * (par == 1)[None, :, :, :, :, None, None]
            ref = dwf.wilson_hop(U, src, bc)
            if schur:
                ref = dwf.apply_s(Gp, Gm, ref)
            ref = ref * (par == 0)[None, :, :, :, :, None, None]
            dev = torch.from_numpy(src.copy()).cuda()
            ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
            od = torch.empty_like(ev)
            out = torch.empty_like(ev)
            zero = torch.zeros_like(ev)
            lat.pack_dev(prec, dev, ev, od)
            lat.pack_dev(prec, torch.zeros_like(dev), zero, zero)
            if schur:
                lat.schur_hop_dev(prec, 0, 0, od, out, alpha, M5, mf)
            else:
                lat.hop_dev(prec, 0, 0, od, out)
            res = torch.empty_like(dev)
            lat.unpack_dev(prec, out, zero, res)
            torch.cuda.synchronize()
            assert _rel(res.cpu().numpy(), ref) < tol, (cfg, prec, schur)
    lat.check_device()  # no bounded wait of a staged launch ran out
    lat.close()


def test_staged_wait_runs_out_and_reports(eofa, monkeypatch):
    """Failure detection of the staged dslash without a GPU fault: with the
    EOFA_TEST_STALL hook its producer warp issues no copy, so the consumers'
    first bounded wait runs out (about a second), the launch finishes, and the
    host reads EOFA_ETIMEOUT; the context stays usable and the next launch is
    correct."""
    import torch
    monkeypatch.setenv("EOFA_DSLASH_CONFIG", "4,1,2")
    monkeypatch.setenv("EOFA_TEST_STALL", "1")
    dims, Ls, bc = (4, 4, 2, 6), 24, -1
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 7)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    par = (x + y + z + t) % 2
    src = psi * (par == 1)[None, :, :, :, :, None, None]
    ref = dwf.wilson_hop(U, src, bc) * (par == 0)[None, :, :, :, :, None, None]
    prec = 1
    nb = lat.field_bytes(prec)
    ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
    od, out = torch.empty_like(ev), torch.empty_like(ev)
    zero = torch.zeros_like(ev)
    lat.pack_dev(prec, torch.from_numpy(src.copy()).cuda(), ev, od)
    lat.pack_dev(prec, torch.zeros(lat.shape5, dtype=torch.complex128, device="cuda"), zero, zero)
    lat.hop_dev(prec, 0, 0, od, out)  # stalls
    with pytest.raises(eofa.EOFAError) as ei:
        lat.check_device()
    assert ei.value.code == eofa.ETIMEOUT
    lat.check_device()  # the flag was cleared
    lat.hop_dev(prec, 0, 0, od, out)
    res = torch.empty(lat.shape5, dtype=torch.complex128, device="cuda")
    lat.unpack_dev(prec, out, zero, res)
    lat.check_device()
    torch.cuda.synchronize()
    assert _rel(res.cpu().numpy(), ref) < 2e-6
    lat.close()


@pytest.mark.parametrize("cfg", ["4,1,2", "3,1,-2", "4,1,-3"])
@pytest.mark.parametrize("Ls", [5, 8, 12, 16])
def test_variant_kernels_every_ls(eofa, cfg, Ls, monkeypatch):
    """The staged and pipelined dslash variants at the other compile-time Ls
    extents (8, 12, 16) and the generic one (Ls = 5), both dagger and both
    output parities, against the oracle hop and dense 5D blocks.  Shapes a
    variant cannot take (FP16 staging needs Ls % 4 == 0) fall back to the
    direct kernel and must still agree."""
    import torch
    monkeypatch.setenv("EOFA_DSLASH_CONFIG", cfg)
    dims, alpha, M5, mf, bc = (4, 2, 2, 6), 2.0, 1.8, 0.1, -1
    lat, U = _setup(eofa, dims, Ls, bc)
    psi = inputs.fermion5d(dims, Ls, 8)
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in (T, Z, Y, X)], indexing="ij")
    par = (x + y + z + t) % 2
    Gp, Gm = _ginv_blocks(Ls, alpha, M5, mf)
    for prec, tol in ((0, 1e-12), (1, 2e-6), (2, 3e-3)):
        nb = lat.field_bytes(prec)
        for out_par in (0, 1):
            for dag in (0, 1):
                src = psi * (par == 1 - out_par)[None, :, :, :, :, None, None]
                hop = dwf.wilson_hop(U, src, bc, dagger=bool(dag))
                ref = dwf.apply_s(Gp.T, Gm.T, hop) if dag else dwf.apply_s(Gp, Gm, hop)
                ref = ref * (par == out_par)[None, :, :, :, :, None, None]
                dev = torch.from_numpy(src.copy()).cuda()
                ev = torch.empty(nb, dtype=torch.uint8, device="cuda")
                od, out = torch.empty_like(ev), torch.empty_like(ev)
                zero = torch.zeros_like(ev)
                lat.pack_dev(prec, dev, ev, od)
                lat.pack_dev(prec, torch.zeros_like(dev), zero, zero)
                lat.schur_hop_dev(prec, out_par, dag, od if out_par == 0 else ev, out, alpha, M5, mf)
                res = torch.empty_like(dev)
                if out_par == 0:
                    lat.unpack_dev(prec, out, zero, res)
                else:
                    lat.unpack_dev(prec, zero, out, res)
                torch.cuda.synchronize()
                assert _rel(res.cpu().numpy(), ref) < tol, (cfg, Ls, prec, out_par, dag)
    lat.check_device()
    lat.close()


def test_fp64_fma_probe_reports_a_plausible_rate(eofa):
    """eofa_probe_fp64_fma: a positive, finite FP64 rate below GB300's nominal FP64
    vector rate of ~1.3 TFLOP/s with headroom (it is a denominator of the FP64 hop)."""
    v = eofa.probe_fp64_fma()
    assert 0.05 < v < 5.0, v
