"""The C-ABI library builds, loads and exports every symbol include/eofa.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1611_00298_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "eofa.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(eofa_\w+)\s*\(", src, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("eofa_gauge_load", "eofa_dwf_apply", "eofa_solve", "eofa_action", "eofa_force"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header(libpath):
    from paper_1611_00298_gb300 import eofa
    assert sorted(eofa.EXPORTS) == _declared()
    eofa.load_library(libpath)


def test_coefficients_without_gpu(libpath):
    # eofa_coefficients is host-only: compare with the closed forms of the oracle
    import numpy as np
    from oracle import eofa as oeofa
    from paper_1611_00298_gb300 import eofa
    for alpha, Ls in ((2.0, 8), (1.0, 12), (4.0, 24)):
        k, Op, Om = eofa.coefficients(Ls, alpha, 0.0362, 1.0)
        Op2, Om2 = oeofa.omega(Ls, alpha)
        assert np.isclose(k, oeofa.k_coefficient(Ls, alpha, 0.0362, 1.0), rtol=1e-14)
        assert np.allclose(Op, Op2, rtol=1e-14) and np.allclose(Om, Om2, rtol=1e-14)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1611_00298_gb300 import eofa
    saved = eofa._lib
    eofa._lib = None
    try:
        with pytest.raises(RuntimeError):
            eofa.load_library(str(tmp_path / "nope.so"))
    finally:
        eofa._lib = saved


def test_create_without_gpu_reports_error(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1611_00298_gb300 import eofa
    with pytest.raises(eofa.EOFAError):
        eofa.Lattice((4, 4, 4, 4), 8)


@pytest.mark.parametrize("n,lmin,lmax", [(4, 0.1, 2.0), (8, 1e-3, 10.0), (12, 1e-4, 50.0)])
def test_rational_inv_sqrt_is_minimax(libpath, n, lmin, lmax):
    """Host-only Zolotarev coefficients (Sec. 3.2): the relative error of
    alpha0 + sum alpha/(x + beta) against x^-1/2 stays within the reported
    bound and equioscillates at 2n + 2 extrema (Chebyshev's alternation
    theorem for the optimal (n, n) approximant)."""
    import numpy as np
    from paper_1611_00298_gb300 import eofa
    eofa.load_library(libpath)
    a0, al, be, err = eofa.rational_inv_sqrt(n, lmin, lmax)
    assert np.all(be > 0) and np.all(al > 0) and a0 > 0
    x = np.exp(np.linspace(np.log(lmin), np.log(lmax), 200001))
    f = a0 + (al[None, :] / (x[:, None] + be[None, :])).sum(1)
    e = f * np.sqrt(x) - 1.0
    assert np.abs(e).max() < err * (1 + 1e-6) + 1e-14
    assert np.abs(e).max() > err * (1 - 1e-3)
    # sign alternations between successive near-extremal points
    ext = np.flatnonzero(np.abs(e) > 0.999 * err)
    groups = np.split(ext, np.flatnonzero(np.diff(ext) > 1) + 1)
    signs = [np.sign(e[g[np.argmax(np.abs(e[g]))]]) for g in groups]
    assert len(signs) == 2 * n + 2
    assert all(signs[i] != signs[i + 1] for i in range(len(signs) - 1))


def test_rational_inv_sqrt_error_shrinks_with_poles(libpath):
    from paper_1611_00298_gb300 import eofa
    eofa.load_library(libpath)
    errs = [eofa.rational_inv_sqrt(n, 1e-3, 10.0)[3] for n in (2, 4, 8, 16)]
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(3))
    assert eofa.rational_inv_sqrt(16, 1e-3, 10.0)[3] < 1e-10


def test_check_device_rejects_null_context(libpath):
    from paper_1611_00298_gb300 import eofa
    lib = eofa.load_library(libpath)
    assert lib.eofa_check_device(None, None) == eofa.EINVAL


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of
    its C struct in include/eofa.h (compiled here with the host C compiler),
    so that a field added on one side only is caught without a GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1611_00298_gb300 import eofa as e
    pairs = {"eofa_solve_params": e.SolveParams, "eofa_solve_info": e.SolveInfo, "eofa_md_params": e.MDParams,
             "eofa_md_info": e.MDInfo, "eofa_hmc_traj_info": e.HMCTrajInfo, "eofa_profile": e.Profile}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "eofa.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
