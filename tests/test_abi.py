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
