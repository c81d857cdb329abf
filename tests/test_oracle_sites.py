"""The oracle's single-site operator forms agree with the whole-lattice ones.

dwf.dwf_at and eofa.system_apply_at evaluate D_DWF (Eq. (3)) and the Eq. (8)
system at one 4D site from its neighbours; the GPU tests use them to check
solutions on lattices too large for whole-field numpy.  Here they are pinned
to the whole-field definitions, on both time boundary conditions and at the
lattice edges.
"""
import numpy as np
import pytest

from oracle import dwf, eofa
from paper_1611_00298_gb300 import inputs

SITES = [(0, 0, 0, 0), (3, 1, 1, 3), (2, 0, 1, 1), (3, 0, 1, 0)]


@pytest.mark.parametrize("bc", [-1, 1])
@pytest.mark.parametrize("Ls,alpha", [(5, 2.0), (4, 1.0)])
def test_dwf_at_matches_whole_field(bc, Ls, alpha):
    dims = (4, 2, 2, 4)
    U = inputs.gauge_field(dims, 0.6, 3)
    psi = inputs.fermion5d(dims, Ls, 1, stream=3)
    full = dwf.dwf(U, psi, alpha, 1.8, 0.1, bc)
    scale = np.abs(full).max()
    Lpsi = dwf.L_apply(psi, 0.1)
    for site in SITES:
        got = dwf.dwf_at(U, psi, alpha, 1.8, 0.1, bc, site)
        assert np.abs(got - full[(slice(None),) + site]).max() < 1e-14 * scale
        got2 = dwf.dwf_at(U, psi, alpha, 1.8, 0.1, bc, site, Lpsi=Lpsi)
        assert np.array_equal(got, got2)


@pytest.mark.parametrize("bc", [-1, 1])
@pytest.mark.parametrize("which,a", [("L", 0.0), ("R", -1.0), ("L", -0.3), ("R", -0.7)])
def test_system_apply_at_matches_whole_field(bc, which, a):
    dims, Ls = (4, 2, 2, 4), 6
    U = inputs.gauge_field(dims, 0.6, 4)
    psi = inputs.fermion5d(dims, Ls, 2, stream=5)
    full = eofa.system_apply(U, psi, 2.0, 1.8, 0.04, 0.6, which, a, bc)
    scale = np.abs(full).max()
    for site in SITES:
        got = eofa.system_apply_at(U, psi, 2.0, 1.8, 0.04, 0.6, which, a, bc, site)
        assert np.abs(got - full[(slice(None),) + site]).max() < 1e-14 * scale
    if a != 0.0:
        # the Delta term is really there: dropping it changes the result
        plain = eofa.system_apply_at(U, psi, 2.0, 1.8, 0.04, 0.6, which, 0.0, bc, SITES[1])
        assert np.abs(plain - full[(slice(None),) + SITES[1]]).max() > 1e-3 * scale
