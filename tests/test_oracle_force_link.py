"""The single-link force of the oracle agrees with the whole-lattice one."""
import numpy as np

from oracle import eofa
from paper_1611_00298_gb300 import inputs


def test_force_at_link_matches_force_from_chi():
    dims, Ls = (2, 2, 2, 4), 4
    U = inputs.gauge_field(dims, 0.6, 3)
    chiL = inputs.fermion5d(dims, Ls, 1, stream=21)
    chiR = inputs.fermion5d(dims, Ls, 1, stream=22)
    for bc in (-1, 1):
        F, _ = eofa.force_from_chi(U, chiL, chiR, 0.7, bc)
        rng = np.random.default_rng(0)
        for _ in range(6):
            site = (int(rng.integers(4)), int(rng.integers(2)), int(rng.integers(2)), int(rng.integers(2)))
            mu = int(rng.integers(4))
            Fl = eofa.force_at_link(U, chiL, chiR, 0.7, bc, site, mu)
            assert np.abs(Fl - F[site + (mu,)]).max() < 1e-13 * max(1.0, np.abs(F).max())
        # the t-boundary links
        for site in ((3, 0, 1, 0), (3, 1, 0, 1)):
            Fl = eofa.force_at_link(U, chiL, chiR, 0.7, bc, site, 3)
            assert np.abs(Fl - F[site + (3,)]).max() < 1e-13 * max(1.0, np.abs(F).max())
