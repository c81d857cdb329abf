"""CPU oracle for the EOFA / Moebius domain-wall hot path (FP64, numpy).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA path is checked against.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product library never
does, and it shares no code with the CUDA path.

Every operator is written as its plain definition from D. Murphy, "Domain Wall
Fermion Simulations with the Exact One-Flavor Algorithm" (Lattice 2016):
Sec. 2 Eq. (3) for D_DWF, D_EOFA and D-tilde, Eq. (4) for det D-tilde,
Eq. (5) for the EOFA action, Eq. (6) for the heatbath, Eq. (7) for the force
and Eq. (8) for the EOFA linear systems; ``gauge.py`` adds the Wilson gauge
action and the force-gradient integrators of the HMC runs of Sec. 5.  Conventions the paper leaves open (gamma basis, boundary
conditions, the sign of the m_f corner of L, the su(3) generator
normalisation, the scale of Omega) are fixed in ``dwf.py`` and documented
there; every function cites the equation it follows.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
something other than itself (momentum-space closed forms, dense determinants,
the Eq. (1) determinant identity, Hermiticity, gauge covariance, finite
differences, dense rational functions of M_EOFA, integrator orders).
Nothing in this package is "parity unpinned".
"""
from . import dwf, solve, eofa, gauge  # noqa: F401
