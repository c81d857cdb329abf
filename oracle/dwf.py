"""Plain FP64 definitions of the domain-wall operators (oracle; test infrastructure).

Paper: D. Murphy, "Domain Wall Fermion Simulations with the Exact One-Flavor
Algorithm", Lattice 2016, Sec. 2.

Fields (numpy complex128):
  U    (T, Z, Y, X, 4, 3, 3)      links U_mu(x), mu = x, y, z, t -> 0..3
  psi  (Ls, T, Z, Y, X, 4, 3)     5D fermion, spin then colour
  phi  (T, Z, Y, X, 4, 3)         4D fermion

Readings of what the paper leaves open (each is pinned by a test):
  * Euclidean chiral basis: gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] for
    k = 1, 2, 3, gamma_4 = [[0, 1], [1, 0]], gamma_5 = g1 g2 g3 g4 =
    diag(1, 1, -1, -1); P_pm = (1 pm gamma_5)/2.
  * D_w is the Wilson operator with domain-wall height M5 (Wilson mass -M5):
    D_w = (4 - M5) - 1/2 sum_mu [(1 - g_mu) U_mu(x) d_{x+mu,y}
                                 + (1 + g_mu) U_mu(x-mu)^+ d_{x-mu,y}].
  * Boundary conditions: periodic in x, y, z; the t-links from T-1 to 0
    carry the phase bc_t (+1 periodic, -1 antiperiodic).
  * L = P_+ L_+ + P_- L_-, with (L_+)_{s,s-1} = 1 for s >= 1,
    (L_+)_{0,Ls-1} = -m_f and L_- = L_+^T.  This is the sign for which the
    closed form Eq. (4) holds.
  * Eq. (3) with c = alpha/2, d = 1/2:
    D_DWF = ((c+d) D_w + 1) delta_{ss'} + ((c-d) D_w - 1) L_{ss'}, the
    D_w factor acting after L.
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- spin algebra

_SIGMA = np.array([[[0, 1], [1, 0]],
                   [[0, -1j], [1j, 0]],
                   [[1, 0], [0, -1]]], dtype=np.complex128)


def gammas() -> np.ndarray:
    """gamma_mu for mu = x, y, z, t in the chiral basis; shape (4, 4, 4)."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z2 = np.zeros((2, 2))
    for k in range(3):
        g[k] = np.block([[z2, -1j * _SIGMA[k]], [1j * _SIGMA[k], z2]])
    g[3] = np.block([[z2, np.eye(2)], [np.eye(2), z2]])
    return g


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
P_PLUS = 0.5 * (np.eye(4) + GAMMA5)
P_MINUS = 0.5 * (np.eye(4) - GAMMA5)

# axis of direction mu in a (..., T, Z, Y, X, <2 trailing>) array
_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}


def spin_mul(S: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to (..., 4, 3)."""
    return np.einsum("st,...tc->...sc", S, psi)


def colour_mul(Um: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply site-dependent 3x3 matrices (T,Z,Y,X,3,3) to (..., T,Z,Y,X,4,3)."""
    return np.einsum("...ab,...sb->...sa", Um, psi)


def dagger3(Um: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(Um, -1, -2))


def shift(f: np.ndarray, mu: int, sign: int, bc_t: float) -> np.ndarray:
    """g(x) = f(x + sign*mu) with the t-boundary phase on wrapped entries."""
    ax = _AXIS[mu]
    g = np.roll(f, -sign, axis=ax)
    if mu == 3 and bc_t != 1:
        idx = [slice(None)] * g.ndim
        idx[ax] = -1 if sign > 0 else 0
        g[tuple(idx)] *= bc_t
    return g


def shift_links(Um: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """Um(x + sign*mu) for a (T,Z,Y,X,3,3) array (no phase)."""
    return np.roll(Um, -sign, axis=_AXIS[mu])


# ---------------------------------------------------------------- Wilson D_w

def wilson_hop(U: np.ndarray, psi: np.ndarray, bc_t: float, dagger: bool = False) -> np.ndarray:
    """-1/2 sum_mu [(1 -+ g_mu) U_mu(x) psi(x+mu) + (1 +- g_mu) U_mu(x-mu)^+ psi(x-mu)].

    The hopping part of D_w (Sec. 2, symbol D_w in Eq. (3)); ``dagger`` gives
    the hopping part of D_w^+, which swaps the two projectors.
    """
    sgn = -1.0 if dagger else 1.0
    out = np.zeros_like(psi)
    one = np.eye(4)
    for mu in range(4):
        Um = U[..., mu, :, :]
        fwd = colour_mul(Um, shift(psi, mu, +1, bc_t))
        Ub = dagger3(shift_links(Um, mu, -1))
        bwd = colour_mul(Ub, shift(psi, mu, -1, bc_t))
        out -= 0.5 * (spin_mul(one - sgn * GAMMA[mu], fwd) + spin_mul(one + sgn * GAMMA[mu], bwd))
    return out


def wilson(U, psi, M5, bc_t, dagger=False):
    """D_w psi (or D_w^+ psi) on every s-slice; Sec. 2, the D_w of Eq. (3)."""
    return (4.0 - M5) * psi + wilson_hop(U, psi, bc_t, dagger)


# ---------------------------------------------------------------- fifth dimension

def coefficients(alpha: float):
    """Moebius weights of Eq. (3): c = alpha/2, d = 1/2; returns (c, d)."""
    return 0.5 * alpha, 0.5


def L_matrices(Ls: int, mf: float):
    """(L_+, L_-) as dense Ls x Ls real matrices (the 5D hopping of Eq. (3))."""
    Lp = np.zeros((Ls, Ls))
    for s in range(1, Ls):
        Lp[s, s - 1] = 1.0
    Lp[0, Ls - 1] += -mf
    return Lp, Lp.T.copy()


def apply_s(Mp: np.ndarray, Mm: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """P_+ (Mp psi) + P_- (Mm psi) for Ls x Ls matrices acting on the s index."""
    a = np.einsum("st,t...->s...", Mp, psi)
    b = np.einsum("st,t...->s...", Mm, psi)
    return spin_mul(P_PLUS, a) + spin_mul(P_MINUS, b)


def L_apply(psi, mf):
    Lp, Lm = L_matrices(psi.shape[0], mf)
    return apply_s(Lp, Lm, psi)


def L_dag_apply(psi, mf):
    Lp, Lm = L_matrices(psi.shape[0], mf)
    return apply_s(Lp.T, Lm.T, psi)


def R5(psi):
    """(R_5)_{ss'} = delta_{s, Ls-1-s'} (Sec. 2)."""
    return psi[::-1].copy()


def gamma5(psi):
    return spin_mul(GAMMA5, psi)


# ---------------------------------------------------------------- Eq. (3)

def dwf(U, psi, alpha, M5, mf, bc_t):
    """D_DWF psi, first line of Eq. (3)."""
    c, d = coefficients(alpha)
    Lpsi = L_apply(psi, mf)
    return ((c + d) * wilson(U, psi, M5, bc_t) + psi) + ((c - d) * wilson(U, Lpsi, M5, bc_t) - Lpsi)


def dwf_dag(U, psi, alpha, M5, mf, bc_t):
    """D_DWF^+ psi: the adjoint of the first line of Eq. (3).

    D_DWF = ((c+d) D_w + 1) + ((c-d) D_w - 1) L, so
    D_DWF^+ = ((c+d) D_w^+ + 1) + L^+ ((c-d) D_w^+ - 1).
    """
    c, d = coefficients(alpha)
    Dd = wilson(U, psi, M5, bc_t, dagger=True)
    return ((c + d) * Dd + psi) + L_dag_apply((c - d) * Dd - psi, mf)


def dtilde_matrices(Ls, alpha, mf):
    """Per-chirality Ls x Ls blocks of D-tilde = d(1 - L) + c(1 + L), Eq. (3)."""
    c, d = coefficients(alpha)
    one = np.eye(Ls)
    Lp, Lm = L_matrices(Ls, mf)
    return d * (one - Lp) + c * (one + Lp), d * (one - Lm) + c * (one + Lm)


def dtilde(psi, alpha, mf):
    """D-tilde psi, the right factor of Eq. (3)."""
    Tp, Tm = dtilde_matrices(psi.shape[0], alpha, mf)
    return apply_s(Tp, Tm, psi)


def dperp_matrices(Ls, alpha, mf):
    """Per-chirality blocks of D^perp = (1 - L) D-tilde^{-1} (Eq. (3))."""
    Tp, Tm = dtilde_matrices(Ls, alpha, mf)
    Lp, Lm = L_matrices(Ls, mf)
    one = np.eye(Ls)
    return (one - Lp) @ np.linalg.inv(Tp), (one - Lm) @ np.linalg.inv(Tm)


def deofa(U, psi, alpha, M5, mf, bc_t):
    """D_EOFA psi = D_w psi + D^perp psi, middle line of Eq. (3)."""
    Pp, Pm = dperp_matrices(psi.shape[0], alpha, mf)
    return wilson(U, psi, M5, bc_t) + apply_s(Pp, Pm, psi)


def hermitian_H(U, psi, alpha, M5, mf, bc_t):
    """H(m) = gamma_5 R_5 D_EOFA(m) (Sec. 2, after Eq. (4))."""
    return gamma5(R5(deofa(U, psi, alpha, M5, mf, bc_t)))


def wilson_hop_at(U, psi, site, s, bc_t, dagger=False):
    """The hopping part of D_w at one output site (t, z, y, x) = site and slice s.

    Same definition as wilson_hop, evaluated from the eight neighbours only,
    for checking kernels on lattices too large for whole-field numpy.
    """
    sgn = -1.0 if dagger else 1.0
    dims = U.shape[:4]
    one = np.eye(4)
    out = np.zeros((4, 3), dtype=np.complex128)
    for mu in range(4):
        axis = {0: 3, 1: 2, 2: 1, 3: 0}[mu]
        fwd, bwd = list(site), list(site)
        fwd[axis] += 1
        bwd[axis] -= 1
        pf = pb = 1.0
        if fwd[axis] == dims[axis]:
            fwd[axis] = 0
            pf = bc_t if mu == 3 else 1.0
        if bwd[axis] < 0:
            bwd[axis] = dims[axis] - 1
            pb = bc_t if mu == 3 else 1.0
        fwd, bwd = tuple(fwd), tuple(bwd)
        Uf = U[site + (mu,)]
        Ub = U[bwd + (mu,)]
        vf = pf * (psi[s][fwd] @ Uf.T)                 # U_mu(x) psi(x + mu), colour on the right index
        vb = pb * (psi[s][bwd] @ np.conj(Ub))          # U_mu(x - mu)^+ psi(x - mu)
        out -= 0.5 * ((one - sgn * GAMMA[mu]) @ vf + (one + sgn * GAMMA[mu]) @ vb)
    return out


def _site_slab(psi, site):
    """psi at one 4D site for every s, keeping singleton lattice axes: (Ls, 1, 1, 1, 1, 4, 3)."""
    t, z, y, x = site
    return psi[:, t:t + 1, z:z + 1, y:y + 1, x:x + 1]


def wilson_at(U, psi, M5, site, bc_t):
    """D_w psi at one 4D site for every s: (4 - M5) psi + the hop (Sec. 2), shape (Ls, 4, 3)."""
    Ls = psi.shape[0]
    t, z, y, x = site
    return np.stack([(4.0 - M5) * psi[s, t, z, y, x] + wilson_hop_at(U, psi, site, s, bc_t) for s in range(Ls)])


def dwf_at(U, psi, alpha, M5, mf, bc_t, site, Lpsi=None):
    """(D_DWF psi) at one 4D site for every s, the first line of Eq. (3) evaluated
    from that site's neighbours only; shape (Ls, 4, 3).  Lpsi = L psi on the
    whole lattice may be passed in (it is site-local in 4D and reused across
    sites)."""
    c, d = coefficients(alpha)
    if Lpsi is None:
        Lpsi = L_apply(psi, mf)
    t, z, y, x = site
    return ((c + d) * wilson_at(U, psi, M5, site, bc_t) + psi[:, t, z, y, x]
            + (c - d) * wilson_at(U, Lpsi, M5, site, bc_t) - Lpsi[:, t, z, y, x])
