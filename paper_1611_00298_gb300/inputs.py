"""Seeded synthetic inputs: gauge fields, 5D sources and 4D pseudofermions.

This module only draws random numbers and builds input fields.  It holds none
of the Dirac-operator, solver, action or force arithmetic, so that both the
CUDA path and the CPU oracle can be fed the very same arrays.

Random numbers
--------------
A counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the n-th 64-bit output of the
stream with key ``k`` is ``mix64(k + (n + 1) * 0x9E3779B97F4A7C15)`` with the
published finaliser ``mix64``.  Uniforms take the top 53 bits; normals come in
pairs from the Box-Muller transform.  Draws run in lexicographic site order
(i = x + X(y + Y(z + Z t))), then direction mu, then generator index a.

Canonical host layouts (complex128, interleaved re/im in memory)
------------------------------------------------------------------
* gauge   U[t, z, y, x, mu, a, b]          (mu = x, y, z, t -> 0..3)
* 5D field psi[s, t, z, y, x, spin, colour]
* 4D field phi[t, z, y, x, spin, colour]

Synthetic gauge links follow the workload recipe of the paper's ensembles
(Sec. 3, Table 1 shapes): U = exp(i eps sum_a h_a lambda_a) with h_a ~ N(0,1)
and Gell-Mann lambda_a, then reunitarised (Gram-Schmidt of rows 0 and 1, row 2
= conj(row0 x row1)).  Sources are complex Gaussian with re, im ~ N(0,1).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of an independent stream, derived from (seed, stream)."""
    z = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019)
                  & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return int(_mix64(z)[0])


def splitmix64(key: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 sequence started at state ``key``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        state = np.uint64(key) + ctr * _GOLDEN
        return _mix64(state)


def uniform(key: int, n: int) -> np.ndarray:
    """n uniforms in [0, 1) from the top 53 bits of each output."""
    return (splitmix64(key, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(key: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(key, 2 * m).reshape(m, 2)
    rad = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((m, 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)[:n]


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0, 0, 1] = lam[0, 1, 0] = 1
    lam[1, 0, 1] = -1j
    lam[1, 1, 0] = 1j
    lam[2, 0, 0] = 1
    lam[2, 1, 1] = -1
    lam[3, 0, 2] = lam[3, 2, 0] = 1
    lam[4, 0, 2] = -1j
    lam[4, 2, 0] = 1j
    lam[5, 1, 2] = lam[5, 2, 1] = 1
    lam[6, 1, 2] = -1j
    lam[6, 2, 1] = 1j
    lam[7, 0, 0] = lam[7, 1, 1] = 1 / np.sqrt(3)
    lam[7, 2, 2] = -2 / np.sqrt(3)
    return lam


def reunitarise(U: np.ndarray) -> np.ndarray:
    """Project (..., 3, 3) matrices onto SU(3): Gram-Schmidt rows 0, 1; row 2 = conj(r0 x r1)."""
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _exp_i_hermitian(Hm: np.ndarray) -> np.ndarray:
    w, v = np.linalg.eigh(Hm)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * w), np.conj(v))


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 18) -> np.ndarray:
    """Synthetic SU(3) gauge field, shape (T, Z, Y, X, 4, 3, 3).

    dims = (X, Y, Z, T).  Links are exp(i eps sum_a h_a lambda_a), reunitarised.
    eps = 0 gives the unit (free) field.
    """
    X, Y, Z, T = dims
    V = X * Y * Z * T
    key = stream_key(seed, 0)
    lam = gell_mann()
    U = np.empty((V * 4, 3, 3), dtype=np.complex128)
    nlinks = V * 4
    for start in range(0, nlinks, chunk):
        stop = min(nlinks, start + chunk)
        h = normal_range(key, 8 * start, 8 * (stop - start)).reshape(stop - start, 8)
        Hm = eps * np.einsum("la,aij->lij", h, lam)
        U[start:stop] = reunitarise(_exp_i_hermitian(Hm))
    return U.reshape(T, Z, Y, X, 4, 3, 3)


def normal_range(key: int, first: int, n: int) -> np.ndarray:
    """Normals first .. first+n-1 of stream ``key`` (first must be even)."""
    assert first % 2 == 0
    m = (n + 1) // 2
    raw = splitmix64(key, 2 * m, offset=first)
    u = (raw >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    u = u.reshape(m, 2)
    rad = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((m, 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    return out.reshape(-1)[:n]


def fermion5d(dims, Ls: int, seed: int, stream: int = 1) -> np.ndarray:
    """Complex Gaussian 5D field, shape (Ls, T, Z, Y, X, 4, 3)."""
    X, Y, Z, T = dims
    n = Ls * X * Y * Z * T * 12
    g = normal(stream_key(seed, stream), 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(Ls, T, Z, Y, X, 4, 3)


def fermion4d(dims, seed: int, stream: int = 2) -> np.ndarray:
    """Complex Gaussian 4D pseudofermion field, shape (T, Z, Y, X, 4, 3)."""
    X, Y, Z, T = dims
    n = X * Y * Z * T * 12
    g = normal(stream_key(seed, stream), 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(T, Z, Y, X, 4, 3)


def gauge_transform(dims, seed: int, stream: int = 3) -> np.ndarray:
    """Random site-local SU(3) matrices g(x), shape (T, Z, Y, X, 3, 3)."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    h = normal(stream_key(seed, stream), 8 * V).reshape(V, 8)
    Hm = np.einsum("la,aij->lij", h, gell_mann())
    return reunitarise(_exp_i_hermitian(Hm)).reshape(T, Z, Y, X, 3, 3)


def momenta(dims, seed: int, stream: int = 4) -> np.ndarray:
    """Gaussian su(3) momenta P = sum_a p_a lambda_a / 2, p_a ~ N(0,1); (T,Z,Y,X,4,3,3)."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    p = normal(stream_key(seed, stream), 8 * 4 * V).reshape(V * 4, 8)
    P = 0.5 * np.einsum("la,aij->lij", p, gell_mann())
    return P.reshape(T, Z, Y, X, 4, 3, 3)
