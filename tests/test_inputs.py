"""Pins of the seeded input generators (SplitMix64, Box-Muller, SU(3) links)."""
import numpy as np

from paper_1611_00298_gb300 import inputs


def test_splitmix64_published_sequence():
    # SplitMix64 started from state 0: the first outputs of the published
    # generator (Steele, Lea, Flood 2014; Vigna's reference splitmix64.c).
    out = [int(v) for v in inputs.splitmix64(0, 3)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_offsets_are_counter_based():
    full = inputs.splitmix64(12345, 10)
    tail = inputs.splitmix64(12345, 4, offset=6)
    assert np.array_equal(full[6:], tail)


def test_box_muller_moments():
    g = inputs.normal(inputs.stream_key(9, 1), 400_000)
    assert abs(g.mean()) < 5e-3
    assert abs(g.var() - 1.0) < 1e-2
    assert abs(np.mean(g ** 4) - 3.0) < 5e-2  # Gaussian kurtosis


def test_normal_range_matches_normal():
    key = inputs.stream_key(3, 7)
    a = inputs.normal(key, 100)
    b = inputs.normal_range(key, 40, 30)
    assert np.array_equal(a[40:70], b)


def test_gauge_field_is_su3_and_seeded():
    dims = (4, 2, 2, 4)
    U = inputs.gauge_field(dims, 0.6, 2)
    assert U.shape == (4, 2, 2, 4, 4, 3, 3)
    UdU = np.einsum("...ji,...jk->...ik", np.conj(U), U)
    assert np.abs(UdU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    assert np.array_equal(U, inputs.gauge_field(dims, 0.6, 2))
    assert not np.allclose(U, inputs.gauge_field(dims, 0.6, 3))


def test_gauge_field_eps_zero_is_unit():
    U = inputs.gauge_field((2, 2, 2, 2), 0.0, 1)
    assert np.abs(U - np.eye(3)).max() < 1e-15


def test_gauge_field_chunking_invariant():
    dims = (4, 4, 2, 2)
    a = inputs.gauge_field(dims, 0.5, 4, chunk=1 << 18)
    b = inputs.gauge_field(dims, 0.5, 4, chunk=7)
    assert np.array_equal(a, b)


def test_gell_mann_algebra():
    lam = inputs.gell_mann()
    tr = np.einsum("aij,bji->ab", lam, lam)
    assert np.allclose(tr, 2 * np.eye(8))
    assert np.allclose(np.einsum("aii->a", lam), 0)
