"""Checkpoint files of the gauge field and the momenta (host-only library calls,
no GPU): round trips are bit-exact, the header holds what it states and the
FNV-1a checksum of the data, and every damaged or mismatched file is refused."""
import struct

import numpy as np
import pytest

from paper_1611_00298_gb300 import inputs


@pytest.fixture(scope="module")
def eofa():
    from paper_1611_00298_gb300 import build
    from paper_1611_00298_gb300 import eofa as e
    e.load_library(build.build())
    return e


def _fnv1a64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h ^= b
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


DIMS = (4, 2, 2, 6)


def test_round_trip_and_header(eofa, tmp_path):
    U = inputs.gauge_field(DIMS, 0.5, 3)
    P = inputs.momenta(DIMS, 4)
    pu, pp = tmp_path / "u.ckpt", tmp_path / "p.ckpt"
    eofa.checkpoint_write(pu, eofa.CKPT_GAUGE, U, traj=17)
    eofa.checkpoint_write(pp, eofa.CKPT_MOMENTA, P, traj=-3)
    U2, t2 = eofa.checkpoint_read(pu, eofa.CKPT_GAUGE, DIMS)
    P2, t3 = eofa.checkpoint_read(pp, eofa.CKPT_MOMENTA, DIMS)
    assert np.array_equal(U2, U) and t2 == 17
    assert np.array_equal(P2, P) and t3 == -3
    raw = pu.read_bytes()
    magic, version, kind, X, Y, Z, T, n, traj, cks, res = struct.unpack("<8sII4iQqQQ", raw[:64])
    assert magic == b"EOFACKPT" and version == 1 and kind == eofa.CKPT_GAUGE
    assert (X, Y, Z, T) == DIMS and n == 72 * np.prod(DIMS) and traj == 17 and res == 0
    data = raw[64:]
    assert len(data) == 8 * n
    assert cks == _fnv1a64(data)
    assert np.array_equal(np.frombuffer(data, dtype=np.complex128), U.reshape(-1))


def test_damaged_or_mismatched_files_are_refused(eofa, tmp_path):
    U = inputs.gauge_field(DIMS, 0.5, 3)
    good = tmp_path / "u.ckpt"
    eofa.checkpoint_write(good, eofa.CKPT_GAUGE, U, traj=1)
    raw = bytearray(good.read_bytes())
    cases = {}
    flipped = bytearray(raw)
    flipped[64 + 1000] ^= 0x01
    cases["flipped data bit"] = bytes(flipped)
    cases["truncated"] = bytes(raw[:-8])
    cases["trailing byte"] = bytes(raw) + b"\0"
    badmagic = bytearray(raw)
    badmagic[0:1] = b"X"
    cases["magic"] = bytes(badmagic)
    for name, content in cases.items():
        p = tmp_path / (name.replace(" ", "_") + ".ckpt")
        p.write_bytes(content)
        with pytest.raises(eofa.EOFAError) as ei:
            eofa.checkpoint_read(p, eofa.CKPT_GAUGE, DIMS)
        assert ei.value.code == eofa.EINVAL, name
    with pytest.raises(eofa.EOFAError):
        eofa.checkpoint_read(good, eofa.CKPT_MOMENTA, DIMS)          # another kind
    with pytest.raises(eofa.EOFAError):
        eofa.checkpoint_read(good, eofa.CKPT_GAUGE, (4, 2, 2, 4))    # another lattice
    with pytest.raises(eofa.EOFAError):
        eofa.checkpoint_read(tmp_path / "missing.ckpt", eofa.CKPT_GAUGE, DIMS)
    with pytest.raises(eofa.EOFAError):
        eofa.checkpoint_write(tmp_path / "no" / "dir" / "x.ckpt", eofa.CKPT_GAUGE, U)
