"""The checkpoint file format (pure functions, CPU): round trip, and the documented error
for a truncated, corrupted or foreign file."""
import numpy as np
import pytest

from paper_2011_02600_gb300 import checkpoint as ck


def _data():
    rng = np.random.default_rng(0)
    arrays = [rng.normal(size=1000).astype(np.float32), rng.normal(size=1000)]
    return ck.pack(dict(nodes=[10, 10, 10], order=4, time=1.25, step=7), arrays), arrays


def test_round_trip_is_exact():
    data, arrays = _data()
    header, got = ck.unpack(data)
    assert header["order"] == 4 and header["time"] == 1.25 and header["step"] == 7
    for a, b in zip(arrays, got):
        assert a.dtype == b.dtype and np.array_equal(a, b)


@pytest.mark.parametrize("cut", [0, 5, 11, 100, -1, -5])
def test_truncated_file_is_rejected(cut):
    data, _ = _data()
    with pytest.raises(ck.CheckpointError):
        ck.unpack(data[:cut] if cut >= 0 else data[:len(data) + cut])


def test_corrupted_byte_is_rejected():
    data, _ = _data()
    bad = bytearray(data)
    bad[len(bad) // 2] ^= 0x40
    with pytest.raises(ck.CheckpointError, match="checksum"):
        ck.unpack(bytes(bad))


def test_foreign_file_is_rejected():
    import struct
    import zlib
    hb = b'{"tag": "something-else", "arrays": []}'
    body = struct.pack("<Q", len(hb)) + hb
    with pytest.raises(ck.CheckpointError, match="format"):
        ck.unpack(body + struct.pack("<I", zlib.crc32(body)))
