"""Checkpoint files of a solver's state (pure functions; the solver reads and writes them).

Layout: an 8-byte little-endian header length, a JSON header (format tag, grid, layout,
time, step), the raw arrays in the solver's own layout (the state of every batch member,
then the Runge-Kutta register), and a CRC32 of everything before it.  A checkpoint is taken
between steps (the Runge-Kutta stage counter is zero), so resuming from it continues the run
bit for bit.
"""
import json
import struct
import zlib

import numpy as np

TAG = "sbp-checkpoint-1"


class CheckpointError(ValueError):
    """The file is not a checkpoint, is truncated or corrupted, or does not fit the grid."""


def pack(header, arrays):
    """Bytes of a checkpoint: header (JSON-serialisable dict) and a list of numpy arrays."""
    h = dict(header)
    h["tag"] = TAG
    h["arrays"] = [[str(a.dtype), int(a.size)] for a in arrays]
    hb = json.dumps(h, sort_keys=True).encode()
    body = struct.pack("<Q", len(hb)) + hb + b"".join(np.ascontiguousarray(a).tobytes() for a in arrays)
    return body + struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF)


def unpack(data):
    """(header, arrays) of checkpoint bytes; CheckpointError for anything that is not one."""
    if len(data) < 12:
        raise CheckpointError("checkpoint truncated (shorter than its framing)")
    body, (crc,) = data[:-4], struct.unpack("<I", data[-4:])
    if zlib.crc32(body) & 0xFFFFFFFF != crc:
        raise CheckpointError("checkpoint checksum mismatch (truncated or corrupted)")
    (n,) = struct.unpack("<Q", body[:8])
    if 8 + n > len(body):
        raise CheckpointError("checkpoint header runs past the end of the file")
    try:
        header = json.loads(body[8:8 + n])
    except ValueError as ex:
        raise CheckpointError(f"checkpoint header is not JSON: {ex}") from None
    if header.get("tag") != TAG:
        raise CheckpointError(f"not a checkpoint of this format (tag {header.get('tag')!r})")
    arrays, off = [], 8 + n
    for dt, size in header["arrays"]:
        nb = np.dtype(dt).itemsize * size
        if off + nb > len(body):
            raise CheckpointError("checkpoint arrays run past the end of the file")
        arrays.append(np.frombuffer(body, dtype=dt, count=size, offset=off).copy())
        off += nb
    if off != len(body):
        raise CheckpointError("checkpoint has trailing bytes")
    return header, arrays
