"""The tcgen05 GEMM's descriptors on the CPU (csrc/umma_desc.h compiled as host C++).

1. Packing: every field of the shared-memory matrix descriptor and of the kind::f16 instruction
   descriptor lands at the bit position and width of the PTX ISA's field tables, written out
   separately here.
2. Layout: the address at which the descriptors (start address, leading and stride byte offsets,
   the per-16-k advance) place each element of an operand tile, under the canonical layouts of
   128-byte swizzled K-major and MN-major operands, is the address at which a 2D TMA load with
   128-byte swizzling writes that element (the XOR of address bits 4-6 with bits 7-9 inside each
   1 KB block), for whole 128 x 64 and 256 x 64 tiles in both orientations."""
import ctypes

import pytest

from host_build import build

# (name, lowest bit, width) of the shared-memory matrix descriptor
SMEM_FIELDS = [("start", 0, 14), ("lbo", 16, 14), ("sbo", 32, 14), ("fixed", 46, 3), ("base_offset", 49, 3),
               ("lbo_mode", 52, 1), ("swizzle", 61, 3)]
# (name, lowest bit, width) of the instruction descriptor, .kind::f16
INSTR_FIELDS = [("sparse_sel", 0, 2), ("sparse", 2, 1), ("saturate", 3, 1), ("d_fmt", 4, 2), ("a_fmt", 7, 3),
                ("b_fmt", 10, 3), ("neg_a", 13, 1), ("neg_b", 14, 1), ("a_major", 15, 1), ("b_major", 16, 1),
                ("n", 17, 6), ("m", 24, 5), ("max_shift", 30, 2)]


def pack(fields, values):
    out = 0
    for name, lo, width in fields:
        v = values.get(name, 0)
        assert 0 <= v < (1 << width), name
        out |= v << lo
    return out


@pytest.fixture(scope="module")
def umma(tmp_path_factory):
    lib = ctypes.CDLL(build("host_umma.cpp", tmp_path_factory.mktemp("umma") / "libumma.so", shared=True))
    U32, I = ctypes.c_uint32, ctypes.c_int
    lib.host_smem_desc.argtypes = [U32] * 4
    lib.host_smem_desc.restype = ctypes.c_uint64
    lib.host_kmajor_desc.argtypes = [U32, I]
    lib.host_kmajor_desc.restype = ctypes.c_uint64
    lib.host_mnmajor_desc.argtypes = [U32, I]
    lib.host_mnmajor_desc.restype = ctypes.c_uint64
    lib.host_instr_desc.argtypes = [I] * 4
    lib.host_instr_desc.restype = ctypes.c_uint32
    return lib


def test_smem_descriptor_fields(umma):
    for addr, lbo, sbo, sw in [(0x400, 16, 1024, 2), (0x3FC00, 8192, 1024, 2), (0x12340, 256, 2048, 4),
                               (0x1000, 128, 128, 0), (0x2A00, 0x3FFF0, 0x3FFF0, 6)]:
        want = pack(SMEM_FIELDS, dict(start=(addr & 0x3FFFF) >> 4, lbo=lbo >> 4, sbo=sbo >> 4, fixed=1, swizzle=sw))
        assert umma.host_smem_desc(addr, lbo, sbo, sw) == want


def test_instruction_descriptor_fields(umma):
    for M, N, amn, bmn in [(128, 256, 0, 0), (128, 256, 1, 0), (128, 256, 0, 1), (128, 256, 1, 1), (64, 8, 0, 0),
                           (128, 16, 1, 1)]:
        want = pack(INSTR_FIELDS, dict(d_fmt=1, a_fmt=1, b_fmt=1, a_major=amn, b_major=bmn, n=N >> 3, m=M >> 4))
        assert umma.host_instr_desc(M, N, amn, bmn) == want
    # M = 128, N = 256, both K-major: the values a reader can check by hand
    assert umma.host_instr_desc(128, 256, 0, 0) == (1 << 4) | (1 << 7) | (1 << 10) | (32 << 17) | (8 << 24)


def _unpack(desc):
    f = {name: (desc >> lo) & ((1 << w) - 1) for name, lo, w in SMEM_FIELDS}
    return f["start"] << 4, f["lbo"] << 4, f["sbo"] << 4, f["swizzle"]


def _swz(a):
    """128-byte swizzle on an absolute shared-memory byte address (1 KB-aligned blocks)."""
    return a ^ (((a >> 7) & 7) << 4)


def _tma(base, inner, outer):
    """Address at which a 2D TMA box of 128-byte rows with 128-byte swizzling puts element
    (inner, outer) of a bf16 box starting at base."""
    return _swz(base + outer * 128 + inner * 2)


@pytest.mark.parametrize("rows", [128, 256])
def test_kmajor_descriptor_addresses_match_tma(umma, rows):
    base = 0x8000                      # 1 KB aligned
    for k16 in range(4):
        start, lbo, sbo, sw = _unpack(umma.host_kmajor_desc(base, k16))
        assert sw == 2
        for r in range(rows):
            for k in range(16):
                # canonical K-major 128B layout: 8-row core groups at sbo, rows at 128 B, k at 2 B
                addr = _swz(start + (r // 8) * sbo + (r % 8) * 128 + 2 * k)
                assert addr == _tma(base, 16 * k16 + k, r)


@pytest.mark.parametrize("rows", [128, 256])
def test_mnmajor_descriptor_addresses_match_tma(umma, rows):
    base = 0x10000
    box = 64 * 64 * 2                  # one TMA box: 64 rows of the operand (m or n) x 64 k
    for k16 in range(4):
        start, lbo, sbo, sw = _unpack(umma.host_mnmajor_desc(base, k16))
        assert sw == 2
        for mn in range(rows):
            for k in range(16):
                # canonical MN-major 128B layout: 64 mn at 2 B, 64-mn groups at lbo, k rows at
                # 128 B, 8-k groups at sbo
                addr = _swz(start + (mn // 64) * lbo + (mn % 64) * 2 + (k // 8) * sbo + (k % 8) * 128)
                kk = 16 * k16 + k
                assert addr == _tma(base + (mn // 64) * box, mn % 64, kk)
