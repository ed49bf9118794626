"""CPU test: the ctypes binding declares every entry point of include/sbp.h with the header's
parameter types (scalar widths exactly; pointers as void* or a pointer to the same type), and
the two structs it passes by pointer have the header's field order, types and array lengths."""
import ctypes
import os
import re

import pytest

from paper_2011_02600_gb300 import _lib as L
from paper_2011_02600_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = open(os.path.join(ROOT, "include", "sbp.h")).read()

SCALARS = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint32_t": ctypes.c_uint32,
           "double": ctypes.c_double, "float": ctypes.c_float}
STRUCTS = {"SbpGridDesc": L.SbpGridDesc, "SbpSource": L.SbpSource}


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def _strip_comments(text):
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def _prototypes():
    text = _strip_comments(HEADER)
    out = {}
    for m in re.finditer(r"^\s*(?:int|const char\*)\s+(sbp_\w+)\s*\(([^)]*)\)\s*;", text, re.M | re.S):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",")]
        out[m.group(1)] = [] if params == ["void"] else params
    return out


def _ctype_of(param):
    """(is_pointer, base C type, pointer depth) of one declared parameter."""
    p = re.sub(r"\bconst\b", "", param).strip()
    depth = p.count("*")
    base = p.replace("*", " ").split()[0]
    return depth, base


def _matches(depth, base, ct):
    if depth == 0:
        return ct is SCALARS[base]
    if ct is ctypes.c_void_p:
        return True
    if not (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)):
        return False
    inner = ct._type_
    if depth == 2:                                   # SbpGrid** out: pointer to an opaque handle
        return inner is ctypes.c_void_p
    if base in SCALARS:
        return inner is SCALARS[base]
    return inner is STRUCTS.get(base)


def test_every_prototype_matches_the_binding(lib):
    protos = _prototypes()
    assert len(protos) >= 40
    for name, params in protos.items():
        fn = getattr(lib, name)
        if name == "sbp_last_error":
            assert fn.restype is ctypes.c_char_p
            continue
        assert fn.restype is ctypes.c_int, name
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for p, ct in zip(params, fn.argtypes):
            depth, base = _ctype_of(p)
            assert _matches(depth, base, ct), (name, p, ct)


def _struct_fields(name):
    m = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", _strip_comments(HEADER), re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        ctype, rest = decl.split(None, 1)
        for item in rest.split(","):
            item = item.strip()
            am = re.match(r"(\w+)\s*(?:\[(\d+)\])?$", item)
            fields.append((am.group(1), ctype, int(am.group(2)) if am.group(2) else 0))
    return fields


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layouts_match_the_header(name):
    want = _struct_fields(name)
    got = STRUCTS[name]._fields_
    assert [f[0] for f in want] == [g[0] for g in got]
    for (fname, ctype, n), (_, ct) in zip(want, got):
        if n:
            assert issubclass(ct, ctypes.Array) and ct._length_ == n and ct._type_ is SCALARS[ctype], fname
        else:
            assert ct is SCALARS[ctype], fname
