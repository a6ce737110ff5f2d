"""Host-side test (no GPU): the Python binding declares every entry point of
include/lrcc.h with the header's arity and argument types, so no pointer or 64-bit
argument is truncated at the boundary."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCALARS = {"int32_t": C.c_int32, "int64_t": C.c_int64, "uint64_t": C.c_uint64, "double": C.c_double,
            "size_t": C.c_size_t}
_RETURNS = {"lrcc_status": C.c_int, "int32_t": C.c_int32, "int64_t": C.c_int64, "const char*": C.c_char_p,
            "void": None, "double": C.c_double}


def _declarations():
    hdr = open(os.path.join(ROOT, "include", "lrcc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", " ", hdr, flags=re.S)
    out = {}
    for ret, name, params in re.findall(
            r"^(lrcc_status|void|int32_t|int64_t|const char\*|double)\s+(lrcc_\w+)\s*\(([^)]*)\)\s*;", hdr, re.M):
        ps = [q.strip() for q in params.replace("\n", " ").split(",")]
        if ps == ["void"] or ps == [""]:
            ps = []
        out[name] = (ret, ps)
    return out


@pytest.fixture(scope="module")
def sigs():
    import __graft_entry__ as g
    g.build()
    from paper_2508_01266_gb300 import _lib
    return _lib._SIGS


def test_every_declaration_has_a_matching_signature(sigs):
    decls = _declarations()
    assert len(decls) >= 25
    assert set(decls) == set(sigs), sorted(set(decls) ^ set(sigs))
    for name, (ret, params) in decls.items():
        res, args = sigs[name]
        assert res is _RETURNS[ret], (name, ret, res)
        assert len(args) == len(params), (name, params, args)
        for p, a in zip(params, args):
            if "*" in p:  # any pointer: void*, typed pointer, string, or a ctypes POINTER type
                assert a in (C.c_void_p, C.c_char_p) or issubclass(a, C._Pointer), (name, p, a)
            else:
                ctype = p.replace("const ", "").split()[0]
                assert a is _SCALARS[ctype], (name, p, a)
