"""The binding declares every entry point with the header's signature: same
number of arguments, and each argument of the same kind (pointer, int,
long long, unsigned, float, double), and the same return kind."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HANDLES = ("srw_handle", "srw_group", "srw_surrogate")
ENUMS = ("srw_status", "srw_precision", "srw_where", "srw_scan_rule")


@pytest.fixture(scope="module")
def lib():
    from paper_2607_00488_gb300 import build
    build.build()
    import paper_2607_00488_gb300 as pkg
    return pkg.lib()


def _prototypes():
    text = open(os.path.join(ROOT, "include", "srw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"(\b[\w ]+?[\s\*]+)(srw_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        ret, name, params = m.group(1), m.group(2), " ".join(m.group(3).split())
        if "typedef" in ret:
            continue
        ps = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        out[name] = (ret.strip(), ps)
    return out


def _c_kind(decl):
    if "*" in decl or any(re.search(r"\b%s\b" % h, decl) for h in HANDLES):
        return "ptr"
    if "long long" in decl:
        return "longlong"
    if "unsigned" in decl:
        return "uint"
    if re.search(r"\bdouble\b", decl):
        return "double"
    if re.search(r"\bfloat\b", decl):
        return "float"
    if re.search(r"\bint\b", decl) or any(re.search(r"\b%s\b" % e, decl) for e in ENUMS):
        return "int"
    raise AssertionError("unclassified C type: " + decl)


def _py_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_uint: "uint", ctypes.c_longlong: "longlong", ctypes.c_double: "double",
            ctypes.c_float: "float"}[t]


def test_every_prototype_is_parsed():
    protos = _prototypes()
    from paper_2607_00488_gb300 import srw as binding
    assert set(binding.EXPORTS) == set(protos)


def test_argument_and_return_kinds_match(lib):
    for name, (ret, params) in _prototypes().items():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert [_py_kind(t) for t in f.argtypes] == [_c_kind(p) for p in params], name
        if ret.startswith("const char"):
            assert f.restype == ctypes.c_char_p, name
        else:
            assert ret == "srw_status" and f.restype == ctypes.c_int, name
