"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/rqrcp.h declares; the Python binding names the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rqrcp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1509_06820_gb300 import build
    return build.build()


def test_header_parses():
    names = declared_functions()
    for must in ["rqrcp_factor", "qr_factor", "trqrcp", "tuxv", "rqrcp_create", "rqrcp_destroy",
                 "rqrcp_sync_info", "rqrcp_workspace_bytes", "rqrcp_status_string"]:
        assert must in names


def test_library_exports_header(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1509_06820_gb300 as rq
    bound = {s[0] for s in rq.SIGNATURES}
    assert bound == set(declared_functions())


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.rqrcp_status_string.restype = ctypes.c_char_p
    assert lib.rqrcp_status_string(0) == b"ok"
    assert b"invalid" in lib.rqrcp_status_string(-3)
    assert lib.rqrcp_status_string(2).startswith(b"singular")


def test_null_handle_rejected_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.rqrcp_factor.restype = ctypes.c_int
    lib.rqrcp_factor.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.c_void_p, ctypes.c_void_p]
    assert lib.rqrcp_factor(None, 10, 10, None, 10, 4, 2, 0, None, None) == -1


def declared_prototypes():
    """{name: [parameter declarations]} from include/rqrcp.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s+\**([A-Za-z_]\w*)\s*\(([^;]*?)\)\s*;",
                         text, flags=re.M | re.S):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",") if p.strip()]
        if params == ["void"]:
            params = []
        protos[m.group(1)] = params
    return protos


def _ctype_kind(decl):
    """Coarse class of a C parameter: pointer, 64-bit integer, 32-bit integer,
    char, double or float -- what the ctypes argtype must agree with."""
    if "*" in decl or decl.startswith("rqrcp_handle_t"):   # the handle is a pointer typedef
        return "ptr"
    if "int64_t" in decl or "uint64_t" in decl or "size_t" in decl:
        return "i64"
    if "uint32_t" in decl or re.match(r"^(const\s+)?int\b", decl):
        return "i32"
    if re.match(r"^(const\s+)?char\b", decl):
        return "char"
    if re.match(r"^(const\s+)?double\b", decl):
        return "f64"
    if re.match(r"^(const\s+)?float\b", decl):
        return "f32"
    return "other"


def _argtype_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and t.__name__.startswith("LP_"):
        return "ptr"
    if t in (ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t):
        return "i64"
    if t in (ctypes.c_int, ctypes.c_uint32, ctypes.c_int32):
        return "i32"
    if t is ctypes.c_char:
        return "char"
    if t is ctypes.c_double:
        return "f64"
    if t is ctypes.c_float:
        return "f32"
    return "other"


def test_binding_argtypes_match_header():
    """Every ctypes signature has the header prototype's arity and, argument by
    argument, the same class of C type (pointer / 64-bit / 32-bit integer /
    char / double / float): a shifted or missing argument fails here."""
    import paper_1509_06820_gb300 as rq
    protos = declared_prototypes()
    bad = []
    for name, _, argtypes in rq.SIGNATURES:
        params = protos[name]
        if len(params) != len(argtypes):
            bad.append((name, "arity", len(params), len(argtypes)))
            continue
        for i, (p, t) in enumerate(zip(params, argtypes)):
            kp, kt = _ctype_kind(p), _argtype_kind(t)
            if kp != kt and not (kp == "ptr" and kt == "ptr"):
                bad.append((name, i + 1, p, kp, kt))
    assert not bad, bad
