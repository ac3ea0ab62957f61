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
