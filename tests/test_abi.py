"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/gwfa.h declares (no compute calls here)."""
import ctypes
import os
import re

import paper_2206_13574_gb300 as gw
from paper_2206_13574_gb300 import _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gwfa.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gwfa_[a-z_0-9]+)\s*\(", text)))


def test_library_builds_and_exports_header_symbols():
    _build.build()
    lib = gw.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert n in gw.SIGNATURES, n
    assert set(gw.SIGNATURES) == set(names)


def test_struct_layouts_match_header():
    assert ctypes.sizeof(gw.gwfa_result) == 64
    assert gw.RESULT_DTYPE.itemsize == 64
    assert ctypes.sizeof(gw.gwfa_opts) == 28
    assert ctypes.sizeof(gw.gwfa_engine_config) == 128   # 108 bytes of u32 fields, padded to 8
    assert ctypes.sizeof(gw.gwfa_schedule) == 8
    assert gw.CIGAR_RESULT_DTYPE.itemsize == 24
    for name, _ in gw.gwfa_result._fields_:
        assert name in gw.RESULT_DTYPE.names


def test_strerror_without_gpu():
    lib = gw.load()
    assert lib.gwfa_strerror(gw.GWFA_ERR_CAPACITY) == b"workspace capacity exceeded"
    assert lib.gwfa_strerror(0) == b"ok"


def test_invalid_arguments_rejected_on_host():
    """Argument checks that return before any CUDA call."""
    lib = gw.load()
    h = ctypes.c_void_p()
    assert lib.gwfa_graph_create(0, None, None, 0, None, None, 0, ctypes.byref(h)) == gw.GWFA_ERR_INVALID
    assert lib.gwfa_graph_destroy(None) == gw.GWFA_ERR_INVALID
    assert lib.gwfa_engine_destroy(None) == gw.GWFA_ERR_INVALID
