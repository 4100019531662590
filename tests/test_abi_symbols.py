"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

CPU-only: no compute call is made (there may be no GPU here).
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(did_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["did_create", "did_create_ex", "did_sweep", "did_factor", "did_objective",
                     "did_refresh_residual", "did_get_factors", "did_set_factors", "did_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi(lib):
    import paper_1802_08938_gb300 as did
    for n in declared_functions():
        if n in ("did_default_options", "did_last_error", "did_status_string", "did_get_info",
                 "did_get_phase_times"):
            continue
        assert hasattr(did, n) or n in ("did_create_ex",), n


def test_status_strings(lib):
    import paper_1802_08938_gb300 as did
    assert did.status_string(did.DID_ETIMEOUT) == "DID_ETIMEOUT"
    assert did.status_string(did.DID_OK) == "DID_OK"


def test_options_struct_layout(lib):
    import paper_1802_08938_gb300 as did
    o = did.default_options()
    assert o.precision == did.DID_FP32 and o.order == did.DID_ORDER_INTERLEAVED
    assert o.refresh_every == 0 and o.debug_barrier_extra == 0
    # 6 int32 + 3 pointers + uint64 + 2 int32 on an LP64 ABI
    assert ctypes.sizeof(did.did_options) == 6 * 4 + 3 * 8 + 8 + 4 * 4


def test_host_side_argument_checks_need_no_gpu(lib):
    import paper_1802_08938_gb300 as did
    h = ctypes.c_void_p()
    # NULL X, K > min(M, N), and zero sizes are rejected before any CUDA call
    assert did._lib.did_create(None, 4, 4, 2, 0, ctypes.byref(h)) == did.DID_EINVAL
    x = (ctypes.c_float * 16)()
    assert did._lib.did_create(x, 4, 4, 5, 0, ctypes.byref(h)) == did.DID_EINVAL
    assert did._lib.did_create(x, 0, 4, 1, 0, ctypes.byref(h)) == did.DID_EINVAL
    assert not h.value
