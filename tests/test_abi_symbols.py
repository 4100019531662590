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


@pytest.mark.parametrize("change", [
    dict(flags=1 << 12),                                             # unknown flag bit
    dict(flags=4, order=2),                                          # a flag bit this library no longer takes
    dict(flags=8 | 16),                                              # eager and lazy write-back together
    dict(inner_c=2),                                                 # inner repeats outside the batched order
    dict(order=2, inner_b=65),                                       # more than 64 repeats
    dict(order=2, inner_c=-1),
    dict(order=2, precision=1),                                      # batched order with a bfloat16 residual
    dict(order=3),                                                   # no such order
    dict(precision=2),                                               # no such precision
    dict(stop=2),
    dict(refresh_every=-1),
])
def test_invalid_options_rejected_before_any_cuda_call(lib, change):
    import paper_1802_08938_gb300 as did
    o = did.default_options()
    for k, v in change.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    x = (ctypes.c_float * 64)()
    assert did._lib.did_create_ex(x, 8, 8, 2, 0, ctypes.byref(o), ctypes.byref(h)) == did.DID_EINVAL
    assert not h.value


# ---------------------------------------------- struct layouts and constants
STRUCTS = ["did_options", "did_info", "did_request", "did_result", "did_server_stats_t"]


def c_struct_layout(tmp_path, did, cc):
    """sizeof and field offsets of every public struct, as a C compiler lays
    them out from include/did.h (host ABI)."""
    import subprocess
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "did.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (s, s))
        for f, _ in getattr(did, s)._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(cc + ["-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(line.split()[:2]): int(line.split()[2]) for line in out.splitlines()}


def test_struct_layouts_match_the_header(tmp_path, c_compiler):
    import paper_1802_08938_gb300 as did
    layout = c_struct_layout(tmp_path, did, c_compiler)
    for s in STRUCTS:
        cls = getattr(did, s)
        assert layout[(s, "sizeof")] == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert layout[(s, f)] == getattr(cls, f).offset, (s, f)
    # every field the header declares is bound (none missing from the binding)
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "did.h")).read(), flags=re.S)
    for s in STRUCTS:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*%s;" % s, text).group(1)
        names = set()
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                names.add(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part)[-1])
        assert names == {f for f, _ in getattr(did, s)._fields_}, s


def test_constants_match_the_header():
    import paper_1802_08938_gb300 as did
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "did.h")).read(), flags=re.S)
    found = 0
    for name, val in re.findall(r"#define\s+(DID_[A-Z0-9_]+)\s+(-?\d+)", text):
        assert getattr(did, name) == int(val), name
        found += 1
    for body in re.findall(r"typedef enum \{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(DID_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            assert getattr(did, name) == int(val), name
            found += 1
    assert found >= 20
