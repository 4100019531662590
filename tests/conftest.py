import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# The property-based oracle tests need hypothesis, which a GPU image may lack;
# there the file is not collected at all (rather than reported as skipped).
try:
    import hypothesis  # noqa: F401
except ImportError:
    collect_ignore = ["test_oracle_properties.py"]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def find_c_compiler():
    """argv prefix of a working C compiler, or None.  A box that builds the
    library has a host compiler for nvcc, but it may be installed only as
    g++ or under a versioned name, so those are tried too (g++ with -x c
    compiles C)."""
    cands = [[c] for c in ("gcc", "cc", "clang", "gcc-14", "gcc-13", "gcc-12")]
    cands += [[c, "-x", "c"] for c in ("g++", "c++", "clang++", "g++-14", "g++-13", "g++-12")]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        with open(src, "w") as f:
            f.write("#include <stdio.h>\nint main(void) { return 0; }\n")
        for c in cands:
            exe = shutil.which(c[0])
            if exe is None:
                continue
            argv = [exe] + c[1:]
            r = subprocess.run(argv + ["-std=c99", src, "-o", os.path.join(d, "t")], capture_output=True)
            if r.returncode == 0:
                return argv
    return None


@pytest.fixture(scope="session")
def c_compiler():
    cc = find_c_compiler()
    if cc is None:
        pytest.skip("no C compiler")
    return cc
