"""The C ABI used from C: tests/c_api_example.c includes only include/did.h
and links libdid.so (no Python, no PyTorch on its path).  On the CPU it must
compile and link; on the GPU its factorisation must match the oracle's."""

import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_api_example.c")


@pytest.fixture(scope="module")
def exe(tmp_path_factory, c_compiler):
    import __graft_entry__
    lib = __graft_entry__._builder().build()
    out = str(tmp_path_factory.mktemp("capi") / "c_api_example")
    libdir = os.path.dirname(lib)
    # the source first: a "-x c" in the compiler's argv applies to it, not to the library
    subprocess.run(c_compiler + ["-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
                                 "-x", "none", "-o", out, "-L", libdir, "-ldid", "-Wl,-rpath," + libdir], check=True)
    return out


def test_c_program_compiles_and_links(exe):
    assert os.path.exists(exe)


def _x(M, N, K):
    m = np.arange(M)[:, None]
    j = np.arange(N)[None, :]
    X = np.zeros((M, N))
    for k in range(K + 2):
        X += (1.0 + (m + k) % 7) / 7.0 * (1.0 + (j + 2 * k) % 5) / 5.0
    return X.astype(np.float32)


@pytest.mark.gpu
def test_c_program_matches_oracle(exe):
    from oracle import did_oracle as O
    from synth import workloads as W
    M, N, K, sweeps = 300, 2000, 6, 20
    r = subprocess.run([exe, str(M), str(N), str(K), str(sweeps)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    fields = r.stdout.split()
    assert fields[0] == "ok", r.stdout
    iters, f, t0, t1, bmin, cmin = int(fields[1]), *map(float, fields[2:])
    X = _x(M, N, K)
    B0, C0 = W.init_factors(M, N, K, 11)
    ref = O.factor(X, B0, C0, order="hals", max_iter=sweeps, stop="none")
    print("C program: %d sweeps, f %.9g (oracle %.9g), trace %.6g -> %.6g" % (iters, f, ref["trace"][-1], t0, t1))
    assert iters == sweeps
    assert abs(t0 - ref["trace"][0]) <= 1e-5 * ref["trace"][0]
    assert abs(f - ref["trace"][-1]) <= 1e-5 * ref["trace"][-1]
    assert bmin >= 0 and cmin >= 0
