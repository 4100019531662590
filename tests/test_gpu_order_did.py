"""The C-first block order of DBCD / DID (Algorithms 2 and 3) on the GPU.

The GPU runs the C step (c_1..c_K with b fixed, equations up:c) and then the
B step (b_1..b_K, each followed by E := E - delta b_i c_i) as column passes.
It is compared with the oracle's DBCD sweep with a kept residual, which the
oracle pins to Algorithm 3 (W, V, delta b) to 1e-12.
"""

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def run(did, X, B0, C0, sweeps, **kw):
    M, N = X.shape
    K = B0.shape[1]
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(B0.T),
                     C_init=np.ascontiguousarray(C0), order=did.DID_ORDER_DID, **kw) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return B, C, ctx.trace(), ctx.residual()


@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (37, 53, 3), (784, 700, 16), (2001, 311, 5), (64, 3000, 8)])
def test_c_first_order_matches_oracle(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=M + 3 * N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 2)
    sweeps = 20 if M * N < 1e6 else 10
    ref = O.factor(X, B0, C0, order="dbcd", max_iter=sweeps, stop="none")
    B, C, t, R = run(did, X, B0, C0, sweeps)
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    eF = abs(t[-1] - ref["trace"][-1]) / ref["trace"][-1]
    print("C-first M=%d N=%d K=%d: relB %.3g relC %.3g relf %.3g" % (M, N, K, eB, eC, eF))
    assert eB <= 1e-4 and eC <= 1e-4 and eF <= 1e-5
    assert np.all(np.diff(t) <= 1e-6 * t[:-1])
    Rd = X.astype(np.float64) - B.astype(np.float64) @ C.astype(np.float64)
    assert np.max(np.abs(R - Rd)) <= 1e-4 * max(1.0, np.abs(X).max())


def test_c_first_order_large_with_units(did):
    """Enough columns for dynamic column units; deterministic across runs."""
    M, N, K = 500, 60000, 12
    X, _, _ = W.planted(M, N, K, seed=4, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 4)
    ref = O.factor(X, B0, C0, order="dbcd", max_iter=4, stop="none")
    B1, C1, t1, _ = run(did, X, B0, C0, 4)
    B2, C2, t2, _ = run(did, X, B0, C0, 4)
    np.testing.assert_array_equal(B1, B2)
    np.testing.assert_array_equal(t1, t2)
    assert rel_fro(B1, ref["B"]) <= 1e-4 and rel_fro(C1, ref["C"]) <= 1e-4
    assert abs(t1[-1] - ref["trace"][-1]) / ref["trace"][-1] <= 1e-5


def test_c_first_order_bf16_and_stopping(did):
    M, N, K = 300, 4000, 10
    X, _, _ = W.planted(M, N, K, seed=8, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 8)
    ref = O.factor(X, B0, C0, order="dbcd", max_iter=15, stop="none")
    B, C, t, _ = run(did, X, B0, C0, 15, precision=did.DID_BF16R, refresh_every=5)
    f = O.objective(X, B, C)
    assert abs(f - ref["trace"][-1]) / ref["trace"][-1] <= 1e-3
    # the paper's stopping rule ||E^t||^2 <= eps ||E^0||^2 on an exact low-rank X
    B0p, C0p = np.random.default_rng(1).uniform(0, 1, (40, 3)), np.random.default_rng(2).uniform(0, 1, (3, 600))
    Xl = (B0p @ C0p).astype(np.float32)
    Bi, Ci = W.init_factors(40, 600, 3, 3)
    r = O.factor(Xl, Bi, Ci, order="dbcd", max_iter=2000, tol=1e-4, stop="paper_eps")
    with did.Context(np.ascontiguousarray(Xl.T), 40, 600, 3, B_init=np.ascontiguousarray(Bi.T), C_init=Ci,
                     order=did.DID_ORDER_DID, stop=did.DID_STOP_PAPER_EPS) as ctx:
        it, _ = ctx.factor(2000, 1e-4)
    print("paper eps rule: GPU %d sweeps, oracle %d" % (it, r["iters"]))
    assert abs(it - r["iters"]) <= 1
