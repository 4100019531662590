"""Batched DID (Algorithm 3: one reduction per sweep) on the GPU.

Compared with the oracle's Algorithm 3 as the paper writes it (E recomputed
from X, the up:c updates, W = E C^T, V = tril(C C^T), the delta-b rule), and
with the GPU's column-pass C-first order, which takes the same blocks.
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


def run(did, X, B0, C0, sweeps, order, **kw):
    M, N = X.shape
    K = B0.shape[1]
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(B0.T),
                     C_init=np.ascontiguousarray(C0), order=order, **kw) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return B, C, ctx.trace(), ctx.residual(), ctx.objective()


# Shapes over one and several 128-row blocks, 64-row chunks and 32/64-column
# tiles, with ragged tails in both directions, K from 3 to the supported 64
# (every row-slot count ceil(K/8) = 1..8 of the column solve).
@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (37, 53, 3), (784, 700, 16), (2001, 311, 5), (300, 5000, 64),
                                   (129, 257, 64), (1000, 4099, 50), (5000, 1500, 50), (333, 777, 29),
                                   (450, 611, 37), (257, 903, 45), (190, 640, 57)])
def test_batched_matches_algorithm3(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=M + 5 * N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 6)
    sweeps = 20
    ref = O.factor(X, B0, C0, order="did", max_iter=sweeps, stop="none")
    B, C, t, R, fx = run(did, X, B0, C0, sweeps, did.DID_ORDER_DID_BATCHED)
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    eF = abs(t[-1] - ref["trace"][-1]) / ref["trace"][-1]
    eT = float(np.max(np.abs(t - ref["trace"]) / ref["trace"]))
    print("batched M=%d N=%d K=%d: relB %.3g relC %.3g relf %.3g (max over sweeps %.3g, exact f %.3g)" % (
        M, N, K, eB, eC, eF, eT, abs(fx - ref["trace"][-1]) / ref["trace"][-1]))
    assert eB <= 1e-4 and eC <= 1e-4 and eF <= 1e-5 and eT <= 1e-5
    assert B.min() >= 0 and C.min() >= 0
    Rd = X.astype(np.float64) - B.astype(np.float64) @ C.astype(np.float64)
    assert np.max(np.abs(R - Rd)) <= 1e-4 * max(1.0, np.abs(X).max())


def test_batched_equals_column_pass_order(did):
    M, N, K = 500, 20000, 12
    X, _, _ = W.planted(M, N, K, seed=4, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 4)
    Bb, Cb, tb, _, _ = run(did, X, B0, C0, 10, did.DID_ORDER_DID_BATCHED)
    Bp, Cp, tp, _, _ = run(did, X, B0, C0, 10, did.DID_ORDER_DID)
    print("batched vs column passes: relB %.3g relC %.3g relf %.3g" % (
        rel_fro(Bb, Bp), rel_fro(Cb, Cp), abs(tb[-1] - tp[-1]) / tp[-1]))
    assert rel_fro(Bb, Bp) <= 1e-4 and rel_fro(Cb, Cp) <= 1e-4
    assert np.max(np.abs(tb - tp) / tp) <= 1e-5


def test_batched_refresh_and_stopping(did):
    M, N, K = 400, 3000, 8
    X, _, _ = W.planted(M, N, K, seed=9, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 9)
    ref = O.factor(X, B0, C0, order="did", max_iter=12, stop="none")
    B, C, t, R, fx = run(did, X, B0, C0, 12, did.DID_ORDER_DID_BATCHED, refresh_every=4)
    assert rel_fro(B, ref["B"]) <= 1e-4 and abs(t[-1] - ref["trace"][-1]) / ref["trace"][-1] <= 1e-5
    # the paper's eps rule on an exact low-rank X: same sweep count as the oracle
    B0p, C0p = np.random.default_rng(1).uniform(0, 1, (40, 3)), np.random.default_rng(2).uniform(0, 1, (3, 600))
    Xl = (B0p @ C0p).astype(np.float32)
    Bi, Ci = W.init_factors(40, 600, 3, 3)
    r = O.factor(Xl, Bi, Ci, order="did", max_iter=2000, tol=1e-4, stop="paper_eps")
    with did.Context(np.ascontiguousarray(Xl.T), 40, 600, 3, B_init=np.ascontiguousarray(Bi.T), C_init=Ci,
                     order=did.DID_ORDER_DID_BATCHED, stop=did.DID_STOP_PAPER_EPS) as ctx:
        it, _ = ctx.factor(2000, 1e-4)
    print("paper eps rule (batched): GPU %d sweeps, oracle %d" % (it, r["iters"]))
    assert abs(it - r["iters"]) <= 1


def test_batched_rejects_bf16_and_large_k(did):
    X = np.ones((300, 200), np.float32)
    with pytest.raises(did.DIDError):
        did.Context(X, 200, 300, 4, order=did.DID_ORDER_DID_BATCHED, precision=did.DID_BF16R)
    for K in (65, 150):
        with pytest.raises(did.DIDError) as e:
            did.Context(X, 200, 300, K, order=did.DID_ORDER_DID_BATCHED)
        assert e.value.status == did.DID_EINVAL
    with did.Context(X, 200, 300, 64, order=did.DID_ORDER_DID_BATCHED) as ctx:   # the largest K taken
        ctx.sweep(1)


@pytest.mark.parametrize("reps", [(3, 3), (6, 1), (1, 5)])
@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (784, 700, 16), (65, 3001, 24)])
def test_inner_repeats_match_oracle(did, M, N, K, reps):
    X, _, _ = W.planted(M, N, K, seed=M + N + K, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 8)
    sweeps = 10
    ref = O.factor(X, B0, C0, order="did", max_iter=sweeps, stop="none", inner_c=reps[0], inner_b=reps[1])
    B, C, t, R, fx = run(did, X, B0, C0, sweeps, did.DID_ORDER_DID_BATCHED, inner_c=reps[0], inner_b=reps[1])
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    eF = np.max(np.abs(t - ref["trace"]) / ref["trace"])
    print("repeats %s M=%d N=%d K=%d: relB %.3g relC %.3g max relf %.3g" % (reps, M, N, K, eB, eC, eF))
    assert eB <= 1e-4 and eC <= 1e-4 and eF <= 1e-5
    assert np.all(np.diff(t) <= 1e-6 * t[0])
    assert B.min() >= 0 and C.min() >= 0


def test_inner_repeats_lower_the_objective_per_sweep(did):
    M, N, K = 300, 4000, 12
    X, _, _ = W.planted(M, N, K, seed=21, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 21)
    f1 = run(did, X, B0, C0, 5, did.DID_ORDER_DID_BATCHED)[2][-1]
    f4 = run(did, X, B0, C0, 5, did.DID_ORDER_DID_BATCHED, inner_c=4, inner_b=4)[2][-1]
    r1 = O.factor(X, B0, C0, order="did", max_iter=5, stop="none")["trace"][-1]
    r4 = O.factor(X, B0, C0, order="did", max_iter=5, stop="none", inner_c=4, inner_b=4)["trace"][-1]
    print("5 sweeps: f(1,1) %.6g oracle %.6g ; f(4,4) %.6g oracle %.6g" % (f1, r1, f4, r4))
    assert (f4 < f1) == (r4 < r1)


def test_inner_repeats_rejected_outside_batched_order(did):
    X, _, _ = W.planted(40, 60, 3, seed=1, sigma=0.01)
    for order, kw in [(did.DID_ORDER_INTERLEAVED, dict(inner_c=2)), (did.DID_ORDER_DID, dict(inner_b=3)),
                      (did.DID_ORDER_DID_BATCHED, dict(inner_c=65)), (did.DID_ORDER_DID_BATCHED, dict(inner_b=-1))]:
        with pytest.raises(did.DIDError):
            did.Context(np.ascontiguousarray(X.T), 40, 60, 3, order=order, **kw)
