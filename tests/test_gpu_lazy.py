"""Deferred write-back of the interleaved sweep on the GPU.

The pass for k (k even, with a partner k+1) stores nothing; the pass for k+1
applies the pending rank-one change b_k c_k - b_k' c_k' to the column it reads
and writes R once for both.  The blocks and their closed forms are those of
HALS (Section 2), so the result is compared with the oracle's HALS sweep, with
the eager kernel (one write per k), for odd and even K, in both precisions.
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def run(did, X, B0, C0, sweeps, **kw):
    M, N = X.shape
    K = B0.shape[1]
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(np.asarray(B0, np.float32).T),
                     C_init=np.ascontiguousarray(np.asarray(C0, np.float32)), **kw) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return dict(B=B, C=C, R=ctx.residual(), trace=ctx.trace(), info=ctx.info(), obj=ctx.objective())


@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (37, 53, 3), (300, 4000, 7), (130, 2000, 1), (64, 5000, 2),
                                   (1000, 3000, 5)])
def test_lazy_matches_oracle_and_eager(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=3 * M + N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 5)
    sweeps = 20
    ref = O.factor(X, B0, C0, order="hals", max_iter=sweeps, stop="none")
    lz = run(did, X, B0, C0, sweeps)
    eg = run(did, X, B0, C0, sweeps, flags=did.DID_FLAG_EAGER_WRITEBACK)
    assert lz["info"]["lazy_writeback"] == (1 if K >= 2 else lz["info"]["lazy_writeback"])
    assert eg["info"]["lazy_writeback"] == 0
    eB, eC = rel_fro(lz["B"], ref["B"]), rel_fro(lz["C"], ref["C"])
    eF = float(np.max(np.abs(lz["trace"] - ref["trace"]) / ref["trace"]))
    print("lazy M=%d N=%d K=%d stages=%d: relB %.3g relC %.3g max relf %.3g (eager relB %.3g)" % (
        M, N, K, lz["info"]["ring_stages"], eB, eC, eF, rel_fro(eg["B"], ref["B"])))
    assert eB <= 1e-4 and eC <= 1e-4 and eF <= 1e-5
    # every pending change reached R: the stored residual is X - B C
    Rd = X.astype(np.float64) - lz["B"].astype(np.float64) @ lz["C"].astype(np.float64)
    assert np.max(np.abs(lz["R"] - Rd)) <= 1e-4 * max(1.0, float(np.abs(X).max()))


def test_lazy_dynamic_units_and_refresh(did):
    M, N, K = 64, 500000, 4             # short columns, many of them: column units from a counter
    X, _, _ = W.planted(M, N, K, seed=77, sigma=0.05)
    B0, C0 = W.init_factors(M, N, K, 77)
    sweeps = 6
    ref = O.factor(X, B0, C0, order="hals", max_iter=sweeps, stop="none")
    a = run(did, X, B0, C0, sweeps, refresh_every=4)
    b = run(did, X, B0, C0, sweeps, refresh_every=4)
    assert a["info"]["lazy_writeback"] == 1 and a["info"]["dynamic_units"] == 1
    assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["C"], b["C"])   # bitwise deterministic
    eF = float(np.max(np.abs(a["trace"] - ref["trace"]) / ref["trace"]))
    print("lazy dynamic units: relB %.3g relC %.3g max relf %.3g" % (
        rel_fro(a["B"], ref["B"]), rel_fro(a["C"], ref["C"]), eF))
    assert rel_fro(a["B"], ref["B"]) <= 1e-4 and rel_fro(a["C"], ref["C"]) <= 1e-4 and eF <= 1e-5


@pytest.mark.parametrize("K", [6, 5])
def test_lazy_bf16_residual(did, K):
    M, N = 800, 6000
    X, _, _ = W.planted(M, N, K, seed=K, sigma=0.02)
    B0, C0 = W.init_factors(M, N, K, K)
    sweeps = 15
    ref = O.factor(X, B0, C0, order="hals", max_iter=sweeps, stop="none")
    lz = run(did, X, B0, C0, sweeps, precision=did.DID_BF16R, refresh_every=5, flags=did.DID_FLAG_LAZY_WRITEBACK)
    eg = run(did, X, B0, C0, sweeps, precision=did.DID_BF16R, refresh_every=5)
    f_ref = ref["trace"][-1]
    print("bf16 lazy K=%d: f rel %.3g (eager %.3g), lazy=%d" % (
        K, abs(lz["obj"] - f_ref) / f_ref, abs(eg["obj"] - f_ref) / f_ref, lz["info"]["lazy_writeback"]))
    assert lz["info"]["lazy_writeback"] == 1 and eg["info"]["lazy_writeback"] == 0
    assert abs(lz["obj"] - f_ref) / f_ref <= 1e-3
    assert abs(lz["obj"] - eg["obj"]) / f_ref <= 1e-3


def test_lazy_stopping_and_resume(did):
    M, N, K = 120, 900, 4
    X, _, _ = W.planted(M, N, K, seed=8, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 8)
    ref = O.factor(X, B0, C0, order="hals", max_iter=500, tol=1e-2, stop="relchange")
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(B0.T.astype(np.float32)),
                     C_init=np.ascontiguousarray(C0.astype(np.float32))) as ctx:
        iters, f = ctx.factor(500, 1e-2)
        assert ctx.info()["lazy_writeback"] == 1
    print("lazy stopping: GPU %d sweeps, oracle %d" % (iters, ref["iters"]))
    assert iters == ref["iters"]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_lazy_bitwise_deterministic(did, prec):
    M, N, K = 2000, 30000, 6
    X, _, _ = W.planted(M, N, K, seed=11, sigma=0.02)
    B0, C0 = W.init_factors(M, N, K, 11)
    kw = dict(flags=did.DID_FLAG_LAZY_WRITEBACK)
    if prec == "bf16":
        kw["precision"] = did.DID_BF16R
    a = run(did, X, B0, C0, 6, **kw)
    b = run(did, X, B0, C0, 6, **kw)
    assert a["info"]["lazy_writeback"] == 1
    assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["C"], b["C"])
    assert np.array_equal(a["trace"], b["trace"])


@pytest.mark.parametrize("lazy", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_column_pairs_equal_single_columns(did, prec, lazy):
    """Pairs take the same sums in the same order: bitwise equal results."""
    M, N, K = 1500, 20001, 5                   # odd N: units end with a single column
    X, _, _ = W.planted(M, N, K, seed=12, sigma=0.02)
    B0, C0 = W.init_factors(M, N, K, 12)
    kw = dict(precision=did.DID_BF16R) if prec == "bf16" else {}
    kw["flags"] = did.DID_FLAG_LAZY_WRITEBACK if lazy else did.DID_FLAG_EAGER_WRITEBACK
    a = run(did, X, B0, C0, 4, **kw)
    kw["flags"] |= did.DID_FLAG_SINGLE_COLUMNS
    b = run(did, X, B0, C0, 4, **kw)
    print("pairs %s lazy=%s: pair=%d stages=%d" % (prec, lazy, a["info"]["column_pairs"], a["info"]["ring_stages"]))
    assert b["info"]["column_pairs"] == 0
    assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["C"], b["C"])
    assert np.array_equal(a["trace"], b["trace"])
