"""GPU parity: the CUDA sweep through the C ABI against the FP64 oracle.

Tolerances (FP32 path vs FP64 oracle, same seeded inputs and start point):
after 20 sweeps B and C within 1e-4 relative Frobenius error and the
objective within 1e-5 relative error.  The measured errors are printed.
"""

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu

TOL_FACTOR = 1e-4
TOL_OBJ = 1e-5
# When the fit is exact (f -> 0) a relative objective error is meaningless: a
# float32 residual carries rounding of about u |X| per entry (u = 2^-24), so
# its 1/2 ||R||^2 cannot go below ~u^2 ||X||^2.  The objective error is taken
# relative to max(f, 1e-10 ||X||^2), far above that floor.
OBJ_FLOOR = 1e-10


def rel_obj(f_got, f_ref, X):
    floor = OBJ_FLOOR * float(np.sum(np.asarray(X, np.float64) ** 2))
    return abs(f_got - f_ref) / max(abs(f_ref), floor)


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(did, X, B0, C0, sweeps, **kw):
    M, N = X.shape
    K = B0.shape[1]
    Xc = np.ascontiguousarray(X.T)                       # (N, M) row-major == M x N column-major
    Bc = np.ascontiguousarray(np.asarray(B0, np.float32).T)
    Cc = np.ascontiguousarray(np.asarray(C0, np.float32))
    with did.Context(Xc, M, N, K, B_init=Bc, C_init=Cc, **kw) as ctx:
        if sweeps:
            ctx.sweep(sweeps)
        B, C = ctx.factors()
        R = ctx.residual()
        return dict(B=B, C=C, R=R, trace=ctx.trace(), info=ctx.info(), obj=ctx.objective())


def parity_case(did, X, K, seed, sweeps=20, order="hals"):
    M, N = X.shape
    B0, C0 = W.init_factors(M, N, K, seed)
    ref = O.factor(X, B0, C0, order=order, max_iter=sweeps, stop="none")
    got = run_gpu(did, X, B0, C0, sweeps)
    eB, eC = rel_fro(got["B"], ref["B"]), rel_fro(got["C"], ref["C"])
    eF = rel_obj(got["trace"][-1], ref["trace"][-1], X)
    print("M=%d N=%d K=%d sweeps=%d: relB=%.3g relC=%.3g relf=%.3g" % (M, N, K, sweeps, eB, eC, eF))
    return got, ref, eB, eC, eF


def test_planted_200x1000_k10_20_sweeps(did):
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=0)
    got, ref, eB, eC, eF = parity_case(did, X, K, seed=0, sweeps=20)
    assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ
    # the trace after every sweep, not only the last
    tr = np.abs(got["trace"] - ref["trace"]) / ref["trace"]
    assert tr.max() <= TOL_OBJ, tr.max()
    assert got["B"].min() >= 0 and got["C"].min() >= 0


def test_planted_200x1000_k10_100_sweeps_invariants(did):
    """100 sweeps: nonnegativity, monotone trace, R == X - BC, trace vs oracle."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=0)
    B0, C0 = W.init_factors(M, N, K, 0)
    ref = O.factor(X, B0, C0, order="hals", max_iter=100, stop="none")
    got = run_gpu(did, X, B0, C0, 100)
    assert got["B"].min() >= 0 and got["C"].min() >= 0
    t = got["trace"]
    assert np.all(np.diff(t) <= 1e-6 * t[:-1]), "objective increased"
    R_def = X.astype(np.float64) - got["B"].astype(np.float64) @ got["C"].astype(np.float64)
    err = np.max(np.abs(got["R"] - R_def)) / max(1.0, np.max(np.abs(X)))
    print("100 sweeps: max |R - (X-BC)| / max(1,|X|) = %.3g" % err)
    assert err < 1e-4
    eF = abs(t[-1] - ref["trace"][-1]) / ref["trace"][-1]
    print("100 sweeps: relf=%.3g" % eF)
    assert eF <= 1e-4
    # the exact objective from a fresh pass agrees with the kept residual's
    assert abs(got["obj"] - t[-1]) / t[-1] < 1e-4


@pytest.mark.parametrize("M,N,K", [(37, 53, 3), (1, 40, 1), (40, 1, 1), (5, 5, 5), (203, 997, 7),
                                   (64, 300, 16), (1000, 129, 4), (784, 700, 16), (2001, 311, 5)])
def test_ragged_shapes(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=M * 7 + N, sigma=0.01)
    got, ref, eB, eC, eF = parity_case(did, X, K, seed=3, sweeps=10)
    assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ


def test_image_like_scaled_down(did):
    X = W.image_like(784, 2000, seed=1)
    K = 16
    B0, C0 = W.init_factors(784, 2000, K, 1)
    B0s, C0s = O.init_scale(X, B0, C0)
    ref = O.factor(X, B0s, C0s, order="hals", max_iter=20, stop="none")
    got = run_gpu(did, X, B0s.astype(np.float32), C0s.astype(np.float32), 20)
    eB, eC = rel_fro(got["B"], ref["B"]), rel_fro(got["C"], ref["C"])
    eF = abs(got["trace"][-1] - ref["trace"][-1]) / ref["trace"][-1]
    print("image-like 784x2000 K=16: relB=%.3g relC=%.3g relf=%.3g" % (eB, eC, eF))
    assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ


def test_seeded_start_point_matches_generator(did):
    """did_create's device-drawn start point equals the host generator bit for bit."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=0)
    B0, C0 = W.init_factors(M, N, K, 11)
    with did.Context(np.ascontiguousarray(X.T), M, N, K, seed=11) as ctx:
        B, C = ctx.factors()
    np.testing.assert_array_equal(B, B0)
    np.testing.assert_array_equal(C, C0)


def test_init_scale_matches_oracle(did):
    X = W.image_like(200, 500, seed=2)
    B0, C0 = W.init_factors(200, 500, 8, 2)
    Bs, Cs = O.init_scale(X, B0, C0)
    with did.Context(np.ascontiguousarray(X.T), 200, 500, 8, seed=2, init_scale=True) as ctx:
        B, C = ctx.factors()
    assert rel_fro(B, Bs) < 1e-6 and rel_fro(C, Cs) < 1e-6


def test_determinism_bitwise(did):
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=4)
    B0, C0 = W.init_factors(M, N, K, 4)
    a = run_gpu(did, X, B0, C0, 15)
    b = run_gpu(did, X, B0, C0, 15)
    np.testing.assert_array_equal(a["B"], b["B"])
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["trace"], b["trace"])


def test_refresh_and_resume(did):
    """Refresh recomputes X - BC; get/set factors resumes a run."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=5)
    B0, C0 = W.init_factors(M, N, K, 5)
    full = run_gpu(did, X, B0, C0, 12, refresh_every=6)
    half = run_gpu(did, X, B0, C0, 6)
    resumed = run_gpu(did, X, half["B"], half["C"], 6)
    # a refresh falls at sweep 6 in the full run: resuming is the same computation
    np.testing.assert_array_equal(full["B"], resumed["B"])
    np.testing.assert_array_equal(full["C"], resumed["C"])
    assert full["info"]["refreshes"] == 1
    R_def = X.astype(np.float64) - full["B"].astype(np.float64) @ full["C"].astype(np.float64)
    assert np.max(np.abs(full["R"] - R_def)) < 1e-4 * max(1.0, np.abs(X).max())


def test_rejected_set_factors_leaves_context_unchanged(did):
    """Factors with a negative or non-finite entry are refused (DID_EINVAL)
    before anything is copied, from host or device memory: the run then
    continues bit for bit as if the call had not been made."""
    import torch
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=8, M=150, N=700, K=6)
    B0, C0 = W.init_factors(M, N, K, 8)
    Xc = np.ascontiguousarray(X.T)
    kw = dict(B_init=np.ascontiguousarray(B0.T), C_init=C0, refresh_every=3)
    with did.Context(Xc, M, N, K, **kw) as a, did.Context(Xc, M, N, K, **kw) as b:
        a.sweep(2)
        b.sweep(2)
        B, C = a.factors()
        bad = []
        Bn = B.copy()
        Bn[7, 2] = -1e-3
        bad.append((Bn, C))
        Cn = C.copy()
        Cn[1, 11] = np.nan
        bad.append((B, Cn))
        Ci = C.copy()
        Ci[5, 0] = np.inf
        bad.append((B, Ci))
        for Bx, Cx in bad:
            with pytest.raises(did.DIDError) as e:
                a.set_factors(Bx, Cx)
            assert e.value.status == did.DID_EINVAL
        # device sources: B transposed to the library's column-major layout
        Bd = torch.as_tensor(np.ascontiguousarray(Bn.T), device="cuda")
        Cd = torch.as_tensor(np.ascontiguousarray(C), device="cuda")
        with pytest.raises(did.DIDError) as e:
            did.did_set_factors(a.h, Bd, Cd)
        assert e.value.status == did.DID_EINVAL
        a.sweep(4)
        b.sweep(4)
        Ba, Ca = a.factors()
        Bb, Cb = b.factors()
        ta, tb = a.trace(), b.trace()
    np.testing.assert_array_equal(Ba, Bb)
    np.testing.assert_array_equal(Ca, Cb)
    np.testing.assert_array_equal(ta, tb)


def test_factor_stopping_rule(did):
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=6, M=100, N=400, K=5)
    B0, C0 = W.init_factors(M, N, K, 6)
    Xc = np.ascontiguousarray(X.T)
    with did.Context(Xc, M, N, K, B_init=np.ascontiguousarray(B0.T), C_init=C0) as ctx:
        it, f = ctx.factor(500, 1e-2)
        t = ctx.trace()
    assert it == len(t) - 1 and it < 500
    assert abs(t[-2] - t[-1]) / t[-2] < 1e-2
    assert all(abs(t[i - 1] - t[i]) / t[i - 1] >= 1e-2 for i in range(1, len(t) - 1))
    # the oracle stops at 45 sweeps here, with relative changes 1.06e-2 then 0.97e-2
    ref = O.factor(X, B0, C0, order="hals", max_iter=500, tol=1e-2, stop="relchange")
    print("stop at %d sweeps (oracle %d)" % (it, ref["iters"]))
    assert abs(it - ref["iters"]) <= 1


def test_degenerate_zero_row(did):
    """A zero row of C leaves b_k unchanged and is counted (the zero-norm rule)."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=7, M=50, N=80, K=3)
    B0, C0 = W.init_factors(M, N, K, 7)
    C0[1, :] = 0.0
    ref = O.factor(X, B0, C0, order="hals", max_iter=3, stop="none")
    got = run_gpu(did, X, B0, C0, 3)
    assert got["info"]["degenerate_events"] >= 1
    assert rel_fro(got["B"], ref["B"]) <= TOL_FACTOR and rel_fro(got["C"], ref["C"]) <= TOL_FACTOR


def test_invalid_inputs_rejected(did):
    X = np.ones((20, 10), np.float32)
    X[3, 4] = -1.0
    with pytest.raises(did.DIDError) as e:
        did.Context(X, 10, 20, 2)
    assert e.value.status == did.DID_EINVAL
    X[3, 4] = np.nan
    with pytest.raises(did.DIDError):
        did.Context(X, 10, 20, 2)
    with pytest.raises(did.DIDError):
        did.Context(np.ones((20, 10), np.float32), 10, 20, 11)


def test_barrier_timeout_is_reported_and_context_survives(did):
    """A grid wait that can never complete returns DID_ETIMEOUT within its limit."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=8, M=64, N=256, K=4)
    Xc = np.ascontiguousarray(X.T)
    ctx = did.Context(Xc, M, N, K, seed=8, timeout_ns=20_000_000, debug_barrier_extra=1)
    with pytest.raises(did.DIDError) as e:
        ctx.sweep(1)
    assert e.value.status == did.DID_ETIMEOUT
    B, C = ctx.factors()                      # the context is still usable
    assert B.min() >= 0 and C.min() >= 0
    f = ctx.objective()
    assert np.isfinite(f)
    ctx.close()
    with did.Context(Xc, M, N, K, seed=8) as ok:   # and so is the CUDA context
        ok.sweep(2)
        assert len(ok.trace()) == 3


def test_tiny_wait_limit_is_raised(did):
    """A wait limit of 1 ns is raised to the 10 ms floor, so the waits for a
    CTA's own copies and tensor-core work never give up: the sweeps (with a
    tensor-core refresh, and in the batched order) equal those of the default
    limit bit for bit."""
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=9, M=300, N=900, K=8)
    Xc = np.ascontiguousarray(X.T)
    for order in (did.DID_ORDER_INTERLEAVED, did.DID_ORDER_DID_BATCHED):
        out = []
        for t in (1, 0):
            with did.Context(Xc, M, N, K, seed=9, order=order, refresh_every=2, timeout_ns=t) as ctx:
                ctx.sweep(4)
                out.append(ctx.factors())
        assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_contexts_of_different_sizes_interleave(did):
    """Two live contexts whose plans share a kernel variant but differ in shared
    memory (M = 200 and M = 216, ld 208 and 224) sweep alternately."""
    out = []
    for M in (200, 216):
        X, _, _ = W.planted(M, 500, 6, seed=M, sigma=0.01)
        out.append((X, did.Context(np.ascontiguousarray(X.T), M, 500, 6, seed=M)))
    try:
        for _ in range(2):
            for X, ctx in out:
                ctx.sweep(2)
        for X, ctx in out:
            M = X.shape[0]
            B0, C0 = W.init_factors(M, 500, 6, M)
            ref = O.factor(X, B0, C0, order="hals", max_iter=4, stop="none")
            B, C = ctx.factors()
            assert rel_fro(B, ref["B"]) <= TOL_FACTOR and rel_fro(C, ref["C"]) <= TOL_FACTOR
    finally:
        for _, ctx in out:
            ctx.close()


def test_device_pointer_inputs(did):
    import torch
    X, M, N, K = W.make("planted_uniform_200x1000_k10", seed=9, M=120, N=333, K=6)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    B0, C0 = W.init_factors(M, N, K, 9)
    with did.Context(Xd, M, N, K, seed=9) as ctx:
        ctx.sweep(5)
        Bd = torch.empty((K, M), device="cuda")
        Cd = torch.empty((K, N), device="cuda")
        did.did_get_factors(ctx.h, Bd, Cd)
        B, C = ctx.factors()
    np.testing.assert_array_equal(Bd.cpu().numpy().T, B)
    np.testing.assert_array_equal(Cd.cpu().numpy(), C)
    ref = O.factor(X, B0, C0, order="hals", max_iter=5, stop="none")
    assert rel_fro(B, ref["B"]) <= TOL_FACTOR


def test_device_generator_matches_host_generator(did):
    import torch
    from synth import rng
    n = 100000
    u = torch.empty(n, device="cuda")
    did.did_generate_uniform(u, n, 123, rng.STREAM_INIT_B)
    np.testing.assert_array_equal(u.cpu().numpy(), rng.uniform_f32(123, rng.STREAM_INIT_B, np.arange(n)))
    M, N, K = 300, 700, 9
    Xd = torch.empty((N, M), device="cuda")
    did.did_generate_planted(Xd, M, N, K, 5, coords=1, zero_frac=0.3, sigma=0.05)
    Xh, _, _ = W.planted(M, N, K, 5, coords="exp", zero_frac=0.3, sigma=0.05)
    assert np.max(np.abs(Xd.cpu().numpy().T - Xh)) <= 1e-5 * np.abs(Xh).max()
    Xd = torch.empty((N, M), device="cuda")
    did.did_generate_planted(Xd, M, N, K, 6, coords=0, salt_frac=0.01, salt_value=5.0)
    Xh, _, _ = W.planted(M, N, K, 6, salt_frac=0.01)
    np.testing.assert_array_equal(Xd.cpu().numpy().T == 5.0, Xh == 5.0)
    assert np.max(np.abs(Xd.cpu().numpy().T - Xh)) <= 1e-5 * np.abs(Xh).max()
    Xd = torch.empty((N, M), device="cuda")
    did.did_generate_image(Xd, M, N, 7, 0.8)
    np.testing.assert_array_equal(Xd.cpu().numpy().T, W.image_like(M, N, 7))


@pytest.mark.parametrize("order,flags", [("hals", "eager"), ("hals", "lazy"), ("dbcd", "eager")])
def test_one_group_takes_consecutive_units(did, order, flags):
    """One CTA with one 512-thread column group and dynamic units: the group
    takes every unit in turn, so each new unit starts right after the previous
    one -- the case where a stale prefetch of c once went unnoticed."""
    M, N, K = 10000, 400, 3
    X, _, _ = W.planted(M, N, K, seed=31, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 31)
    ref = O.factor(X, B0, C0, order=order, max_iter=10, stop="none")
    kw = dict(grid_ctas=1, order=did.DID_ORDER_INTERLEAVED if order == "hals" else did.DID_ORDER_DID,
              flags=did.DID_FLAG_LAZY_WRITEBACK if flags == "lazy" else did.DID_FLAG_EAGER_WRITEBACK)
    if order == "dbcd":
        kw["flags"] = 0
    got = run_gpu(did, X, B0, C0, 10, **kw)
    info = got["info"]
    print("one group, %s/%s: units %d dynamic %d GS %d grid %d" % (order, flags, info["column_units"],
                                                                   info["dynamic_units"], info["group_threads"],
                                                                   info["grid_ctas"]))
    assert info["grid_ctas"] == 1 and info["group_threads"] == 512 and info["dynamic_units"] == 1
    assert info["column_units"] >= 3
    eB, eC = rel_fro(got["B"], ref["B"]), rel_fro(got["C"], ref["C"])
    eF = rel_obj(got["trace"][-1], ref["trace"][-1], X)
    assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ
