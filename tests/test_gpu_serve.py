"""Serving: continuous batching of factorisation requests on one GPU.

Each request's result must be the same whether it runs alone or among other
requests (within the parity tolerances: the CTA split, hence the reduction
order, differs), the HBM budget must never be exceeded, and requests that
arrive while others run must join them on the device.
"""

import time

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_request_matches_oracle(did):
    M, N, K, seed, it = 300, 2000, 8, 77, 15
    with did.Server(4 * GB, max_slots=8, round_sweeps=4) as srv:
        t = srv.submit(M, N, K, seed, max_iter=it, tol=0.0)
        res = srv.wait(t)
        B, C = srv.fetch(t)
    assert res["status"] == did.DID_OK and res["iters"] == it
    X, _, _ = W.planted(M, N, K, seed, sigma=0.01)        # the serving recipe, on the host
    B0, C0 = W.init_factors(M, N, K, seed)
    ref = O.factor(X, B0, C0, order="hals", max_iter=it, stop="none")
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    eF = abs(res["obj"] - ref["trace"][-1]) / ref["trace"][-1]
    print("served request vs oracle: relB %.3g relC %.3g relf %.3g" % (eB, eC, eF))
    assert eB < 1e-4 and eC < 1e-4 and eF < 1e-5


def test_alone_equals_in_mix(did):
    probe = (700, 5000, 16, 1234)
    others = [W.request_shape(0, r) for r in range(24)]
    with did.Server(16 * GB, max_slots=32, round_sweeps=3) as srv:
        t = srv.submit(*probe, max_iter=12, tol=0.0)
        alone = srv.wait(t)
        Ba, Ca = srv.fetch(t)
    with did.Server(16 * GB, max_slots=32, round_sweeps=3) as srv:
        ts = [srv.submit(m, min(n, 20000), k, 9000 + i, max_iter=10, tol=0.0) for i, (m, n, k) in enumerate(others[:12])]
        t = srv.submit(*probe, max_iter=12, tol=0.0)
        ts += [srv.submit(m, min(n, 20000), k, 9100 + i, max_iter=10, tol=0.0) for i, (m, n, k) in enumerate(others[12:])]
        mix = srv.wait(t)
        Bm, Cm = srv.fetch(t)
        for x in ts:
            assert srv.wait(x)["status"] == did.DID_OK
        st = srv.stats()
    print("alone vs mix: relB %.3g relC %.3g relf %.3g, peak active %d" % (
        rel_fro(Bm, Ba), rel_fro(Cm, Ca), abs(mix["obj"] - alone["obj"]) / alone["obj"], st["peak_active"]))
    assert mix["iters"] == alone["iters"] == 12
    assert rel_fro(Bm, Ba) < 1e-4 and rel_fro(Cm, Ca) < 1e-4
    assert abs(mix["obj"] - alone["obj"]) <= 1e-5 * alone["obj"]
    assert st["peak_active"] > 1


def test_budget_and_slots_respected(did):
    shapes = [(1024, 8192, 16)] * 8
    per = 1024 * 8192 * 8           # X + R in FP32
    budget = int(3.5 * per)         # about three requests at once
    with did.Server(budget, max_slots=6, round_sweeps=2) as srv:
        ts = [srv.submit(m, n, k, 50 + i, max_iter=6, tol=0.0) for i, (m, n, k) in enumerate(shapes)]
        rs = [srv.wait(t) for t in ts]
        st = srv.stats()
    assert all(r["status"] == did.DID_OK for r in rs)
    print("budget %.3g GB: peak %.3g GB, peak active %d, rounds %d" % (
        budget / GB, st["peak_bytes"] / GB, st["peak_active"], st["rounds"]))
    assert st["peak_bytes"] <= budget
    assert 1 < st["peak_active"] <= 3


def test_late_arrivals_join_running_requests(did):
    with did.Server(16 * GB, max_slots=16, round_sweeps=2) as srv:
        long_t = srv.submit(2048, 40000, 32, 1, max_iter=60, tol=0.0)
        time.sleep(0.05)
        late = [srv.submit(256, 4000, 8, 100 + i, max_iter=8, tol=0.0) for i in range(6)]
        rl = srv.wait(long_t)
        rs = [srv.wait(t) for t in late]
        st = srv.stats()
    # the small late requests were admitted and finished while the long one ran
    assert all(r["t_start"] < rl["t_done"] for r in rs)
    assert sum(r["t_done"] < rl["t_done"] for r in rs) >= 3
    assert st["peak_active"] >= 2


def test_stopping_rule_and_bf16(did):
    # On this problem the oracle's relative change crosses 1e-2 at sweep 99
    # (1.08e-2 then 0.96e-2), so the stop is well separated from rounding.
    for prec in (did.DID_FP32, did.DID_BF16R):
        with did.Server(8 * GB, precision=prec, max_slots=8, round_sweeps=4) as srv:
            t = srv.submit(400, 3000, 8, 5, max_iter=300, tol=1e-2)
            r = srv.wait(t)
        print("precision %d: stopped after %d sweeps (oracle 99)" % (prec, r["iters"]))
        assert r["status"] == did.DID_OK
        assert abs(r["iters"] - 99) <= (1 if prec == did.DID_FP32 else 5)


def test_bf16r_served_result(did):
    """A request served with a bfloat16 residual: the factorisation it returns
    reaches f(B, C) (evaluated in float64 on the host from the returned factors)
    within 1e-3 of the same request served in float32, and of the oracle."""
    M, N, K, seed, it = 500, 6000, 12, 88, 20
    out = {}
    for prec in (did.DID_FP32, did.DID_BF16R):
        with did.Server(4 * GB, precision=prec, max_slots=4, round_sweeps=4) as srv:
            t = srv.submit(M, N, K, seed, max_iter=it, tol=0.0)
            r = srv.wait(t)
            assert r["status"] == did.DID_OK and r["iters"] == it
            out[prec] = srv.fetch(t)
    X, _, _ = W.planted(M, N, K, seed, sigma=0.01)      # the serving recipe, on the host
    B0, C0 = W.init_factors(M, N, K, seed)
    ref = O.factor(X, B0, C0, order="hals", max_iter=it, stop="none")
    f = {p: O.objective(X, np.asarray(b, np.float64), np.asarray(c, np.float64)) for p, (b, c) in out.items()}
    f_ref = ref["trace"][-1]
    d32 = abs(f[did.DID_BF16R] - f[did.DID_FP32]) / f[did.DID_FP32]
    dref = abs(f[did.DID_BF16R] - f_ref) / f_ref
    print("served f(B,C): fp32 %.9g, bf16r %.9g, oracle %.9g: bf16r vs fp32 %.3g, vs oracle %.3g"
          % (f[did.DID_FP32], f[did.DID_BF16R], f_ref, d32, dref))
    assert d32 <= 1e-3 and dref <= 1e-3
    assert abs(f[did.DID_FP32] - f_ref) / f_ref <= 1e-5


def test_oversize_rejected(did):
    with did.Server(1 * GB, max_slots=4) as srv:
        with pytest.raises(did.DIDError) as e:
            srv.submit(40000, 1000, 8, 1)            # M beyond the serving kernel's rows
        assert e.value.status == did.DID_E_TOO_LARGE
        with pytest.raises(did.DIDError) as e:
            srv.submit(4096, 65536, 8, 1)            # 2 GB of X + R: above the budget
        assert e.value.status == did.DID_E_TOO_LARGE


def test_invalid_input_fails_alone(did):
    """A request whose X has a negative or non-finite entry fails with
    DID_EINVAL at admission; the requests around it are served as usual, and
    a caller-supplied X gives the oracle's result."""
    import torch
    M, N, K, it = 200, 1500, 6, 10
    X, _, _ = W.planted(M, N, K, 31, sigma=0.01)
    Xc = np.ascontiguousarray(X.T).astype(np.float32)       # (N, M) == M x N column-major
    Xneg = Xc.copy()
    Xneg[17, 3] = -0.5
    Xnan = torch.as_tensor(Xc, device="cuda").clone()
    Xnan[100, 9] = float("nan")
    with did.Server(4 * GB, max_slots=8, round_sweeps=4) as srv:
        t_bad = srv.submit(M, N, K, 31, max_iter=it, tol=0.0, X=Xneg)
        t_ok = srv.submit(M, N, K, 31, max_iter=it, tol=0.0, X=Xc)
        t_nan = srv.submit(M, N, K, 31, max_iter=it, tol=0.0, X=Xnan)
        t_gen = srv.submit(300, 2000, 8, 77, max_iter=5, tol=0.0)
        r_bad, r_ok, r_nan, r_gen = (srv.wait(t) for t in (t_bad, t_ok, t_nan, t_gen))
        B, C = srv.fetch(t_ok)
        with pytest.raises(did.DIDError) as e:
            srv.fetch(t_bad)
        assert e.value.status == did.DID_EINVAL
        st = srv.stats()
    assert r_bad["status"] == did.DID_EINVAL and r_nan["status"] == did.DID_EINVAL
    assert r_ok["status"] == did.DID_OK and r_gen["status"] == did.DID_OK
    assert st["failed"] == 2 and st["completed"] == 2
    B0, C0 = W.init_factors(M, N, K, 31)
    ref = O.factor(X, B0, C0, order="hals", max_iter=it, stop="none")
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    print("caller-supplied X vs oracle: relB %.3g relC %.3g" % (eB, eC))
    assert eB < 1e-4 and eC < 1e-4


def test_failed_admission_returns_its_budget(did):
    """A request larger than the GPU's memory (but within the budget) fails
    with DID_ENOMEM when its allocation is refused.  Its share of the budget
    must come back: the next request fits the budget only then, and admission
    is first come, first served, so a lost share would hold it forever."""
    import torch
    free, total = torch.cuda.mem_get_info()
    big = (4096, 11_000_000, 8)
    small = (4096, 500_000, 8)
    est = lambda m, n, k: m * n * 8 + k * n * 4 + m * k * 4      # X, R (float32), C, B
    if est(*big) <= total:
        pytest.skip("the GPU has more memory than the large request needs")
    budget = est(*big) + est(*small) // 2       # the small one fits only after the large one left
    with did.Server(budget, max_slots=4, round_sweeps=2) as srv:
        t_big = srv.submit(*big, 1, max_iter=2, tol=0.0)
        t_small = srv.submit(*small, 2, max_iter=2, tol=0.0)
        r_big = srv.wait(t_big, timeout_ms=120000)
        r_small = srv.wait(t_small, timeout_ms=120000)
        st = srv.stats()
    print("large request: status %d; small request: status %d, %d sweeps" % (r_big["status"], r_small["status"],
                                                                           r_small["iters"]))
    assert r_big["status"] == did.DID_ENOMEM
    assert r_small["status"] == did.DID_OK and r_small["iters"] == 2
    assert st["failed"] == 1 and st["completed"] == 1
