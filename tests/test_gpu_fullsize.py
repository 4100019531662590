"""The full-size workloads in the launch configuration the benchmark times.

The oracle cannot run these sizes in test time, so the checks are properties
that hold at any size, each evaluated in float64 on the host:
  * the objective trace does not increase (every block step is an exact
    minimiser, Section 2);
  * R == X - B C on sampled columns (the incremental residual update);
  * the block updated last in a sweep, c_K, is a fixed point of its own closed
    form c_K = [b_K^T (R + b_K c_K) / ||b_K||^2]_+ on sampled columns;
  * the exact f(B, C) equals the trace value 1/2 ||R||^2;
  * two runs are bitwise equal.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def generate(did, M, N, K, kind):
    X = torch.empty((N, M), dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    if kind == "planted_exp":
        did.did_generate_planted(X, M, N, K, 0, coords=1, zero_frac=0.3, sigma=0.05, salt_frac=0.0, salt_value=5.0,
                                 stream=st)
    else:
        did.did_generate_image(X, M, N, 0, 0.8, stream=st)
    torch.cuda.synchronize()
    return X, st


def run(did, X, M, N, K, st, sweeps, **kw):
    with did.Context(X, M, N, K, seed=0, stream=st, **kw) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return dict(B=B, C=C, trace=ctx.trace(), f=ctx.objective(), info=ctx.info(), R=ctx.residual())


def check_properties(X, out, M, tol_r, tol_fix, tol_f, label):
    B = out["B"].astype(np.float64)
    C = out["C"].astype(np.float64)
    t = out["trace"]
    rs = np.random.default_rng(0)
    cols = np.sort(rs.choice(C.shape[1], 256, replace=False))
    Xs = X[torch.as_tensor(cols, device=X.device)].cpu().numpy().astype(np.float64).T     # M x 256
    Rs = out["R"][:, cols].astype(np.float64)
    Rd = Xs - B @ C[:, cols]
    # The rounding of the incremental updates stays in R even where the final
    # factors have become exactly zero, so the error of an entry is measured
    # against the largest |X| + sum |B||C| of its column.
    scale = (np.abs(Xs) + np.abs(B) @ np.abs(C[:, cols])).max(axis=0, keepdims=True)
    err_r = float(np.max(np.abs(Rs - Rd) / scale))
    # last block of the sweep: c_K at its own closed form
    bK = B[:, -1]
    cK = C[-1, cols]
    bb = float(bK @ bK)
    cK_star = np.maximum((bK @ (Rs + np.outer(bK, cK))) / bb, 0.0)
    fix_scale = (np.abs(bK) @ (np.abs(Rs) + np.abs(np.outer(bK, cK)))) / bb
    err_fix = float(np.max(np.abs(cK - cK_star) / (fix_scale + 1e-30)))
    err_f = abs(out["f"] - t[-1]) / t[-1]
    rises = np.diff(t) / t[:-1]
    print("%s: trace %.6g -> %.6g, max rise %.3g, R err %.3g, c_K fixed-point err %.3g, f vs trace %.3g, lazy %d "
          "pairs %d units %d" % (label, t[0], t[-1], rises.max(), err_r, err_fix, err_f,
                                 out["info"]["lazy_writeback"], out["info"]["column_pairs"], out["info"]["column_units"]))
    assert rises.max() <= 1e-6
    assert err_r <= tol_r
    assert err_fix <= tol_fix
    assert err_f <= tol_f
    assert B.min() >= 0 and C.min() >= 0


def test_planted_exp_5000x200000_k50_fp32(did):
    M, N, K = 5000, 200000, 50
    X, st = generate(did, M, N, K, "planted_exp")
    a = run(did, X, M, N, K, st, 12, refresh_every=10)
    assert a["info"]["lazy_writeback"] == 1 and a["info"]["dynamic_units"] == 1 and a["info"]["tc_refreshes"] == 2
    check_properties(X, a, M, tol_r=2.0 ** -16, tol_fix=1e-5, tol_f=1e-5, label="fp32 5000x200000x50")
    b = run(did, X, M, N, K, st, 12, refresh_every=10)
    assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["C"], b["C"])


def test_planted_exp_5000x200000_k50_bf16r(did):
    M, N, K = 5000, 200000, 50
    X, st = generate(did, M, N, K, "planted_exp")
    a = run(did, X, M, N, K, st, 12, refresh_every=10, precision=did.DID_BF16R)
    # R is stored in bfloat16: each of the 2 K updates since the refresh (two
    # sweeps) rounds it by half an ulp (2^-9), a random walk bounded as in the
    # bfloat16 tests by 4 sqrt(updates) 2^-9
    check_properties(X, a, M, tol_r=4.0 * np.sqrt(2 * K) * 2.0 ** -9, tol_fix=1e-2, tol_f=2e-2,
                     label="bf16r 5000x200000x50")


def test_image_like_784x70000_k16_fp32(did):
    M, N, K = 784, 70000, 16
    X, st = generate(did, M, N, K, "image")
    a = run(did, X, M, N, K, st, 30, init_scale=True)
    check_properties(X, a, M, tol_r=2.0 ** -16, tol_fix=1e-5, tol_f=1e-5, label="fp32 784x70000x16")


def check_batched(X, out, tol_r, tol_fix, tol_f, label):
    """The batched order (C step, then B step): the last block of a sweep is
    b_K, at its own closed form b_K = [b_K + R c_K^T / ||c_K||^2]_+ on sampled
    rows of the true residual; R == X - B C on sampled columns; f(B, C) equals
    the trace value; the trace does not rise."""
    B = out["B"].astype(np.float64)
    C = out["C"].astype(np.float64)
    R = out["R"]
    t = out["trace"]
    rs = np.random.default_rng(1)
    cols = np.sort(rs.choice(C.shape[1], 256, replace=False))
    Xs = X[torch.as_tensor(cols, device=X.device)].cpu().numpy().astype(np.float64).T
    Rs = R[:, cols].astype(np.float64)
    scale = (np.abs(Xs) + np.abs(B) @ np.abs(C[:, cols])).max(axis=0, keepdims=True)
    err_r = float(np.max(np.abs(Rs - (Xs - B @ C[:, cols])) / scale))
    rows = np.sort(rs.choice(B.shape[0], 64, replace=False))
    cK = C[-1]
    cc = float(cK @ cK)
    Rr = R[rows].astype(np.float64)                      # 64 full rows
    bK = B[rows, -1]
    bK_star = np.maximum(bK + (Rr @ cK) / cc, 0.0)
    fix_scale = (np.abs(Rr) @ np.abs(cK)) / cc + np.abs(bK)
    err_fix = float(np.max(np.abs(bK - bK_star) / (fix_scale + 1e-30)))
    err_f = abs(out["f"] - t[-1]) / t[-1]
    rises = np.diff(t) / t[:-1]
    print("%s: trace %.6g -> %.6g, max rise %.3g, R err %.3g, b_K fixed-point err %.3g, f vs trace %.3g"
          % (label, t[0], t[-1], rises.max(), err_r, err_fix, err_f))
    assert rises.max() <= 1e-6
    assert err_r <= tol_r
    assert err_fix <= tol_fix
    assert err_f <= tol_f
    assert B.min() >= 0 and C.min() >= 0


def test_planted_exp_5000x200000_k50_batched(did):
    """The batched order at the size and cadence its benchmark line runs."""
    M, N, K = 5000, 200000, 50
    X, st = generate(did, M, N, K, "planted_exp")
    a = run(did, X, M, N, K, st, 12, refresh_every=10, order=did.DID_ORDER_DID_BATCHED)
    check_batched(X, a, tol_r=2.0 ** -16, tol_fix=1e-5, tol_f=1e-5, label="batched 5000x200000x50")
    b = run(did, X, M, N, K, st, 12, refresh_every=10, order=did.DID_ORDER_DID_BATCHED)
    assert np.array_equal(a["B"], b["B"]) and np.array_equal(a["C"], b["C"])


def test_image_like_784x70000_k16_batched(did):
    M, N, K = 784, 70000, 16
    X, st = generate(did, M, N, K, "image")
    a = run(did, X, M, N, K, st, 30, init_scale=True, order=did.DID_ORDER_DID_BATCHED)
    check_batched(X, a, tol_r=2.0 ** -16, tol_fix=1e-5, tol_f=1e-5, label="batched 784x70000x16")
