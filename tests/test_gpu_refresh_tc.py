"""Tensor-core refresh (tcgen05): BF16x3 for a bfloat16 residual, BF16x6 for a float32 one.

R = X - B C from three bfloat16 products with float32 accumulation must equal
the exact X - B C up to (a) the dropped Bl Cl term and the float32
accumulation, about 2^-16 |B||C| per entry, and (b) the final rounding of R
to bfloat16 (half an ulp, 2^-9 |R|).  It is compared with the float64 product
on the host and with the float32 SIMT refresh of the same factors.
"""

import numpy as np
import pytest

from synth import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def bf16_round(x):
    """Round float32 values to bfloat16 (nearest even) and back, on the host."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (1000, 3000, 100), (517, 777, 64), (128, 64, 16),
                                   (5000, 2100, 50), (128, 130, 128)])
def test_tensor_core_refresh_matches_product(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=M + N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 7)
    Xc = np.ascontiguousarray(X.T)
    kw = dict(B_init=np.ascontiguousarray(B0.T), C_init=C0, precision=did.DID_BF16R)
    with did.Context(Xc, M, N, K, **kw) as tc, did.Context(Xc, M, N, K, flags=did.DID_FLAG_SIMT_REFRESH, **kw) as simt:
        info = tc.info()
        R_tc = tc.residual()
        R_simt = simt.residual()
        f_tc, f_simt = tc.trace()[0], simt.trace()[0]
    assert info["tc_refreshes"] == 1
    P = B0.astype(np.float64) @ C0.astype(np.float64)
    R_exact = X.astype(np.float64) - P
    # (a) product error of BF16x3 with float32 accumulation, (b) bfloat16 rounding of R
    bound = 2.0 ** -15 * (np.abs(B0).astype(np.float64) @ np.abs(C0).astype(np.float64)) + 2.0 ** -8 * np.abs(R_exact)
    err = np.abs(R_tc.astype(np.float64) - R_exact)
    print("M=%d N=%d K=%d: max err %.3g, max err/bound %.3g, bf16 entries equal to SIMT %.4f, f %.8g vs %.8g"
          % (M, N, K, err.max(), (err / bound).max(), np.mean(R_tc == R_simt), f_tc, f_simt))
    assert np.all(err <= bound)
    # rounding the exact residual to bfloat16 gives the same values except at near-ties
    assert np.mean(R_tc == bf16_round(R_exact.astype(np.float32))) > 0.95
    assert abs(f_tc - f_simt) <= 1e-3 * f_simt


def test_tensor_core_refresh_in_a_bf16_run(did):
    """A BF16-R run refreshing every 2 sweeps on the tensor cores matches the SIMT-refresh run."""
    M, N, K = 600, 4000, 24
    X, _, _ = W.planted(M, N, K, seed=3, sigma=0.01)
    Xc = np.ascontiguousarray(X.T)
    out = []
    for flags in (0, did.DID_FLAG_SIMT_REFRESH):
        with did.Context(Xc, M, N, K, seed=3, precision=did.DID_BF16R, refresh_every=2, flags=flags) as ctx:
            ctx.sweep(10)
            out.append((ctx.objective(), ctx.info()["tc_refreshes"]))
    (f_tc, n_tc), (f_simt, n_simt) = out
    print("BF16-R 10 sweeps: f(tc refresh)=%.8g f(simt refresh)=%.8g, tc refreshes %d" % (f_tc, f_simt, n_tc))
    assert n_tc == 5 and n_simt == 0
    assert abs(f_tc - f_simt) <= 1e-3 * f_simt


# ------------------------------------------------- BF16x6 (float32 residual)
@pytest.mark.parametrize("M,N,K", [(200, 1000, 10), (517, 777, 64), (128, 64, 16), (5000, 2100, 50), (129, 130, 64),
                                   (300, 500, 3)])
def test_tensor_core_refresh_fp32_matches_product(did, M, N, K):
    """BF16x6: each float32 operand as three bfloat16 terms and the six
    products whose terms reach 2^-18 of the leading one, accumulated in
    float32: a product is off by about 2^-26 relative, and the float32
    accumulation of the 6 Kp / 16 MMAs adds at most about 2^-18 of sum |B||C|;
    the bound below allows 2^-17 of it."""
    X, _, _ = W.planted(M, N, K, seed=2 * M + N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 9)
    Xc = np.ascontiguousarray(X.T)
    kw = dict(B_init=np.ascontiguousarray(B0.T), C_init=C0)
    with did.Context(Xc, M, N, K, **kw) as tc, did.Context(Xc, M, N, K, flags=did.DID_FLAG_SIMT_REFRESH, **kw) as simt:
        info = tc.info()
        R_tc = tc.residual().astype(np.float64)
        R_simt = simt.residual().astype(np.float64)
        f_tc, f_simt = tc.trace()[0], simt.trace()[0]
        assert simt.info()["tc_refreshes"] == 0
    assert info["tc_refreshes"] == 1
    absP = np.abs(B0).astype(np.float64) @ np.abs(C0).astype(np.float64)
    R_exact = X.astype(np.float64) - B0.astype(np.float64) @ C0.astype(np.float64)
    bound = 2.0 ** -17 * absP + 2.0 ** -22 * np.abs(R_exact)
    err = np.abs(R_tc - R_exact)
    print("BF16x6 M=%d N=%d K=%d: max err/|BC| %.3g, max err/bound %.3g, SIMT max err/|BC| %.3g, f rel %.3g"
          % (M, N, K, (err / absP).max(), (err / bound).max(), (np.abs(R_simt - R_exact) / absP).max(),
             abs(f_tc - f_simt) / f_simt))
    assert np.all(err <= bound)
    # the objective of the refreshed residual, from the elementwise bound
    f_exact = 0.5 * float(np.sum(R_exact ** 2))
    assert abs(f_tc - f_exact) <= float(np.sum(bound * (np.abs(R_exact) + 0.5 * bound)))
    assert abs(f_tc - f_simt) <= 1e-5 * f_simt      # the FP32 objective tolerance


def test_fp32_refresh_above_k64_is_simt(did):
    M, N, K = 300, 400, 100
    X, _, _ = W.planted(M, N, K, seed=5, sigma=0.01)
    with did.Context(np.ascontiguousarray(X.T), M, N, K, seed=5) as ctx:
        assert ctx.info()["tc_refreshes"] == 0


def test_tensor_core_refresh_in_an_fp32_run(did):
    """An FP32 run refreshing every 2 sweeps on the tensor cores stays within
    the FP32 parity tolerances of the oracle (refreshes do not change the
    iterates in exact arithmetic)."""
    from oracle import did_oracle as O
    M, N, K = 600, 4000, 24
    X, _, _ = W.planted(M, N, K, seed=3, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 3)
    ref = O.factor(X, B0, C0, order="hals", max_iter=20, stop="none")
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(B0.T), C_init=C0,
                     refresh_every=2) as ctx:
        ctx.sweep(20)
        B, C = ctx.factors()
        t = ctx.trace()
        n_tc = ctx.info()["tc_refreshes"]
    eB = np.linalg.norm(B - ref["B"]) / np.linalg.norm(ref["B"])
    eF = float(np.max(np.abs(t - ref["trace"]) / ref["trace"]))
    print("FP32 20 sweeps, BF16x6 refresh every 2: tc refreshes %d, relB %.3g, max relf %.3g" % (n_tc, eB, eF))
    assert n_tc == 10
    assert eB <= 1e-4 and eF <= 1e-5


@pytest.mark.parametrize("precision", ["fp32", "bf16r"])
@pytest.mark.parametrize("M,N,K", [(300, 50, 4), (517, 777, 16), (1000, 20000, 20), (130, 3, 3)])
def test_refresh_forms_first_partials(did, M, N, K, precision):
    """The tensor-core refresh also forms the partials of R c_1^T for the next
    sweep's first b-update (no prologue pass over R).  A run with a refresh
    before sweeps 1, 3 and 5 matches the oracle's interleaved sweeps and the
    SIMT-refresh run, which re-forms those partials in a prologue pass.  N = 50
    and N = 3 leave most CTAs of the refresh without a column tile."""
    from oracle import did_oracle as O
    X, _, _ = W.planted(M, N, K, seed=3 * M + N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 5)
    Xc = np.ascontiguousarray(X.T)
    prec = did.DID_FP32 if precision == "fp32" else did.DID_BF16R
    kw = dict(B_init=np.ascontiguousarray(B0.T), C_init=C0, precision=prec, refresh_every=2)
    with did.Context(Xc, M, N, K, **kw) as tc, did.Context(Xc, M, N, K, flags=did.DID_FLAG_SIMT_REFRESH, **kw) as simt:
        tc.sweep(5)
        simt.sweep(5)
        i_tc, i_simt = tc.info(), simt.info()
        B, C = tc.factors()
        Bs, Cs = simt.factors()
    assert i_tc["tc_refreshes"] == 3 and i_tc["prologue_launches"] == 0
    assert i_simt["tc_refreshes"] == 0 and i_simt["prologue_launches"] == 3
    ref = O.factor(X, B0, C0, order="hals", max_iter=5, stop="none")

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))
    eB, eC = rel(B, ref["B"]), rel(C, ref["C"])
    dB, dC = rel(B, Bs.astype(np.float64)), rel(C, Cs.astype(np.float64))
    print("%s M=%d N=%d K=%d: vs oracle B %.3g C %.3g, vs SIMT-refresh run B %.3g C %.3g"
          % (precision, M, N, K, eB, eC, dB, dC))
    # float32: within the parity bound; a bfloat16 residual rounds each stored
    # entry by half an ulp (2^-9), which the oracle does not
    tol = 1e-4 if precision == "fp32" else 4e-3
    assert eB <= tol and eC <= tol
    assert dB <= tol and dC <= tol
