"""Tensor-core refresh (tcgen05, BF16x3) of a bfloat16 residual.

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
