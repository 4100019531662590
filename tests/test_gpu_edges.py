"""Edge cases of every block order and precision: one row, one column, K equal
to both dimensions, and empty or inconsistent sizes (rejected on the host)."""

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(1, 40, 1), (40, 1, 1), (5, 5, 5), (3, 2, 2), (17, 33, 16), (130, 3, 3)]
# f(B, C) evaluated from the factors with float32 products carries about
# u |x| (u = 2^-24) per entry, so at an exact fit it cannot resolve below
# ~u^2 ||X||^2 = 3.6e-15 ||X||^2: its error is taken relative to
# max(f, 1e-8 ||X||^2), which leaves the 1e-5 tolerance above that limit.
F_FLOOR = 1e-8


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def objective_ok(X, B, C, ref, tol):
    """f(B, C) against the oracle's: within tol relative (against
    max(f, F_FLOOR ||X||^2)), or -- near an exact fit, where a relative error
    of f magnifies the factors' rounding -- within twice the first-order
    bound ||R|| ||d|| + ||d||^2 / 2 that the factor difference d = BC - (BC)_ref
    allows, plus the float32 evaluation floor."""
    X64 = X.astype(np.float64)
    f = 0.5 * float(np.sum((X64 - B.astype(np.float64) @ C.astype(np.float64)) ** 2))
    f_ref = float(ref["trace"][-1])
    floor = F_FLOOR * float(np.sum(X64 ** 2))
    if abs(f - f_ref) <= tol * max(f_ref, floor):
        return True, abs(f - f_ref) / max(f_ref, floor)
    d = np.linalg.norm(B.astype(np.float64) @ C.astype(np.float64) - ref["B"] @ ref["C"])
    r = np.linalg.norm(X64 - ref["B"] @ ref["C"])
    allowed = 2.0 * (r * d + 0.5 * d * d) + 1e2 * 2.0 ** -48 * float(np.sum(X64 ** 2))
    return abs(f - f_ref) <= allowed, abs(f - f_ref) / max(f_ref, floor)


def run(did, X, B0, C0, sweeps, **kw):
    M, N = X.shape
    K = B0.shape[1]
    with did.Context(np.ascontiguousarray(X.T), M, N, K, B_init=np.ascontiguousarray(np.asarray(B0, np.float32).T),
                     C_init=np.ascontiguousarray(np.asarray(C0, np.float32)), **kw) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return B, C, ctx.trace(), ctx.objective()


@pytest.mark.parametrize("order", ["did", "did_batched"])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_c_first_orders_on_edge_shapes(did, M, N, K, order):
    X, _, _ = W.planted(M, N, K, seed=M + 3 * N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 4)
    ref = O.factor(X, B0, C0, order="did", max_iter=10, stop="none")
    code = did.DID_ORDER_DID if order == "did" else did.DID_ORDER_DID_BATCHED
    B, C, t, f = run(did, X, B0, C0, 10, order=code)
    ok, eF = objective_ok(X, B, C, ref, 1e-5)
    print("%s M=%d N=%d K=%d: relB %.3g relC %.3g relf %.3g" % (order, M, N, K, rel_fro(B, ref["B"]),
                                                             rel_fro(C, ref["C"]), eF))
    assert rel_fro(B, ref["B"]) <= 1e-4 and rel_fro(C, ref["C"]) <= 1e-4 and ok
    assert B.min() >= 0 and C.min() >= 0


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_bf16_residual_on_edge_shapes(did, M, N, K):
    X, _, _ = W.planted(M, N, K, seed=M + 5 * N, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 6)
    ref = O.factor(X, B0, C0, order="hals", max_iter=10, stop="none")
    B, C, t, f = run(did, X, B0, C0, 10, precision=did.DID_BF16R, refresh_every=3)
    ok, eF = objective_ok(X, B, C, ref, 1e-3)
    print("bf16 M=%d N=%d K=%d: f rel %.3g" % (M, N, K, eF))
    assert ok
    assert B.min() >= 0 and C.min() >= 0


@pytest.mark.parametrize("M,N,K", [(0, 10, 1), (10, 0, 1), (10, 10, 0), (10, 5, 6), (-1, 10, 1)])
def test_empty_or_inconsistent_sizes_rejected(did, M, N, K):
    X = np.ones((max(N, 1), max(M, 1)), np.float32)
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K)
    assert e.value.status in (did.DID_EINVAL, did.DID_E_TOO_LARGE)
