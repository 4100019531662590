"""BF16-residual mode: R stored in bfloat16, FP32 dots, FP64 norms and objective.

Target: the final objective within 1e-3 relative of the FP32 path (and of the
FP64 oracle) on identical seeds, with the dense refresh every 5 sweeps.
"""

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu

TOL_OBJ_BF16 = 1e-3


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def run(did, X, K, seed, sweeps, precision, refresh_every):
    M, N = X.shape
    with did.Context(np.ascontiguousarray(X.T), M, N, K, seed=seed, precision=precision,
                     refresh_every=refresh_every) as ctx:
        ctx.sweep(sweeps)
        B, C = ctx.factors()
        return B, C, ctx.trace(), ctx.objective(), ctx.residual()



@pytest.mark.parametrize("name,M,N,K,refresh", [
    ("salt_10000x500000_k100", 1000, 6000, 40, 5),
    ("planted_exp_5000x200000_k50", 500, 8000, 20, 10),
    ("planted_uniform_200x1000_k10", 200, 1000, 10, 5),
])
def test_bf16r_objective_matches_fp32_and_oracle(did, name, M, N, K, refresh):
    X, _, _, _ = W.make(name, seed=1, M=M, N=N, K=K)
    sweeps = 20
    B16, C16, t16, fx16, R16 = run(did, X, K, 1, sweeps, did.DID_BF16R, refresh)
    B32, C32, t32, fx32, _ = run(did, X, K, 1, sweeps, did.DID_FP32, refresh)
    B0, C0 = W.init_factors(M, N, K, 1)
    ref = O.factor(X, B0, C0, order="hals", max_iter=sweeps, stop="none")
    f_ref = ref["trace"][-1]
    # The target: the objective f(B, C) = 1/2 ||X - BC||^2 of the final factors.
    e32 = abs(fx16 - fx32) / fx32
    eor = abs(fx16 - f_ref) / f_ref
    # The trace monitor is 1/2 ||R||^2 of the stored bfloat16 residual; the
    # sweep minimises that rounded residual, so the monitor reads slightly high.
    etr = abs(t16[-1] - fx32) / fx32
    print("%s %dx%d K=%d: BF16-R f(B,C)=%.7g FP32 f(B,C)=%.7g oracle f=%.7g | rel vs FP32 %.2e, vs oracle "
          "%.2e | trace monitor rel %.2e | relB %.2e relC %.2e" % (
              name, M, N, K, fx16, fx32, f_ref, e32, eor, etr, rel_fro(B16, ref["B"]), rel_fro(C16, ref["C"])))
    assert e32 <= TOL_OBJ_BF16 and eor <= TOL_OBJ_BF16
    assert etr <= 2e-2
    assert B16.min() >= 0 and C16.min() >= 0
    # The kept residual drifts from X - BC by the bfloat16 roundings since the
    # last refresh: each entry is rounded (relative error <= 2^-9) at most
    # refresh * K times, which adds up like a random walk; allow 4 sigma.
    Rd = X.astype(np.float64) - B16.astype(np.float64) @ C16.astype(np.float64)
    drift = np.linalg.norm(R16 - Rd) / np.linalg.norm(Rd)
    bound = 4.0 * np.sqrt(refresh * K) * 2.0 ** -9
    print("residual drift %.3g (bound %.3g)" % (drift, bound))
    assert drift <= bound

