"""did_sweep_static: the sweep for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they run (inside another runtime's
allocator hooks, or under a device memory budget fixed up front); this entry
point keeps its scratch in a static device array instead.  The test calls it
through the C ABI on caller-owned buffers and checks it against the regular
context path (did_create + did_sweep) on two calls in a row.  It lives in its
own file, collected last, and needs nothing from the other tests.
"""

import numpy as np
import pytest

from synth import workloads as W

pytestmark = pytest.mark.gpu

TOL_FACTOR = 1e-4
TOL_OBJ = 1e-5


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_sweep_matches_context_path():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did

    M, N, K = 200, 1000, 10            # M is a multiple of 4: ld = M, no padding rows
    X, _, _ = W.planted(M, N, K, 21, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, 21)
    Xc = np.ascontiguousarray(X.T)
    Bc = np.ascontiguousarray(B0.T)

    with did.Context(Xc, M, N, K, B_init=Bc, C_init=C0) as ref:
        Rd = torch.empty((N, M), device="cuda")          # caller-owned residual, ld = M
        did.did_get_residual(ref.h, Rd)
        Bd = torch.from_numpy(Bc).cuda()                  # ld x K column-major
        Cd = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
        done = 0
        for n in (3, 2):                                  # two calls in a row
            trace = np.zeros(n, np.float64)
            did.did_sweep_static(Rd, M, Bd, Cd, M, N, K, n, trace)
            torch.cuda.synchronize()
            ref.sweep(n)
            done += n
            B_ref, C_ref = ref.factors()
            t_ref = ref.trace()[done - n + 1: done + 1]
            B = Bd.cpu().numpy().T
            C = Cd.cpu().numpy()
            R = Rd.cpu().numpy().T
            eB, eC = rel_fro(B, B_ref), rel_fro(C, C_ref)
            eR = rel_fro(R, ref.residual())
            eF = float(np.max(np.abs(trace - t_ref) / t_ref))
            print("static sweep after %d: relB=%.3g relC=%.3g relR=%.3g relf=%.3g" % (done, eB, eC, eR, eF))
            assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ
            assert eR <= 1e-3
            assert B.min() >= 0 and C.min() >= 0


def test_static_sweep_rejects_oversize():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did

    R = torch.zeros((4, 8200), device="cuda")
    B = torch.zeros((1, 8200), device="cuda")
    C = torch.zeros((1, 4), device="cuda")
    with pytest.raises(did.DIDError) as e:
        did.did_sweep_static(R, 8200, B, C, 8200, 4, 1, 1)
    assert e.value.status == did.DID_E_TOO_LARGE
    with pytest.raises(did.DIDError) as e:
        did.did_sweep_static(R, 8198, B, C, 8198, 4, 1, 1)     # ld not a multiple of 4
    assert e.value.status == did.DID_EINVAL
