"""did_sweep_static: the sweep for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc where they run (inside another runtime's
allocator hooks, or under a device memory budget fixed up front); this entry
point keeps its scratch in a static device array instead.  The tests call it
through the C ABI on caller-owned buffers and check it against the regular
context path (did_create + did_sweep) on two calls in a row, against the FP64
oracle directly, with padding rows (ld > M), at a leading dimension near the
documented limit, and check that a host buffer is refused before any launch.
The file is collected last and needs nothing from the other tests.
"""

import numpy as np
import pytest

from oracle import did_oracle as O
from synth import workloads as W

pytestmark = pytest.mark.gpu

TOL_FACTOR = 1e-4
TOL_OBJ = 1e-5
# The caller's R after the sweeps against X - B C of the returned factors,
# relative to ||X||: float32 rounding of the incremental updates.
TOL_RESIDUAL = 1e-5


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def caller_buffers(X, B0, C0, ld):
    """R = X - B C, B and C as caller-owned device buffers with leading
    dimension ld (rows M..ld-1 of R and B zero)."""
    import torch
    M, N = X.shape
    K = B0.shape[1]
    R = np.zeros((N, ld), np.float32)                     # ld x N column-major
    R[:, :M] = O.residual(X, B0, C0).T.astype(np.float32)
    Bt = np.zeros((K, ld), np.float32)                    # ld x K column-major
    Bt[:, :M] = np.asarray(B0, np.float32).T
    return (torch.from_numpy(R).cuda(), torch.from_numpy(Bt).cuda(),
            torch.from_numpy(np.ascontiguousarray(C0, dtype=np.float32)).cuda())


def check_against_context(did, M, N, K, seed, ld, calls):
    import torch
    X, _, _ = W.planted(M, N, K, seed, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, seed)
    Xc = np.ascontiguousarray(X.T)
    Bc = np.ascontiguousarray(np.asarray(B0, np.float32).T)
    with did.Context(Xc, M, N, K, B_init=Bc, C_init=np.asarray(C0, np.float32)) as ref:
        Rd = torch.zeros((N, ld), device="cuda")
        Rm = torch.empty((N, M), device="cuda")
        did.did_get_residual(ref.h, Rm)                    # the context's R = X - B C
        Rd[:, :M] = Rm
        Bd = torch.zeros((K, ld), device="cuda")
        Bd[:, :M] = torch.from_numpy(Bc).cuda()
        Cd = torch.from_numpy(np.ascontiguousarray(C0, dtype=np.float32)).cuda()
        done = 0
        for n in calls:                                   # calls in a row
            trace = np.zeros(n, np.float64)
            did.did_sweep_static(Rd, ld, Bd, Cd, M, N, K, n, trace)
            torch.cuda.synchronize()
            ref.sweep(n)
            done += n
            B_ref, C_ref = ref.factors()
            t_ref = ref.trace()[done - n + 1: done + 1]
            B = Bd.cpu().numpy().T
            C = Cd.cpu().numpy()
            R = Rd.cpu().numpy().T
            eB, eC = rel_fro(B[:M], B_ref), rel_fro(C, C_ref)
            eF = float(np.max(np.abs(trace - t_ref) / t_ref))
            # R against X - B C of the returned factors, and the padding rows
            Xr = np.asarray(X, np.float64) - B[:M].astype(np.float64) @ C.astype(np.float64)
            eR = float(np.linalg.norm(R[:M] - Xr) / np.linalg.norm(X))
            print("static M=%d ld=%d after %d: relB=%.3g relC=%.3g relf=%.3g |R-(X-BC)|/|X|=%.3g"
                  % (M, ld, done, eB, eC, eF, eR))
            assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ
            assert eR <= TOL_RESIDUAL
            assert B.min() >= 0 and C.min() >= 0
            assert not np.any(R[M:]) and not np.any(B[M:])


def test_static_sweep_matches_context_path(did):
    check_against_context(did, 200, 1000, 10, 21, 200, (3, 2))


def test_static_sweep_padded_rows(did):
    """M not a multiple of 4: ld = 200 > M = 198, padding rows of R and B zero."""
    check_against_context(did, 198, 1500, 7, 22, 200, (2, 3))


def test_static_sweep_large_ld(did):
    """Two calls at ld = 4096, half the documented 8192-row limit."""
    check_against_context(did, 4093, 3000, 12, 23, 4096, (2, 2))


def test_static_sweep_matches_oracle(did):
    """Against the FP64 oracle's HALS sweeps directly: 20 sweeps in two calls."""
    import torch
    M, N, K, seed = 300, 2000, 8, 24
    X, _, _ = W.planted(M, N, K, seed, sigma=0.01)
    B0, C0 = W.init_factors(M, N, K, seed)
    ref = O.factor(X, B0, C0, order="hals", max_iter=20, stop="none")
    Rd, Bd, Cd = caller_buffers(X, B0, C0, M)
    tr = np.zeros(20, np.float64)
    did.did_sweep_static(Rd, M, Bd, Cd, M, N, K, 12, tr[:12])
    did.did_sweep_static(Rd, M, Bd, Cd, M, N, K, 8, tr[12:])
    torch.cuda.synchronize()
    B, C = Bd.cpu().numpy().T, Cd.cpu().numpy()
    eB, eC = rel_fro(B, ref["B"]), rel_fro(C, ref["C"])
    eF = float(np.max(np.abs(tr - ref["trace"][1:]) / ref["trace"][1:]))
    print("static vs oracle after 20 sweeps: relB=%.3g relC=%.3g relf(max over sweeps)=%.3g" % (eB, eC, eF))
    assert eB <= TOL_FACTOR and eC <= TOL_FACTOR and eF <= TOL_OBJ


def test_static_sweep_rejects_host_buffers(did):
    """A host buffer is refused on the host (DID_EINVAL); nothing is launched."""
    import torch
    M, N, K = 16, 32, 2
    Rh = np.zeros((N, M), np.float32)
    Bd = torch.zeros((K, M), device="cuda")
    Cd = torch.zeros((K, N), device="cuda")
    Rd = torch.zeros((N, M), device="cuda")
    for args in ((Rh, Bd, Cd), (Rd, Bd.cpu().numpy(), Cd), (Rd, Bd, Cd.cpu().numpy())):
        with pytest.raises(did.DIDError) as e:
            did.did_sweep_static(args[0], M, args[1], args[2], M, N, K, 1)
        assert e.value.status == did.DID_EINVAL
    # the device buffers themselves are accepted afterwards
    did.did_sweep_static(Rd, M, Bd, Cd, M, N, K, 0)


def test_static_sweep_rejects_oversize(did):
    import torch
    R = torch.zeros((4, 8200), device="cuda")
    B = torch.zeros((1, 8200), device="cuda")
    C = torch.zeros((1, 4), device="cuda")
    with pytest.raises(did.DIDError) as e:
        did.did_sweep_static(R, 8200, B, C, 8200, 4, 1, 1)
    assert e.value.status == did.DID_E_TOO_LARGE
    with pytest.raises(did.DIDError) as e:
        did.did_sweep_static(R, 8198, B, C, 8198, 4, 1, 1)     # ld not a multiple of 4
    assert e.value.status == did.DID_EINVAL
