"""Buffer checks of the Python binding (no GPU needed).

Every buffer the library reads or writes is checked before the library is
called: a float32 (float64 for a trace) dense array with at least the elements
the call touches.  A buffer that fails raises DIDError(DID_EINVAL), so a wrong
dtype, a strided view or a short array can never reach the device.
"""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def did():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_08938_gb300 as did
    return did


def test_dense_float32_buffers_pass(did):
    a = np.zeros((7, 5), np.float32)
    assert did._buf(a, 35, "a") == a.ctypes.data
    f = np.asfortranarray(np.zeros((5, 7), np.float32))     # column-major, still dense
    assert did._buf(f, 35, "f") == f.ctypes.data
    assert did._buf(None, 10, "none") is None
    assert did._buf(1234, 10, "address") == 1234              # a raw address is the caller's
    assert did._buf(np.zeros(3, np.float64), 3, "trace", "float64") is not None


def test_torch_buffers(did):
    torch = pytest.importorskip("torch")
    t = torch.zeros((6, 4), dtype=torch.float32)
    assert did._buf(t, 24, "t") == t.data_ptr()
    assert did._buf(t.t(), 24, "t.T") == t.data_ptr()          # a transposed dense tensor
    with pytest.raises(did.DIDError) as e:
        did._buf(t[:, :2], 12, "strided")
    assert e.value.status == did.DID_EINVAL
    with pytest.raises(did.DIDError):
        did._buf(t.double(), 24, "float64")
    with pytest.raises(did.DIDError):
        did._buf(t, 25, "short")


@pytest.mark.parametrize("bad", ["float64", "strided", "short"])
def test_context_rejects_bad_x(did, bad):
    M, N, K = 6, 9, 2
    X = np.ones((N, M), np.float32)
    if bad == "float64":
        X = X.astype(np.float64)
    elif bad == "strided":
        X = np.ones((N, 2 * M), np.float32)[:, ::2]
    else:
        X = X[:-1]
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K)
    assert e.value.status == did.DID_EINVAL


def test_context_rejects_bad_start_point(did):
    M, N, K = 6, 9, 2
    X = np.ones((N, M), np.float32)
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K, B_init=np.ones((K, M - 1), np.float32))
    assert e.value.status == did.DID_EINVAL
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K, C_init=np.ones((K, N), np.float64))
    assert e.value.status == did.DID_EINVAL


def test_static_sweep_and_generators_check_sizes(did):
    M, N, K, ld = 8, 5, 2, 8
    R = np.zeros((N, ld), np.float32)
    B = np.zeros((K, ld), np.float32)
    C = np.zeros((K, N), np.float32)
    with pytest.raises(did.DIDError) as e:
        did.did_sweep_static(R[:-1], ld, B, C, M, N, K, 3)
    assert e.value.status == did.DID_EINVAL
    with pytest.raises(did.DIDError):
        did.did_sweep_static(R, ld, B, C, M, N, K, 3, trace=np.zeros(3, np.float32))   # trace is float64
    with pytest.raises(did.DIDError):
        did.did_sweep_static(R, ld, B, C, M, N, K, 3, trace=np.zeros(2, np.float64))   # one per sweep
    with pytest.raises(did.DIDError):
        did.did_generate_uniform(np.zeros(9, np.float32), 10, 1, 0)
    with pytest.raises(did.DIDError):
        did.did_generate_image(np.zeros((N, M - 1), np.float32), M, N, 1)


def test_transposed_layout_is_refused(did):
    """X is M x N column-major: a C-contiguous (M, N) array would be read
    transposed, so it is refused; (N, M) C-contiguous and (M, N) Fortran-order
    pass.  The same holds for B (M x K column-major) and C (K x N row-major)."""
    M, N, K = 6, 9, 2
    with pytest.raises(did.DIDError) as e:
        did.Context(np.ones((M, N), np.float32), M, N, K)
    assert e.value.status == did.DID_EINVAL
    assert did._buf(np.ones((N, M), np.float32), M * N, "X", mem=(N, M)) is not None
    assert did._buf(np.asfortranarray(np.ones((M, N), np.float32)), M * N, "X", mem=(N, M)) is not None
    X = np.ones((N, M), np.float32)
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K, B_init=np.ones((M, K), np.float32))      # B as row-major M x K
    assert e.value.status == did.DID_EINVAL
    with pytest.raises(did.DIDError) as e:
        did.Context(X, M, N, K, C_init=np.ones((N, K), np.float32))      # C as column-major K x N
    assert e.value.status == did.DID_EINVAL
    torch = pytest.importorskip("torch")
    with pytest.raises(did.DIDError):
        did._buf(torch.ones((M, N)), M * N, "X", mem=(N, M))
    with pytest.raises(did.DIDError):
        did._buf(torch.ones((M, N)).t(), M * N, "X", mem=(N, M))     # (N, M) view of row-major (M, N) memory
    assert did._buf(torch.ones((N, M)).t(), M * N, "X", mem=(N, M)) is not None
