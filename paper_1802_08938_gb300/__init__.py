"""Python binding of the GB300 DID library (libdid.so, C ABI in include/did.h).

Argument marshalling only: every step of the factorisation runs in the CUDA
library.  Functions keep the C names (``did_create``, ``did_sweep`` ...);
``Context`` wraps a handle for convenience.  Arrays may be torch tensors (on
the GPU or pinned/pageable host memory) or NumPy arrays; their storage is
passed by pointer and must use the C ABI layouts:

* X: M x N column-major == a C-contiguous (N, M) array, or an F-contiguous (M, N) one
* B: M x K column-major == C-contiguous (K, M), or F-contiguous (M, K)
* C: K x N row-major    == C-contiguous (K, N), or F-contiguous (N, K)

A 2-D array of another shape (for instance X as a C-contiguous (M, N) array,
which would be read transposed) is refused with DIDError(DID_EINVAL).

There is no CPU fallback: importing this package without the built library
raises ImportError (build it with ``__graft_entry__.build()`` or
``python paper_1802_08938_gb300/_build.py``).
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdid.so")

DID_OK, DID_PENDING, DID_EINVAL, DID_ENOMEM, DID_ECUDA, DID_ETIMEOUT, DID_E_TOO_LARGE, DID_EBUSY = (
    0, 1, -1, -2, -3, -4, -5, -6)
DID_FP32, DID_BF16R = 0, 1
DID_ORDER_INTERLEAVED, DID_ORDER_DID, DID_ORDER_DID_BATCHED = 0, 1, 2
DID_STOP_RELCHANGE, DID_STOP_PAPER_EPS = 0, 1
DID_FLAG_PHASE_TIMES = 1
DID_FLAG_SIMT_REFRESH = 2
DID_FLAG_EAGER_WRITEBACK = 8
DID_FLAG_LAZY_WRITEBACK = 16
DID_FLAG_SINGLE_COLUMNS = 32


class did_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("refresh_every", ctypes.c_int32),
        ("stop", ctypes.c_int32),
        ("init_scale", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32),
        ("B_init", ctypes.c_void_p),
        ("C_init", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
        ("timeout_ns", ctypes.c_uint64),
        ("debug_barrier_extra", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("inner_c", ctypes.c_int32),
        ("inner_b", ctypes.c_int32),
    ]


class did_info(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("order", ctypes.c_int32),
        ("grid_ctas", ctypes.c_int32), ("group_threads", ctypes.c_int32),
        ("vecs_per_thread", ctypes.c_int32), ("column_units", ctypes.c_int32),
        ("dynamic_units", ctypes.c_int32), ("ld", ctypes.c_int64),
        ("sweeps_done", ctypes.c_int64), ("degenerate_events", ctypes.c_int64),
        ("refreshes", ctypes.c_int64), ("device_bytes", ctypes.c_size_t),
        ("sweep_launches", ctypes.c_int64), ("prologue_launches", ctypes.c_int64),
        ("sweep_kernel_ms", ctypes.c_double), ("dense_launches", ctypes.c_int64),
        ("dense_kernel_ms", ctypes.c_double), ("tc_refreshes", ctypes.c_int64),
        ("tc_refresh_ms", ctypes.c_double),
        ("lazy_writeback", ctypes.c_int32), ("ring_stages", ctypes.c_int32),
        ("column_pairs", ctypes.c_int32),
    ]


class did_request(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double)]


class did_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("obj", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class did_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("solves_per_s", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("peak_bytes", ctypes.c_size_t), ("peak_active", ctypes.c_int32), ("rounds", ctypes.c_int64),
                ("busy_s", ctypes.c_double)]


class DIDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_string(status), msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdid.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, U64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
    CTX = ctypes.c_void_p
    sig = {
        "did_default_options": (None, [ctypes.POINTER(did_options)]),
        "did_create": (I32, [P, I64, I64, I32, U64, ctypes.POINTER(CTX)]),
        "did_create_ex": (I32, [P, I64, I64, I32, U64, ctypes.POINTER(did_options), ctypes.POINTER(CTX)]),
        "did_sweep": (I32, [CTX, I32]),
        "did_sweep_static": (I32, [P, I64, P, P, I64, I64, I32, I32, P, P]),
        "did_factor": (I32, [CTX, I32, D, ctypes.POINTER(I32), ctypes.POINTER(D)]),
        "did_objective": (I32, [CTX, ctypes.POINTER(D)]),
        "did_residual_objective": (I32, [CTX, ctypes.POINTER(D)]),
        "did_refresh_residual": (I32, [CTX]),
        "did_get_factors": (I32, [CTX, P, P]),
        "did_set_factors": (I32, [CTX, P, P]),
        "did_get_residual": (I32, [CTX, P]),
        "did_get_trace": (I32, [CTX, ctypes.POINTER(D), I32, ctypes.POINTER(I32)]),
        "did_get_info": (I32, [CTX, ctypes.POINTER(did_info)]),
        "did_get_phase_times": (I32, [CTX, ctypes.POINTER(ctypes.c_uint64), I32, ctypes.POINTER(I32)]),
        "did_last_error": (ctypes.c_char_p, [CTX]),
        "did_status_string": (ctypes.c_char_p, [I32]),
        "did_destroy": (None, [CTX]),
        "did_generate_planted": (I32, [P, I64, I64, I32, U64, I32, D, D, D, D, P]),
        "did_generate_image": (I32, [P, I64, I64, U64, D, P]),
        "did_generate_uniform": (I32, [P, I64, U64, I32, P]),
        "did_server_create": (I32, [ctypes.c_size_t, I32, I32, I32, P, ctypes.POINTER(CTX)]),
        "did_server_submit": (I32, [CTX, ctypes.POINTER(did_request), ctypes.POINTER(U64)]),
        "did_server_poll": (I32, [CTX, U64, ctypes.POINTER(did_result)]),
        "did_server_wait": (I32, [CTX, U64, I32, ctypes.POINTER(did_result)]),
        "did_server_fetch": (I32, [CTX, U64, P, P]),
        "did_server_stats": (I32, [CTX, ctypes.POINTER(did_server_stats_t)]),
        "did_server_destroy": (None, [CTX]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def status_string(s):
    return _lib.did_status_string(int(s)).decode()


def _buf(a, n, what, dtype="float32", mem=None):
    """Address of a buffer the library reads or writes n elements of, after
    checking that it is a dense array of that dtype with at least n elements
    (a raw integer address is passed as it is; None passes NULL).  With
    mem = (outer, inner), a 2-D array must also have the memory order the C
    ABI wants: C-contiguous of shape (outer, inner), or its transpose in
    Fortran order (shape (inner, outer)).  So an M x N column-major matrix
    (mem = (N, M)) given as a C-contiguous (M, N) array is refused rather
    than read transposed.  A failed check raises DIDError(DID_EINVAL) before
    the library is called."""
    if a is None or isinstance(a, int):
        return a
    n = max(0, int(n))
    if hasattr(a, "data_ptr"):
        import torch
        want = torch.float32 if dtype == "float32" else torch.float64
        c_order = a.is_contiguous()
        f_order = a.dim() == 2 and a.t().is_contiguous()
        ok_type, size, shape = a.dtype == want, a.numel(), tuple(a.shape)
    elif isinstance(a, np.ndarray):
        c_order, f_order = a.flags.c_contiguous, a.ndim == 2 and a.flags.f_contiguous
        ok_type, size, shape = a.dtype == np.dtype(dtype), a.size, a.shape
    else:
        raise TypeError("%s: expected a torch tensor, NumPy array or address, got %r" % (what, type(a)))
    if not ok_type:
        raise DIDError(DID_EINVAL, "%s: expected %s elements, got %s" % (what, dtype, a.dtype))
    if not (c_order or f_order):
        raise DIDError(DID_EINVAL, "%s: expected a dense (contiguous) buffer" % what)
    if size < n:
        raise DIDError(DID_EINVAL, "%s: %d elements, the call needs %d" % (what, size, n))
    if mem is not None and len(shape) == 2:
        outer, inner = (int(v) for v in mem)
        if not ((c_order and shape == (outer, inner)) or (f_order and shape == (inner, outer))):
            raise DIDError(DID_EINVAL, "%s: expected a C-contiguous %s array (or its transpose in Fortran "
                                       "order), got shape %s" % (what, (outer, inner), shape))
    return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data


# (M, N, K) of each live context and of each served request, for the checks
# of the buffers passed to the calls that take only a handle (or a ticket).
_CTX_SHAPE = {}
_TICKET_SHAPE = {}


def _stream_of(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _check(status, ctx=None):
    if status != DID_OK:
        msg = _lib.did_last_error(ctx).decode() if ctx else ""
        raise DIDError(status, msg)


def default_options():
    o = did_options()
    _lib.did_default_options(ctypes.byref(o))
    return o


# ------------------------------------------------------------ C-named calls
def did_create(X, M, N, K, seed, options=None):
    h = ctypes.c_void_p()
    x = _buf(X, max(0, M) * max(0, N), "X", mem=(N, M))
    if options is None:
        st = _lib.did_create(x, M, N, K, seed, ctypes.byref(h))
    else:
        st = _lib.did_create_ex(x, M, N, K, seed, ctypes.byref(options), ctypes.byref(h))
    _check(st)
    _CTX_SHAPE[h.value] = (M, N, K)
    return h


did_create_ex = did_create


def did_sweep(h, n):
    _check(_lib.did_sweep(h, n), h)


def did_sweep_static(R, ld, B, C, M, N, K, n_sweeps, trace=None, stream=None):
    """Sweeps on caller-owned device buffers with no device allocation."""
    ldn, Nn, Kn = max(0, ld), max(0, N), max(0, K)
    _check(_lib.did_sweep_static(_buf(R, ldn * Nn, "R", mem=(N, ld)), ld, _buf(B, ldn * Kn, "B", mem=(K, ld)),
                                 _buf(C, Kn * Nn, "C", mem=(K, N)),
                                 M, N, K, n_sweeps, _buf(trace, n_sweeps, "trace", "float64"),
                                 _stream_of(stream)))


def did_factor(h, max_iter, tol):
    it = ctypes.c_int32()
    f = ctypes.c_double()
    _check(_lib.did_factor(h, max_iter, tol, ctypes.byref(it), ctypes.byref(f)), h)
    return it.value, f.value


def did_objective(h):
    f = ctypes.c_double()
    _check(_lib.did_objective(h, ctypes.byref(f)), h)
    return f.value


def did_residual_objective(h):
    f = ctypes.c_double()
    _check(_lib.did_residual_objective(h, ctypes.byref(f)), h)
    return f.value


def did_refresh_residual(h):
    _check(_lib.did_refresh_residual(h), h)


def _shape_of(h):
    return _CTX_SHAPE.get(h.value if hasattr(h, "value") else h, (0, 0, 0))


def did_get_factors(h, B, C):
    M, N, K = _shape_of(h)
    _check(_lib.did_get_factors(h, _buf(B, M * K, "B", mem=(K, M)), _buf(C, K * N, "C", mem=(K, N))), h)


def did_set_factors(h, B, C):
    M, N, K = _shape_of(h)
    _check(_lib.did_set_factors(h, _buf(B, M * K, "B", mem=(K, M)), _buf(C, K * N, "C", mem=(K, N))), h)


def did_get_residual(h, R):
    M, N, K = _shape_of(h)
    _check(_lib.did_get_residual(h, _buf(R, M * N, "R", mem=(N, M))), h)


def did_get_trace(h):
    n = ctypes.c_int32()
    _check(_lib.did_get_trace(h, None, 0, ctypes.byref(n)), h)
    buf = (ctypes.c_double * max(1, n.value))()
    _check(_lib.did_get_trace(h, buf, n.value, ctypes.byref(n)), h)
    return np.array(buf[: n.value], dtype=np.float64)


def did_get_info(h):
    i = did_info()
    _check(_lib.did_get_info(h, ctypes.byref(i)), h)
    return {k: getattr(i, k) for k, _ in did_info._fields_}


def did_get_phase_times(h):
    """Phase stamps of the last sweep launch as an (steps, 4) uint64 array (ns)."""
    n = ctypes.c_int32()
    _check(_lib.did_get_phase_times(h, None, 0, ctypes.byref(n)), h)
    buf = (ctypes.c_uint64 * max(1, n.value))()
    _check(_lib.did_get_phase_times(h, buf, n.value, ctypes.byref(n)), h)
    return np.array(buf[: n.value], dtype=np.uint64).reshape(-1, 4)


def did_destroy(h):
    _CTX_SHAPE.pop(h.value if hasattr(h, "value") else h, None)
    _lib.did_destroy(h)


def did_generate_planted(X_dev, M, N, K, seed, coords=0, zero_frac=0.0, sigma=0.0, salt_frac=0.0,
                         salt_value=5.0, stream=None):
    _check(_lib.did_generate_planted(_buf(X_dev, max(0, M) * max(0, N), "X", mem=(N, M)), M, N, K, seed, coords,
                                     zero_frac,
                                     sigma, salt_frac,
                                     salt_value, _stream_of(stream)))


def did_generate_image(X_dev, M, N, seed, zero_frac=0.8, stream=None):
    _check(_lib.did_generate_image(_buf(X_dev, max(0, M) * max(0, N), "X", mem=(N, M)), M, N, seed, zero_frac,
                                   _stream_of(stream)))


def did_generate_uniform(out_dev, n, seed, stream_id, stream=None):
    _check(_lib.did_generate_uniform(_buf(out_dev, n, "out"), n, seed, stream_id, _stream_of(stream)))


def did_server_create(hbm_budget_bytes, precision=DID_FP32, max_slots=64, round_sweeps=4, stream=None):
    h = ctypes.c_void_p()
    st = _lib.did_server_create(int(hbm_budget_bytes), precision, max_slots, round_sweeps,
                                stream if isinstance(stream, (int, type(None))) else stream.cuda_stream,
                                ctypes.byref(h))
    _check(st)
    return h


def did_server_submit(h, M, N, K, seed, max_iter, tol, X=None):
    r = did_request(_buf(X, max(0, M) * max(0, N), "X", mem=(N, M)), M, N, K, seed, max_iter, tol)
    t = ctypes.c_uint64()
    _check(_lib.did_server_submit(h, ctypes.byref(r), ctypes.byref(t)))
    _TICKET_SHAPE[(h.value, t.value)] = (M, N, K)
    return t.value


def _result_dict(st, r):
    return {"status": st, "iters": r.iters, "obj": r.obj, "t_submit": r.t_submit, "t_start": r.t_start,
            "t_done": r.t_done}


def did_server_poll(h, ticket):
    r = did_result()
    st = _lib.did_server_poll(h, ticket, ctypes.byref(r))
    return _result_dict(st, r)


def did_server_wait(h, ticket, timeout_ms=-1):
    r = did_result()
    st = _lib.did_server_wait(h, ticket, timeout_ms, ctypes.byref(r))
    return _result_dict(st, r)


def did_server_fetch(h, ticket, B, C):
    M, N, K = _TICKET_SHAPE.get((h.value, ticket), (0, 0, 0))
    _check(_lib.did_server_fetch(h, ticket, _buf(B, M * K, "B", mem=(K, M)), _buf(C, K * N, "C", mem=(K, N))))
    _TICKET_SHAPE.pop((h.value, ticket), None)      # results are released once fetched


def did_server_stats(h):
    s = did_server_stats_t()
    _check(_lib.did_server_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in did_server_stats_t._fields_}


def did_server_destroy(h):
    for key in [k for k in _TICKET_SHAPE if k[0] == h.value]:
        del _TICKET_SHAPE[key]
    _lib.did_server_destroy(h)


# --------------------------------------------------------------- convenience
class Context:
    """Owns one did_ctx.  X is M x N column-major (C-contiguous (N, M))."""

    def __init__(self, X, M, N, K, seed=0, precision=DID_FP32, order=DID_ORDER_INTERLEAVED,
                 refresh_every=0, stop=DID_STOP_RELCHANGE, init_scale=False, grid_ctas=0,
                 B_init=None, C_init=None, stream=None, timeout_ns=0, debug_barrier_extra=0, flags=0,
                 inner_c=1, inner_b=1):
        o = default_options()
        o.precision, o.order, o.refresh_every, o.stop = precision, order, refresh_every, stop
        o.init_scale, o.grid_ctas = int(bool(init_scale)), grid_ctas
        o.B_init = _buf(B_init, max(0, M) * max(0, K), "B_init", mem=(K, M))
        o.C_init = _buf(C_init, max(0, K) * max(0, N), "C_init", mem=(K, N))
        o.stream = _stream_of(stream)
        o.timeout_ns, o.debug_barrier_extra, o.flags = timeout_ns, debug_barrier_extra, flags
        o.inner_c, o.inner_b = inner_c, inner_b
        self.M, self.N, self.K = int(M), int(N), int(K)
        self._keep = (X, B_init, C_init)
        self.h = did_create(X, self.M, self.N, self.K, seed, o)
        self._keep = None

    def sweep(self, n=1):
        did_sweep(self.h, n)

    def factor(self, max_iter, tol):
        return did_factor(self.h, max_iter, tol)

    def objective(self):
        return did_objective(self.h)

    def residual_objective(self):
        return did_residual_objective(self.h)

    def refresh_residual(self):
        did_refresh_residual(self.h)

    def factors(self):
        """(B as (M, K) float32, C as (K, N) float32) NumPy arrays on the host."""
        Bt = np.empty((self.K, self.M), dtype=np.float32)    # column-major M x K
        C = np.empty((self.K, self.N), dtype=np.float32)
        did_get_factors(self.h, Bt, C)
        return Bt.T, C

    def set_factors(self, B, C):
        Bt = np.ascontiguousarray(np.asarray(B, np.float32).T)
        C = np.ascontiguousarray(np.asarray(C, np.float32))
        did_set_factors(self.h, Bt, C)

    def residual(self):
        Rt = np.empty((self.N, self.M), dtype=np.float32)
        did_get_residual(self.h, Rt)
        return Rt.T

    def trace(self):
        return did_get_trace(self.h)

    def info(self):
        return did_get_info(self.h)

    def phase_times(self):
        return did_get_phase_times(self.h)

    def close(self):
        if getattr(self, "h", None):
            did_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns one did_server (continuous batching of factorisation requests)."""

    def __init__(self, hbm_budget_bytes, precision=DID_FP32, max_slots=64, round_sweeps=4, stream=None):
        self.h = did_server_create(hbm_budget_bytes, precision, max_slots, round_sweeps, stream)
        self.shapes = {}
        self.inputs = {}

    def submit(self, M, N, K, seed, max_iter=300, tol=1e-4, X=None):
        t = did_server_submit(self.h, M, N, K, seed, max_iter, tol, X)
        self.shapes[t] = (M, N, K)
        if X is not None:
            self.inputs[t] = X      # read at admission: kept alive until the request finishes
        return t

    def _finished(self, ticket, res):
        if res["status"] != DID_PENDING:
            self.inputs.pop(ticket, None)
        return res

    def poll(self, ticket):
        return self._finished(ticket, did_server_poll(self.h, ticket))

    def wait(self, ticket, timeout_ms=-1):
        return self._finished(ticket, did_server_wait(self.h, ticket, timeout_ms))

    def fetch(self, ticket):
        M, N, K = self.shapes[ticket]
        Bt = np.empty((K, M), dtype=np.float32)
        C = np.empty((K, N), dtype=np.float32)
        did_server_fetch(self.h, ticket, Bt, C)
        return Bt.T, C

    def stats(self):
        return did_server_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            did_server_destroy(self.h)       # finishes every request first
            self.h = None
            self.inputs = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
