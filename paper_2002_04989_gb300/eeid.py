"""Python binding of libeeid (ctypes): argument marshalling only.

Every function here forwards to the C entry point of the same name declared in
``include/eeid.h``; the arithmetic runs in the CUDA kernels of libeeid.so.  Device
arrays are ``torch`` float64 CUDA tensors (PyTorch supplies device memory and the
current stream); index lists are host integer sequences.  There is no CPU path:
if the library cannot be loaded, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

EEID_OK = 0
EEID_WARN_DEGENERATE = 1
EEID_WARN_SMALL_GAP = 2
EEID_ERR_INVALID = -1
EEID_ERR_NOMEM = -2
EEID_ERR_CUDA = -3
EEID_ERR_TIMEOUT = -4
EEID_ERR_BUSY = -5
EEID_ERR_NOT_FOUND = -6
EEID_ERR_CANCELLED = -7
# device-side status bits (EEID_DEV_* in include/eeid.h)
EEID_DEV_DEGENERATE = 1
EEID_DEV_SMALL_GAP = 2
EEID_DEV_BRACKET_FALLBACK = 4
EEID_DEV_BAD_TASK = 8
EEID_DEV_TIMEOUT = 16

_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i64p = ctypes.POINTER(ctypes.c_int64)


class EeidError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"eeid status {status}: {msg}")
        self.status = status


class EeidServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int),
                ("max_inflight", ctypes.c_int), ("max_pending", ctypes.c_int)]


class EeidReqStats(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("batch_id", ctypes.c_int64), ("batch_requests", ctypes.c_int64)]


class EeidServerInfo(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("inflight_batches", ctypes.c_int64),
                ("batches_launched", ctypes.c_int64), ("max_overlapping_batches", ctypes.c_int64),
                ("device_bytes_in_use", ctypes.c_int64), ("device_budget_bytes", ctypes.c_int64)]


class EeidProblem(ctypes.Structure):
    _fields_ = [("dA", _vp), ("lda", _i64), ("n", _i64), ("h_rows", _i64p), ("nrows", _i64),
                ("h_cols", _i64p), ("ncols", _i64), ("d_out", _vp), ("d_lambda", _vp)]


SIGNATURES = {
    "eeid_ctx_create": ([ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(_vp)], ctypes.c_int),
    "eeid_ctx_destroy": ([_vp], None),
    "eeid_last_error": ([], ctypes.c_char_p),
    "eeid_sync": ([_vp, _vp], ctypes.c_int),
    "eeid_eigvals": ([_vp, _vp, _i64, _i64, _vp, _vp], ctypes.c_int),
    "eeid_minor_eigvals": ([_vp, _vp, _i64, _i64, _i64p, _i64, _vp, _vp], ctypes.c_int),
    "eeid_components": ([_vp, _vp, _i64, _i64, _i64p, _i64, _i64p, _i64, _vp, _vp, _vp],
                        ctypes.c_int),
    "eeid_components_host": ([_vp, _vp, _i64, _i64, _i64p, _i64, _i64p, _i64, _vp, _vp, _vp],
                             ctypes.c_int),
    "eeid_components_herm": ([_vp, _vp, _i64, _i64, _i64p, _i64, _i64p, _i64, _vp, _vp, _vp],
                             ctypes.c_int),
    "eeid_eigenvectors": ([_vp, _vp, _i64, _i64, _i64p, _i64, _vp, _vp, _vp], ctypes.c_int),
    "eeid_components_batched": ([_vp, ctypes.POINTER(EeidProblem), _i64, _vp], ctypes.c_int),
    "eeid_launch_count": ([_vp], ctypes.c_int64),
    "eeid_vector_refs": ([_vp], ctypes.c_int64),
    "eeid_set_timing": ([_vp, ctypes.c_int], ctypes.c_int),
    "eeid_tune_tridiag": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "eeid_tune_reset": ([_vp], ctypes.c_int),
    "eeid_autotune": ([_vp, ctypes.c_int, ctypes.c_char_p], ctypes.c_int),
    "eeid_phase_times": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int], ctypes.c_int),
    "eeid_eigvals_noalloc": ([_vp, _i64, _i64, _vp, _vp, _vp], ctypes.c_int),
    "eeid_set_graphs": ([_vp, ctypes.c_int], ctypes.c_int),
    "eeid_set_overlap": ([_vp, ctypes.c_int], ctypes.c_int),
    "eeid_set_clusters": ([_vp, ctypes.c_int], ctypes.c_int),
    "eeid_check_barrier_timeout": ([_vp, _vp], ctypes.c_int),
    "eeid_server_create": ([ctypes.c_int, ctypes.POINTER(EeidServerOpts), ctypes.POINTER(_vp)],
                           ctypes.c_int),
    "eeid_server_destroy": ([_vp], None),
    "eeid_server_submit": ([_vp, _vp, _i64, _i64, _i64p, _i64, _vp, _vp, ctypes.c_int,
                            ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "eeid_server_wait": ([_vp, ctypes.c_uint64, _i64, ctypes.POINTER(EeidReqStats)], ctypes.c_int),
    "eeid_server_cancel": ([_vp, ctypes.c_uint64], ctypes.c_int),
    "eeid_server_info": ([_vp, ctypes.POINTER(EeidServerInfo)], ctypes.c_int),
}

PHASES = ("tridiag", "bisect_A", "denominators", "bisect_minors", "identity")


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libeeid.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libeeid.so not found at {path}: build the CUDA path first")
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def last_error() -> str:
    m = load().eeid_last_error()
    return m.decode() if m else ""


def _check(status: int, allow_warn: bool = True) -> int:
    if status < 0 or (status > 0 and not allow_warn):
        raise EeidError(status, last_error())
    return status


def _idx(ix):
    """(pointer, count, keepalive) for an optional host index list."""
    if ix is None:
        return None, None, None
    a = np.ascontiguousarray(np.asarray(ix, dtype=np.int64).reshape(-1))
    return a.ctypes.data_as(_i64p), a.size, a


def _stream(stream):
    import torch
    if stream is None:
        return _vp(torch.cuda.current_stream().cuda_stream)
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev(t, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    return t


def _mat(A):
    _dev(A, "A")
    if A.dim() != 2 or A.shape[0] != A.shape[1] or A.stride(1) != 1:
        raise ValueError("A must be a square matrix with unit column stride (row-major)")
    return A, int(A.stride(0)) if A.shape[0] > 0 else max(1, A.shape[0])


def _cmat(A):
    """A complex128 CUDA matrix with unit column stride: (A, lda in complex elements)."""
    import torch
    if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype == torch.complex128):
        raise TypeError("A must be a complex128 CUDA tensor")
    if A.dim() != 2 or A.shape[0] != A.shape[1] or A.stride(1) != 1:
        raise ValueError("A must be a square matrix with unit column stride (row-major)")
    return A, int(A.stride(0)) if A.shape[0] > 0 else 1


def _out(t, numel, like, name, dtype=None):
    """A caller-supplied output the kernels write `numel` elements into: it must be a
    contiguous CUDA tensor of the right dtype, on the device of `like`, with room for
    all of them (the library writes through the raw pointer)."""
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype):
        raise TypeError(f"{name} must be a {dtype} CUDA tensor")
    if t.device != like.device:
        raise ValueError(f"{name} is on {t.device}, the matrix on {like.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the call writes {numel}")
    return t


def _hout(a, numel, name):
    """A caller-supplied host output: a C-contiguous float64 numpy array with room for
    `numel` elements (the library writes through the raw pointer)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError(f"{name} must be a C-contiguous float64 numpy array")
    if a.size < numel:
        raise ValueError(f"{name} holds {a.size} elements, the call writes {numel}")
    return a


def eeid_eigvals_noalloc(A, out=None, status=None, stream=None):
    """Eigenvalues of A without any device allocation by the library (n <= 512);
    see eeid_eigvals_noalloc in include/eeid.h.  `out` may be a preallocated
    float64 CUDA tensor of n elements; `status`, an int32 CUDA tensor of one
    element, receives the call's EEID_DEV_* bits once the stream reaches the end
    of the call."""
    import torch
    A, lda = _mat(A)
    n = A.shape[0]
    lam = (_out(out, n, A, "out") if out is not None
           else torch.empty(n, dtype=torch.float64, device=A.device))
    sp = _vp(_out(status, 1, A, "status", torch.int32).data_ptr()) if status is not None else None
    with torch.cuda.device(A.device):
        _check(load().eeid_eigvals_noalloc(_vp(A.data_ptr()), lda, n, _vp(lam.data_ptr()), sp,
                                           _stream(stream)), False)
    return lam


class Context:
    """Owns an eeid_ctx (device workspace within an HBM budget)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        h = _vp()
        _check(self.lib.eeid_ctx_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)), False)
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eeid_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- entry points (same names as the C ABI, without the prefix)
    def eeid_sync(self, stream=None) -> int:
        return _check(self.lib.eeid_sync(self.handle, _stream(stream)))

    def eeid_eigvals(self, A, out=None, stream=None):
        import torch
        A, lda = _mat(A)
        n = A.shape[0]
        lam = (_out(out, n, A, "out") if out is not None
               else torch.empty(n, dtype=torch.float64, device=A.device))
        _check(self.lib.eeid_eigvals(self.handle, _vp(A.data_ptr()), lda, n, _vp(lam.data_ptr()),
                                     _stream(stream)))
        return lam

    def eeid_minor_eigvals(self, A, cols=None, out=None, stream=None):
        import torch
        A, lda = _mat(A)
        n = A.shape[0]
        cp, nc, keep = _idx(cols)
        nc = n if cp is None else nc
        mu = (_out(out, nc * max(n - 1, 0), A, "out") if out is not None
              else torch.empty((nc, max(n - 1, 0)), dtype=torch.float64, device=A.device))
        _check(self.lib.eeid_minor_eigvals(self.handle, _vp(A.data_ptr()), lda, n, cp, nc,
                                           _vp(mu.data_ptr()), _stream(stream)))
        return mu

    def eeid_components(self, A, rows=None, cols=None, out=None, lam=None, stream=None):
        import torch
        A, lda = _mat(A)
        n = A.shape[0]
        rp, nr, k1 = _idx(rows)
        cp, nc, k2 = _idx(cols)
        nr = n if rp is None else nr
        nc = n if cp is None else nc
        o = (_out(out, nr * nc, A, "out") if out is not None
             else torch.empty((nr, nc), dtype=torch.float64, device=A.device))
        if lam is not None:
            _out(lam, n, A, "lam")
        _check(self.lib.eeid_components(self.handle, _vp(A.data_ptr()), lda, n, rp, nr, cp, nc,
                                        _vp(o.data_ptr()),
                                        _vp(lam.data_ptr()) if lam is not None else None,
                                        _stream(stream)))
        return o

    def eeid_components_herm(self, A, rows=None, cols=None, out=None, lam=None, stream=None):
        """|v_ij|^2 of a complex Hermitian A (complex128 CUDA tensor, lower triangle read)."""
        import torch
        A, lda = _cmat(A)
        n = A.shape[0]
        rp, nr, k1 = _idx(rows)
        cp, nc, k2 = _idx(cols)
        nr = n if rp is None else nr
        nc = n if cp is None else nc
        o = (_out(out, nr * nc, A, "out") if out is not None
             else torch.empty((nr, nc), dtype=torch.float64, device=A.device))
        if lam is not None:
            _out(lam, n, A, "lam")
        _check(self.lib.eeid_components_herm(self.handle, _vp(A.data_ptr()), lda, n, rp, nr, cp,
                                             nc, _vp(o.data_ptr()),
                                             _vp(lam.data_ptr()) if lam is not None else None,
                                             _stream(stream)))
        return o

    def eeid_eigenvectors(self, A, rows=None, out=None, lam=None, stream=None):
        """Signed unit eigenvectors: out[r, j] = v_ij for i = rows[r] (all if None)."""
        import torch
        A, lda = _mat(A)
        n = A.shape[0]
        rp, nr, k1 = _idx(rows)
        nr = n if rp is None else nr
        o = (_out(out, nr * n, A, "out") if out is not None
             else torch.empty((nr, n), dtype=torch.float64, device=A.device))
        if lam is not None:
            _out(lam, n, A, "lam")
        _check(self.lib.eeid_eigenvectors(self.handle, _vp(A.data_ptr()), lda, n, rp, nr,
                                          _vp(o.data_ptr()),
                                          _vp(lam.data_ptr()) if lam is not None else None,
                                          _stream(stream)))
        return o

    def eeid_components_host(self, A: np.ndarray, rows=None, cols=None, out=None, lam=None,
                             stream=None):
        A = np.ascontiguousarray(A, dtype=np.float64)
        n = A.shape[0]
        rp, nr, k1 = _idx(rows)
        cp, nc, k2 = _idx(cols)
        nr = n if rp is None else nr
        nc = n if cp is None else nc
        o = _hout(out, nr * nc, "out") if out is not None else np.empty((nr, nc))
        if lam is not None:
            _hout(lam, n, "lam")
        st = self.lib.eeid_components_host(
            self.handle, A.ctypes.data_as(_vp), n, n, rp, nr, cp, nc, o.ctypes.data_as(_vp),
            lam.ctypes.data_as(_vp) if lam is not None else None, _stream(stream))
        _check(st)
        return o

    def eeid_components_batched(self, problems, stream=None):
        """problems: list of dicts {A, rows?, cols?, out, lam?} (torch CUDA tensors)."""
        arr = (EeidProblem * len(problems))()
        keep = []
        for p, d in enumerate(problems):
            A, lda = _mat(d["A"])
            n = A.shape[0]
            rp, nr, k1 = _idx(d.get("rows"))
            cp, nc, k2 = _idx(d.get("cols"))
            keep += [k1, k2]
            arr[p].dA = A.data_ptr()
            arr[p].lda = lda
            arr[p].n = n
            arr[p].h_rows = rp
            arr[p].nrows = n if rp is None else nr
            arr[p].h_cols = cp
            arr[p].ncols = n if cp is None else nc
            arr[p].d_out = _out(d["out"], arr[p].nrows * arr[p].ncols, A, "out").data_ptr()
            lam = d.get("lam")
            arr[p].d_lambda = _out(lam, n, A, "lam").data_ptr() if lam is not None else None
        return _check(self.lib.eeid_components_batched(self.handle, arr, len(problems),
                                                       _stream(stream)))

    def eeid_set_graphs(self, enable: bool = True) -> int:
        return _check(self.lib.eeid_set_graphs(self.handle, 1 if enable else 0), False)

    def eeid_set_overlap(self, enable: bool = True) -> int:
        return _check(self.lib.eeid_set_overlap(self.handle, 1 if enable else 0), False)

    def eeid_set_clusters(self, mode=2) -> int:
        """False/0: off; True/1: the cluster plan only; 2 (default): clusters plus the group
        plan."""
        mode = int(mode)
        if mode not in (0, 1, 2):
            raise ValueError(f"cluster mode {mode} (0, 1 or 2)")
        return _check(self.lib.eeid_set_clusters(self.handle, mode), False)

    def eeid_check_barrier_timeout(self, stream=None) -> int:
        return _check(self.lib.eeid_check_barrier_timeout(self.handle, _stream(stream)), False)

    def launch_count(self) -> int:
        return int(self.lib.eeid_launch_count(self.handle))

    def eeid_launch_count(self) -> int:
        return self.launch_count()

    def eeid_vector_refs(self) -> int:
        return int(self.lib.eeid_vector_refs(self.handle))

    def eeid_tune_tridiag(self, m_lo: int, m_hi: int, path: int, warps: int) -> int:
        return _check(self.lib.eeid_tune_tridiag(self.handle, m_lo, m_hi, path, warps), False)

    def eeid_autotune(self, max_m: int = 1024, cache_path: str | None = None) -> int:
        path = cache_path.encode() if cache_path else None
        return _check(self.lib.eeid_autotune(self.handle, int(max_m), path), False)

    def eeid_tune_reset(self) -> int:
        return _check(self.lib.eeid_tune_reset(self.handle), False)

    def eeid_set_timing(self, enable: bool = True) -> int:
        return _check(self.lib.eeid_set_timing(self.handle, 1 if enable else 0), False)

    def eeid_phase_times(self) -> dict:
        buf = (ctypes.c_double * len(PHASES))()
        k = self.lib.eeid_phase_times(self.handle, buf, len(PHASES))
        if k < 0:
            _check(k, False)
        return {PHASES[i]: float(buf[i]) for i in range(k)}


class Server:
    """The serving loop (eeid_server_*): continuous batching of requests on one GPU.
    submit() copies the host matrix and returns a ticket; wait() blocks for that
    request and returns (out, lam, stats)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_batch: int = 0,
                 max_inflight: int = 0, max_pending: int = 0):
        self.lib = load()
        opts = EeidServerOpts(hbm_budget_bytes, max_batch, max_inflight, max_pending)
        h = _vp()
        _check(self.lib.eeid_server_create(int(device), ctypes.byref(opts), ctypes.byref(h)), False)
        self.handle = h
        self._bufs = {}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.eeid_server_destroy(self.handle)
            self.handle = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def eeid_server_submit(self, A: np.ndarray, cols=None, nonblocking: bool = False) -> int:
        A = np.ascontiguousarray(A, dtype=np.float64)
        n = A.shape[0]
        cp, nc, keep = _idx(cols)
        nc = n if cp is None else nc
        out = np.empty((n, nc))
        lam = np.empty(n)
        t = ctypes.c_uint64()
        _check(self.lib.eeid_server_submit(self.handle, A.ctypes.data_as(_vp), n, n, cp, nc,
                                           out.ctypes.data_as(_vp), lam.ctypes.data_as(_vp),
                                           1 if nonblocking else 0, ctypes.byref(t)), False)
        self._bufs[t.value] = (out, lam)
        return t.value

    def eeid_server_wait(self, ticket: int, timeout_ms: int = -1):
        st = EeidReqStats()
        status = self.lib.eeid_server_wait(self.handle, ctypes.c_uint64(ticket), int(timeout_ms),
                                           ctypes.byref(st))
        if status == EEID_ERR_TIMEOUT:
            raise EeidError(status, last_error())
        out, lam = self._bufs.pop(ticket, (None, None))
        _check(status)
        return out, lam, {"queue_ms": st.queue_ms, "total_ms": st.total_ms,
                          "batch_id": st.batch_id, "batch_requests": st.batch_requests,
                          "status": status}

    def eeid_server_cancel(self, ticket: int) -> int:
        return _check(self.lib.eeid_server_cancel(self.handle, ctypes.c_uint64(ticket)), False)

    def eeid_server_info(self) -> dict:
        info = EeidServerInfo()
        _check(self.lib.eeid_server_info(self.handle, ctypes.byref(info)), False)
        return {f: getattr(info, f) for f, _ in EeidServerInfo._fields_}
