"""CPU oracle for the eigenvector-eigenvalue identity path -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` /
``--impl reference`` legs may import this package.  The product path (the CUDA
library ``libeeid.so`` and its binding in ``paper_2002_04989_gb300``) never imports,
links or runs it, and it shares no code with that path.

The arithmetic lives in ``oracle.c`` (plain C, ``long double``); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Each wrapper names
the definition it follows; see the C file's header for the methods.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP, IEEE semantics)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-std=c11", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_eigvals": [_i64, _dp, _i64, _dp],
                "oracle_eig": [_i64, _dp, _i64, _dp, _dp],
                "oracle_eigvecs": [_i64, _dp, _i64, _dp, _dp],
                "oracle_minor_eigvals": [_i64, _dp, _i64, _ip, _i64, _dp],
                "oracle_identity": [_i64, _dp, _dp, _ip, _i64, _i64, ctypes.c_int, _dp],
                "oracle_components": [_i64, _dp, _i64, _ip, _i64, _ip, _i64, ctypes.c_int,
                                      _dp, _dp, _dp],
                "oracle_secular_minor_eigvals": [_i64, _dp, _dp, _ip, _i64, _dp],
                "oracle_inverse_iteration": [_i64, _dp, _i64, ctypes.c_double, ctypes.c_int, _dp],
                "oracle_real_mant_dig": [],
                "oracle_components_herm": [_i64, _dp, _i64, _ip, _i64, _ip, _i64, ctypes.c_int,
                                           _dp, _dp],
                "oracle_minor_eigvals_herm": [_i64, _dp, _i64, _ip, _i64, _dp],
            }
            for name, args in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


def _mat(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    assert A.ndim == 2 and A.shape[0] == A.shape[1]
    return A


def _idx(ix, n):
    if ix is None:
        return None, n
    a = np.ascontiguousarray(np.asarray(ix, dtype=np.int64).reshape(-1))
    return a, a.size


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with code {rc}")


def real_mant_dig() -> int:
    """Mantissa bits of the oracle's long double on this host (64 x87, 113 quad)."""
    return _load().oracle_real_mant_dig()


def eigvals(A):
    """Ascending eigenvalues of symmetric A by cyclic Jacobi (lower triangle read)."""
    A = _mat(A)
    n = A.shape[0]
    lam = np.empty(n)
    _check(_load().oracle_eigvals(n, _d(A), n, _d(lam)), "oracle_eigvals")
    return lam


def eig_vsq(A):
    """(lam, vsq) with vsq[i, j] = |v_ij|^2 from the Jacobi eigenvectors (V o V)."""
    A = _mat(A)
    n = A.shape[0]
    lam = np.empty(n)
    vsq = np.empty((n, n))
    _check(_load().oracle_eig(n, _d(A), n, _d(lam), _d(vsq)), "oracle_eig")
    return lam, vsq


def eigvecs(A, convention=False):
    """(lam, vec) with vec[i, j] = component j of the unit eigenvector i (signed),
    from cyclic Jacobi with the rotations accumulated.  Each eigenvector is defined
    up to its sign; with ``convention`` the sign is fixed by ``sign_convention``."""
    A = _mat(A)
    n = A.shape[0]
    lam = np.empty(n)
    vec = np.empty((n, n))
    _check(_load().oracle_eigvecs(n, _d(A), n, _d(lam), _d(vec)), "oracle_eigvecs")
    return lam, (sign_convention(vec) if convention else vec)


def sign_convention(vec):
    """The sign convention for signed eigenvectors (rows of ``vec``): the component of
    largest magnitude is made positive (the first such component on exact ties).
    Eq. 1 (Sec. 2) fixes only |v_ij|, so any signed result is compared in this form."""
    vec = np.array(vec, dtype=np.float64, copy=True)
    if vec.size == 0:
        return vec
    jstar = np.argmax(np.abs(vec), axis=1)
    flip = vec[np.arange(vec.shape[0]), jstar] < 0
    vec[flip] *= -1.0
    return vec


def minor_eigvals(A, cols=None):
    """mu[c, k]: ascending eigenvalues of M_j (A without row/column j), j = cols[c]."""
    A = _mat(A)
    n = A.shape[0]
    c, nc = _idx(cols if cols is not None else np.arange(n), n)
    mu = np.empty((nc, max(n - 1, 0)))
    _check(_load().oracle_minor_eigvals(n, _d(A), n, _i(c), nc, _d(mu)), "oracle_minor_eigvals")
    return mu


def identity(lam, mu, rows=None, mode=0):
    """Eq. 1 from given eigenvalues: out[r, c] for eigen-index rows[r] and the minor
    eigenvalues mu[c, :] (mode 0 literal products, mode 1 paired ratios)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = lam.size
    mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(-1, max(n - 1, 0)))
    nc = mu.shape[0]
    r, nr = _idx(rows if rows is not None else np.arange(n), n)
    out = np.empty((nr, nc))
    _check(_load().oracle_identity(n, _d(lam), _d(mu) if n > 1 else None, _i(r), nr, nc, mode,
                                   _d(out)), "oracle_identity")
    return out


def components(A, rows=None, cols=None, method=0, want_eigs=False):
    """|v_ij|^2 for i in rows, j in cols, end to end in long double.

    method 0: Jacobi eigenvalues of A and every M_j, then Eq. 1 literally;
    method 1: same, Eq. 1 as paired ratios; method 2: V o V (plain definition).
    With want_eigs, also returns (lam, mu) (mu is None for method 2)."""
    A = _mat(A)
    n = A.shape[0]
    r, nr = _idx(rows, n)
    c, nc = _idx(cols, n)
    out = np.empty((nr, nc))
    lam = np.empty(n)
    mu = np.empty((nc, max(n - 1, 0))) if method != 2 else None
    _check(_load().oracle_components(n, _d(A), n, _i(r), nr, _i(c), nc, method, _d(out),
                                     _d(lam), _d(mu) if (mu is not None and n > 1) else None),
           "oracle_components")
    return (out, lam, mu) if want_eigs else out


def secular_minor_eigvals(lam, Q, cols):
    """Eigenvalues of the minors of Q diag(lam) Q^T from (lam, Q): the roots of
    sum_i Q_ji^2 / (mu - lam_i) = 0 (Cramer's rule), by bisection per pole gap."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = lam.size
    c, nc = _idx(cols, n)
    mu = np.empty((nc, max(n - 1, 0)))
    _check(_load().oracle_secular_minor_eigvals(n, _d(lam), _d(Q), _i(c), nc, _d(mu)),
           "oracle_secular_minor_eigvals")
    return mu


def inverse_iteration(A, shift, iters=3):
    """Unit eigenvector nearest `shift` by shifted inverse iteration (tiny n)."""
    A = _mat(A)
    n = A.shape[0]
    x = np.empty(n)
    _check(_load().oracle_inverse_iteration(n, _d(A), n, float(shift), int(iters), _d(x)),
           "oracle_inverse_iteration")
    return x


def _herm(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    assert A.ndim == 2 and A.shape[0] == A.shape[1]
    return A, A.view(np.float64)


def components_herm(A, rows=None, cols=None, method=0, want_eigs=False):
    """|v_ij|^2 of a complex Hermitian A (lower triangle read) in long double, through
    the real symmetric embedding [[Re, -Im], [Im, Re]]: method 0 = Jacobi eigenvalues
    of A and every M_j, then Eq. 1; method 2 = the embedding's eigenvectors."""
    A, Af = _herm(A)
    n = A.shape[0]
    r, nr = _idx(rows, n)
    c, nc = _idx(cols, n)
    out = np.empty((nr, nc))
    lam = np.empty(n)
    _check(_load().oracle_components_herm(n, _d(Af), n, _i(r), nr, _i(c), nc, method, _d(out),
                                          _d(lam)), "oracle_components_herm")
    return (out, lam) if want_eigs else out


def minor_eigvals_herm(A, cols=None):
    """mu[c, k]: ascending eigenvalues of the minors M_j of Hermitian A, j = cols[c]."""
    A, Af = _herm(A)
    n = A.shape[0]
    c, nc = _idx(cols if cols is not None else np.arange(n), n)
    mu = np.empty((nc, max(n - 1, 0)))
    _check(_load().oracle_minor_eigvals_herm(n, _d(Af), n, _i(c), nc, _d(mu)),
           "oracle_minor_eigvals_herm")
    return mu
