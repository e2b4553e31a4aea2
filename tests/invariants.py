"""Checks that hold for any correct |v_ij|^2 grid, whatever computed it.

They follow from the definitions around Eq. 1 (Sec. 2): the eigenvectors v_i of a
real symmetric A are orthonormal, so the squared components form a doubly
stochastic matrix; A = sum_i lam_i v_i v_i^T gives sum_i lam_i |v_ij|^2 = a_jj; the
trace and Frobenius norm are spectral sums; and the minor's eigenvalues interlace
A's (Cauchy).  Used on the oracle (pins) and on the CUDA path's outputs.
"""
from __future__ import annotations

import numpy as np


def grid_errors(A, lam, vsq, cols=None):
    """Max abs deviations of the grid invariants.

    vsq[i, c] = |v_{i, cols[c]}|^2 for ALL eigen-indices i (rows = all)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    cols = np.arange(n) if cols is None else np.asarray(cols)
    out = {}
    out["col_sum"] = float(np.max(np.abs(vsq.sum(axis=0) - 1.0))) if vsq.size else 0.0
    if cols.size == n and np.all(cols == np.arange(n)):
        out["row_sum"] = float(np.max(np.abs(vsq.sum(axis=1) - 1.0)))
    diag = np.diag(A)[cols]
    out["diag"] = float(np.max(np.abs(lam @ vsq - diag))) if vsq.size else 0.0
    out["min"] = float(vsq.min()) if vsq.size else 0.0
    return out


def spectrum_errors(A, lam, mu=None, cols=None):
    """Trace / Frobenius / interlacing checks for lam (A) and mu (minors)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    out = {
        "trace": float(abs(lam.sum() - np.trace(A))),
        "frob": float(abs((lam ** 2).sum() - (A ** 2).sum())),
        "sorted": float(max(0.0, -np.min(np.diff(lam)))) if n > 1 else 0.0,
    }
    if mu is not None and n > 1:
        cols = np.arange(n) if cols is None else np.asarray(cols)
        tr = np.trace(A)
        out["minor_trace"] = float(np.max(np.abs(mu.sum(axis=1) - (tr - np.diag(A)[cols]))))
        lo = lam[:-1][None, :] - mu
        hi = mu - lam[1:][None, :]
        out["interlace"] = float(max(0.0, lo.max(), hi.max()))
    return out
