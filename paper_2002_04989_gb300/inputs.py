"""Seeded synthetic inputs for the eigenvector-eigenvalue identity path.

This module only draws random numbers and assembles symmetric matrices; it holds
none of the method's arithmetic (no eigenvalue, tridiagonalisation or identity
code).  It is the one module that both the CUDA path's callers (bench, tests) and
the oracle's callers (tests) use, so the two sides see byte-identical inputs.

Random numbers: numpy ``Generator(PCG64(seed))``; ``standard_normal`` for Gaussian
entries, ``random``/``uniform`` for uniforms.  Seeds are ``(config_id << 32) + item``
unless a workload states otherwise.  Every matrix is returned exactly symmetric
(lower triangle mirrored), float64, C-contiguous, because the library reads only
the lower triangle.

Workloads (the paper states no matrix distribution; these are the synthetic
families the build is measured on):

* ``goe(n, seed)``        A = (G + G^T)/2, G i.i.d. N(0, 1), filled row-major.
* ``wishart(n, seed)``    A = X^T X / (2n), X 2n x n i.i.d. N(0, 1).
* ``toeplitz(n, a, b)``   tridiagonal Toeplitz, diagonal a, off-diagonals b.
* ``goe_herm``, ``planted_herm``  the complex Hermitian counterparts (G = X + iY;
  Q unitary from a complex QR).
* ``planted(n, seed, lo, hi, gap)``  A = Q diag(lam) Q^T with Q the orthogonal
  factor of a Householder QR (LAPACK, via numpy) of a seeded Gaussian matrix and
  lam spread on [lo, hi] with every gap >= ``gap`` (n sorted uniforms on
  [0, hi - lo - (n-1) gap] plus k * gap: uniform over all such configurations).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Workload ids used in seeds.
CFG_GOE64 = 1
CFG_PLANTED1024 = 2
CFG_BATCH4096 = 3
CFG_PLANTED4096 = 4
CFG_SERVING = 5


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def seed_for(config_id: int, item: int) -> int:
    return (int(config_id) << 32) + int(item)


def _mirror_lower(A: np.ndarray) -> np.ndarray:
    L = np.tril(A)
    return np.ascontiguousarray(L + np.tril(L, -1).T)


def goe(n: int, seed: int, g: np.random.Generator | None = None) -> np.ndarray:
    g = g if g is not None else rng(seed)
    G = g.standard_normal((n, n))
    return np.ascontiguousarray((G + G.T) / 2)


def wishart(n: int, seed: int, g: np.random.Generator | None = None) -> np.ndarray:
    g = g if g is not None else rng(seed)
    X = g.standard_normal((2 * n, n))
    return _mirror_lower((X.T @ X) / (2 * n))


def toeplitz(n: int, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    A = np.zeros((n, n))
    idx = np.arange(n)
    A[idx, idx] = a
    A[idx[1:], idx[:-1]] = b
    A[idx[:-1], idx[1:]] = b
    return A


@dataclasses.dataclass
class Planted:
    A: np.ndarray      # n x n symmetric, float64
    lam: np.ndarray    # planted eigenvalues, ascending
    Q: np.ndarray      # Q[:, i] = unit eigenvector for lam[i] (component j = Q[j, i])


def planted_spectrum(n: int, lo: float, hi: float, gap: float, g: np.random.Generator) -> np.ndarray:
    span = (hi - lo) - (n - 1) * gap
    if span < 0:
        raise ValueError("interval too short for the requested minimum gap")
    u = np.sort(g.uniform(0.0, span, n))
    return lo + u + gap * np.arange(n)


def planted(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, gap: float = 1e-4,
            g: np.random.Generator | None = None) -> Planted:
    g = g if g is not None else rng(seed)
    G = g.standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    lam = planted_spectrum(n, lo, hi, gap, g)
    A = _mirror_lower((Q * lam) @ Q.T)
    return Planted(A=A, lam=lam, Q=np.ascontiguousarray(Q))


def _mirror_lower_herm(A: np.ndarray) -> np.ndarray:
    L = np.tril(A)
    H = L + np.tril(L, -1).conj().T
    H[np.diag_indices_from(H)] = H.diagonal().real
    return np.ascontiguousarray(H)


def goe_herm(n: int, seed: int, g: np.random.Generator | None = None) -> np.ndarray:
    """Complex Hermitian A = (G + G^H)/2 with G = X + iY, X, Y i.i.d. N(0, 1)."""
    g = g if g is not None else rng(seed)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    return _mirror_lower_herm((G + G.conj().T) / 2)


def planted_herm(n: int, seed: int, lo: float = -1.0, hi: float = 1.0, gap: float = 1e-4,
                 g: np.random.Generator | None = None) -> Planted:
    """Complex Hermitian A = Q diag(lam) Q^H, Q the unitary factor of a Householder QR
    (LAPACK, via numpy) of a seeded complex Gaussian matrix; lam as in ``planted``."""
    g = g if g is not None else rng(seed)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    lam = planted_spectrum(n, lo, hi, gap, g)
    A = _mirror_lower_herm((Q * lam) @ Q.conj().T)
    return Planted(A=A, lam=lam, Q=np.ascontiguousarray(Q))


def log_uniform_n(a: int, b: int, g: np.random.Generator) -> int:
    """n = round(a * (b/a)^u), u ~ U[0, 1), clamped to [a, b]."""
    u = g.random()
    return int(min(b, max(a, round(a * (b / a) ** u))))


# ----------------------------------------------------------------- workloads

def goe64() -> np.ndarray:
    """One GOE matrix n = 64 from seed 0; all minors and the full 64 x 64 grid."""
    return goe(64, 0)


def planted1024() -> Planted:
    """n = 1024 planted spectrum on [-1, 1], min gap 1e-4; full grid vs Q o Q."""
    return planted(1024, seed_for(CFG_PLANTED1024, 0), -1.0, 1.0, 1e-4)


def planted4096() -> tuple[Planted, np.ndarray]:
    """n = 4096 planted spectrum on [-10, 10], min gap 1e-4, and 256 distinct
    component indices j (sorted), drawn without replacement."""
    p = planted(4096, seed_for(CFG_PLANTED4096, 0), -10.0, 10.0, 1e-4)
    cols = np.sort(rng(seed_for(CFG_PLANTED4096, 1)).choice(4096, 256, replace=False))
    return p, cols.astype(np.int64)


BATCH_KINDS = ("goe", "wishart", "toeplitz")


def batch_item(m: int, nmin: int = 8, nmax: int = 256) -> tuple[str, np.ndarray]:
    """Item m of the uneven batch: n log-uniform in [nmin, nmax]; kind = m mod 3."""
    g = rng(seed_for(CFG_BATCH4096, m))
    n = log_uniform_n(nmin, nmax, g)
    kind = BATCH_KINDS[m % 3]
    if kind == "goe":
        A = goe(n, 0, g)
    elif kind == "wishart":
        A = wishart(n, 0, g)
    else:
        A = toeplitz(n, 0.0, 1.0)
    return kind, A


def batch_sizes(count: int = 4096, nmin: int = 8, nmax: int = 256) -> np.ndarray:
    """Matrix sizes of the uneven batch without building the matrices."""
    out = np.empty(count, dtype=np.int64)
    for m in range(count):
        out[m] = log_uniform_n(nmin, nmax, rng(seed_for(CFG_BATCH4096, m)))
    return out


def batch4096(count: int = 4096) -> list[np.ndarray]:
    return [batch_item(m)[1] for m in range(count)]


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float          # arrival time offset from stream start
    kind: str                 # "goe" or "planted"
    A: np.ndarray
    cols: np.ndarray | None   # None = all components
    planted: Planted | None


def serving_request(rid: int, nmin: int = 16, nmax: int = 2048) -> Request:
    """Request rid of the serving stream (arrival time filled by serving_stream)."""
    g = rng(seed_for(CFG_SERVING, rid + 1))
    n = log_uniform_n(nmin, nmax, g)
    kind = "goe" if g.random() < 0.5 else "planted"
    want_all = g.random() < 0.5
    cols = None
    if not want_all:
        k = int(g.integers(1, min(64, n) + 1))
        cols = np.sort(g.choice(n, k, replace=False)).astype(np.int64)
    if kind == "goe":
        A, pl = goe(n, 0, g), None
    else:
        pl = planted(n, 0, -1.0, 1.0, 1e-4, g)
        A = pl.A
    return Request(rid=rid, arrival_s=0.0, kind=kind, A=A, cols=cols, planted=pl)


def serving_arrivals(count: int, rate_per_s: float) -> np.ndarray:
    """Poisson arrival times (exponential gaps) at the given rate."""
    g = rng(seed_for(CFG_SERVING, 0))
    gaps = g.exponential(1.0 / rate_per_s, count)
    return np.cumsum(gaps)


def serving_sizes(count: int, nmin: int = 16, nmax: int = 2048) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    for r in range(count):
        out[r] = log_uniform_n(nmin, nmax, rng(seed_for(CFG_SERVING, r + 1)))
    return out


def min_relative_gap(lam: np.ndarray) -> float:
    """min_k (lam_{k+1} - lam_k) / max|lam| for an ascending spectrum (inf if n < 2)."""
    lam = np.asarray(lam, dtype=np.float64)
    if lam.size < 2:
        return math.inf
    scale = max(abs(lam[0]), abs(lam[-1]))
    return float(np.min(np.diff(lam)) / scale) if scale > 0 else 0.0
