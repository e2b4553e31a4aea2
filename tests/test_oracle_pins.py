"""Pins for the CPU oracle: checks against facts the paper and the mathematics fix,
not against the oracle itself.  CPU only.

* hand-derived examples (tests/golden/hand_examples.txt, each with its derivation);
* closed forms: 2x2 matrices, diagonal matrices, tridiagonal Toeplitz matrices
  (eigenvalues a + 2b cos(k pi/(n+1)), sine eigenvectors, minors that split into two
  smaller Toeplitz blocks);
* invariants of any orthonormal eigenbasis and Cauchy interlacing;
* brute force: eigenvectors by shifted inverse iteration for n <= 8;
* a library routine: LAPACK's symmetric eigensolver through numpy;
* a planted spectrum with known eigenvectors Q;
* the signed eigenvectors (oracle.eigvecs): the 2x2 eigenvector (b, lam - a), the
  Toeplitz sine vectors, the residual A v = lam v with V^T V = I, inverse iteration,
  planted Q, and the sign convention (largest-magnitude component positive).
A last group plants plausible mistakes (dropped factor, swapped numerator and
denominator, i and j exchanged, wrong minor) into the oracle's inputs and shows
that the pins reject each of them.
"""
import math

import numpy as np
import pytest

from golden_io import hand_examples
from invariants import grid_errors, spectrum_errors
from paper_2002_04989_gb300 import inputs


# ------------------------------------------------------------------ golden

@pytest.mark.parametrize("ex", hand_examples(), ids=lambda e: e["name"])
def test_hand_examples(oracle_mod, ex):
    A, n = ex["A"], ex["n"]
    lam = oracle_mod.eigvals(A)
    assert np.max(np.abs(lam - ex["lam"])) < 1e-15
    for method in (0, 1, 2):
        out = oracle_mod.components(A, method=method)
        assert np.max(np.abs(out - ex["vsq"])) < 2e-16 * 8, (method, out, ex["vsq"])


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("seed", range(6))
def test_2x2_closed_form(oracle_mod, seed):
    g = np.random.default_rng(seed)
    a, b, c = g.standard_normal(3)
    A = np.array([[a, b], [b, c]])
    h = math.sqrt(((a - c) / 2) ** 2 + b * b)
    lp, lm = (a + c) / 2 + h, (a + c) / 2 - h
    # eigenvector of lam_+ is (b, lam_+ - a): an independent route to |v|^2
    p0 = b * b / (b * b + (lp - a) ** 2)
    expect = np.array([[1 - p0, p0], [p0, 1 - p0]])  # rows: lam_-, lam_+
    lam = oracle_mod.eigvals(A)
    assert np.allclose(lam, [lm, lp], rtol=0, atol=4e-16 * (abs(lp) + abs(lm) + 1))
    mu = oracle_mod.minor_eigvals(A)
    assert mu[0, 0] == c and mu[1, 0] == a
    for method in (0, 1, 2):
        out = oracle_mod.components(A, method=method)
        assert np.max(np.abs(out - expect)) < 1e-14, method
    # Eq. 1 read directly for the 2x2 case: |v_{+,0}|^2 = (lam_+ - c)/(lam_+ - lam_-)
    assert abs(oracle_mod.identity([lm, lp], [[c]], rows=[1])[0, 0] - (lp - c) / (lp - lm)) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 5, 17])
def test_diagonal_exact(oracle_mod, n):
    g = np.random.default_rng(100 + n)
    d = g.permutation(np.linspace(-3, 4, n)) if n > 1 else np.array([0.7])
    A = np.diag(d)
    order = np.argsort(d)
    expect = np.zeros((n, n))
    expect[np.arange(n), order] = 1.0   # i-th smallest sits at position order[i]
    for method in (0, 1, 2):
        out = oracle_mod.components(A, method=method)
        assert np.array_equal(out, expect), method   # exact zeros and ones
    mu = oracle_mod.minor_eigvals(A)
    for j in range(n):
        assert np.array_equal(mu[j], np.sort(np.delete(d, j)))


def toeplitz_closed(n, a, b):
    k = np.arange(1, n + 1)
    lam = np.sort(a + 2 * b * np.cos(k * np.pi / (n + 1)))
    i = np.arange(1, n + 1)[:, None]
    j = np.arange(1, n + 1)[None, :]
    vsq = 2.0 / (n + 1) * np.sin(i * j * np.pi / (n + 1)) ** 2
    return lam, vsq


def toeplitz_minor_closed(n, a, b, j):
    parts = []
    for m in (j, n - 1 - j):  # M_j = T_j (+) T_{n-1-j}
        if m > 0:
            parts.append(a + 2 * b * np.cos(np.arange(1, m + 1) * np.pi / (m + 1)))
    return np.sort(np.concatenate(parts)) if parts else np.zeros(0)


@pytest.mark.parametrize("n,a,b", [(1, 0.0, 1.0), (2, 0.0, 1.0), (3, 0.25, -0.5), (8, 0.0, 1.0),
                                   (17, -1.0, 0.75), (32, 0.0, 1.0)])
def test_toeplitz_closed_form(oracle_mod, n, a, b):
    A = inputs.toeplitz(n, a, b)
    lam_c, vsq_c = toeplitz_closed(n, a, b)
    lam = oracle_mod.eigvals(A)
    assert np.max(np.abs(lam - lam_c)) < 1e-14
    mu = oracle_mod.minor_eigvals(A)
    for j in range(n):
        assert np.max(np.abs(mu[j] - toeplitz_minor_closed(n, a, b, j)), initial=0) < 1e-14
    for method in (0, 1, 2):
        out = oracle_mod.components(A, method=method)
        assert np.max(np.abs(out - vsq_c)) < 1e-13, method


def test_toeplitz_odd_middle_minor_zeros(oracle_mod):
    # n odd, j = (n+1)/2 (1-based): both halves are T_{(n-1)/2}, every minor eigenvalue
    # is doubled, and |v_ij|^2 = 0 exactly for every even 1-based i.
    n = 9
    A = inputs.toeplitz(n, 0.0, 1.0)
    j = (n - 1) // 2
    out = oracle_mod.components(A, cols=[j], method=0)[:, 0]
    _, vsq_c = toeplitz_closed(n, 0.0, 1.0)
    assert np.max(np.abs(out - vsq_c[:, j])) < 1e-14
    assert np.all(np.abs(out[1::2]) < 1e-15)


# ------------------------------------------------------------------ invariants

@pytest.mark.parametrize("kind,n", [("goe", 12), ("goe", 40), ("wishart", 24), ("planted", 30)])
def test_invariants(oracle_mod, kind, n):
    if kind == "goe":
        A = inputs.goe(n, 7)
    elif kind == "wishart":
        A = inputs.wishart(n, 8)
    else:
        A = inputs.planted(n, 9, gap=1e-2).A
    out, lam, mu = oracle_mod.components(A, method=0, want_eigs=True)
    g = grid_errors(A, lam, out)
    assert g["col_sum"] < 1e-13 and g["row_sum"] < 1e-13 and g["diag"] < 1e-13
    assert g["min"] >= 0
    s = spectrum_errors(A, lam, mu)
    assert s["trace"] < 1e-12 and s["frob"] < 1e-11 and s["sorted"] == 0
    assert s["minor_trace"] < 1e-12 and s["interlace"] == 0


def test_n1(oracle_mod):
    A = np.array([[3.25]])
    assert oracle_mod.components(A, method=0)[0, 0] == 1.0
    assert oracle_mod.components(A, method=2)[0, 0] == 1.0
    assert oracle_mod.eigvals(A)[0] == 3.25


# ------------------------------------------------------------------ brute force

@pytest.mark.parametrize("n", [3, 5, 8])
def test_inverse_iteration_brute_force(oracle_mod, n):
    A = inputs.goe(n, 40 + n)
    lam = oracle_mod.eigvals(A)
    gaps = np.diff(lam)
    assert gaps.min() > 1e-3  # seeds chosen with separated spectra
    brute = np.empty((n, n))
    for i in range(n):
        x = oracle_mod.inverse_iteration(A, lam[i] + 1e-9 * (1 + abs(lam[i])), iters=4)
        assert abs(x @ A @ x - lam[i]) < 1e-14   # Rayleigh quotient
        brute[i] = x * x
    for method in (0, 1, 2):
        out = oracle_mod.components(A, method=method)
        assert np.max(np.abs(out - brute)) < 1e-15, method


# ------------------------------------------------------------------ library + planted

@pytest.mark.parametrize("seed", [1, 2])
def test_against_lapack(oracle_mod, seed):
    A = inputs.goe(60, seed)
    lam = oracle_mod.eigvals(A)
    w, V = np.linalg.eigh(A)
    assert np.max(np.abs(lam - w)) < 1e-13
    gapmin = np.min(np.diff(w))
    out = oracle_mod.components(A, method=0)
    # LAPACK's vectors carry O(eps ||A|| / gap) error; the bound below is that order.
    assert np.max(np.abs(out - (V * V).T)) < 1e-14 / gapmin


def test_planted_closed_form_and_secular(oracle_mod):
    p = inputs.planted(48, 11, -1.0, 1.0, 1e-2)
    out, lam, mu = oracle_mod.components(p.A, method=0, want_eigs=True)
    assert np.max(np.abs(lam - p.lam)) < 1e-14
    assert np.max(np.abs(out - (p.Q * p.Q).T)) < 1e-12
    cols = np.arange(48)
    mu_sec = oracle_mod.secular_minor_eigvals(p.lam, p.Q, cols)
    assert np.max(np.abs(mu_sec - mu)) < 1e-14
    # identity from the secular roots reproduces Q o Q as well
    out2 = oracle_mod.identity(p.lam, mu_sec)
    assert np.max(np.abs(out2 - (p.Q * p.Q).T)) < 1e-12


def test_secular_deflation(oracle_mod):
    # A block-diagonal Q: component j of eigenvector i is exactly 0 for the other
    # block, so those lam_i are eigenvalues of M_j unchanged.
    lam = np.array([-2.0, -0.5, 0.25, 1.5])
    c, s = math.cos(0.3), math.sin(0.3)
    Q = np.array([[c, s, 0, 0], [-s, c, 0, 0], [0, 0, c, -s], [0, 0, s, c]])
    A = (Q * lam) @ Q.T
    mu_sec = oracle_mod.secular_minor_eigvals(lam, Q, [0, 3])
    mu_jac = oracle_mod.minor_eigvals(A, [0, 3])
    assert np.max(np.abs(mu_sec - mu_jac)) < 1e-15


# ------------------------------------------------------------------ planted mistakes

def test_pins_reject_planted_mistakes(oracle_mod):
    """Feed the oracle's Eq. 1 routine plausible mistakes and show a pin fails."""
    A = inputs.goe(7, 3)
    n = A.shape[0]
    lam = oracle_mod.eigvals(A)
    mu = oracle_mod.minor_eigvals(A)
    good = oracle_mod.identity(lam, mu)
    assert grid_errors(A, lam, good)["col_sum"] < 1e-14

    def rejected(vsq):
        e = grid_errors(A, lam, vsq)
        return max(e["col_sum"], e.get("row_sum", 0), e["diag"]) > 1e-6 or e["min"] < 0

    # (1) a numerator factor lost: the last minor eigenvalue moved far away
    mu_drop = mu.copy()
    mu_drop[:, -1] = mu[:, -1] + 10.0
    assert rejected(oracle_mod.identity(lam, mu_drop))
    # (2) numerator and denominator swapped (the baseline listing's reading)
    assert rejected(1.0 / np.where(good == 0, np.inf, good))
    # (3) i and j exchanged
    assert rejected(good.T.copy())
    # (4) wrong minor: row removed but a different column removed
    bad_mu = np.empty_like(mu)
    for j in range(n):
        M = np.delete(np.delete(A, j, axis=0), (j + 1) % n, axis=1)
        bad_mu[j] = np.sort(np.linalg.eigvals(M).real)
    assert rejected(oracle_mod.identity(lam, bad_mu))
    # (5) one eigenvalue of A with the wrong sign
    lam_bad = lam.copy()
    lam_bad[0] = -lam_bad[0]
    assert rejected(oracle_mod.identity(np.sort(lam_bad), mu))


# ------------------------------------------------------------------ signed eigenvectors
# oracle.eigvecs returns the Jacobi eigenvectors themselves (signed), the oracle for
# signed components.  Each pin below is independent of the oracle's own code: a closed
# form, a defining equation, or brute force.  Vectors are compared up to one sign per
# eigenvector; the convention (largest-magnitude component positive) is pinned too.

def same_up_to_sign(a, b):
    """max over rows of min(|a_i - b_i|, |a_i + b_i|) (elementwise max)."""
    d1 = np.max(np.abs(a - b), axis=1)
    d2 = np.max(np.abs(a + b), axis=1)
    return float(np.max(np.minimum(d1, d2))) if a.size else 0.0


@pytest.mark.parametrize("seed", range(6))
def test_eigvecs_2x2_closed_form(oracle_mod, seed):
    g = np.random.default_rng(200 + seed)
    a, b, c = g.standard_normal(3)
    A = np.array([[a, b], [b, c]])
    h = math.sqrt(((a - c) / 2) ** 2 + b * b)
    lam_c = [(a + c) / 2 - h, (a + c) / 2 + h]
    # row 0 of (A - lam I) x = 0 gives x = (b, lam - a) for either eigenvalue
    expect = np.array([[b, l - a] for l in lam_c])
    expect /= np.linalg.norm(expect, axis=1)[:, None]
    lam, vec = oracle_mod.eigvecs(A)
    assert np.max(np.abs(lam - lam_c)) < 4e-16 * (abs(a) + abs(b) + abs(c) + 1)
    assert same_up_to_sign(vec, expect) < 1e-14


@pytest.mark.parametrize("n,a,b", [(3, 0.25, -0.5), (8, 0.0, 1.0), (17, -1.0, 0.75), (32, 0.0, 1.0)])
def test_eigvecs_toeplitz_sine_vectors(oracle_mod, n, a, b):
    """Tridiagonal Toeplitz: eigenvalue a + 2b cos(k pi/(n+1)) has the eigenvector
    sqrt(2/(n+1)) sin(j k pi/(n+1)), j = 1..n (1-based)."""
    A = inputs.toeplitz(n, a, b)
    k = np.arange(1, n + 1)
    lam_k = a + 2 * b * np.cos(k * np.pi / (n + 1))
    order = np.argsort(lam_k)                       # ascending relabelling
    j = np.arange(1, n + 1)
    vec_c = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(k[order], j) * np.pi / (n + 1))
    lam, vec = oracle_mod.eigvecs(A)
    assert np.max(np.abs(lam - lam_k[order])) < 1e-14
    assert same_up_to_sign(vec, vec_c) < 1e-13


@pytest.mark.parametrize("kind,n", [("goe", 9), ("goe", 40), ("wishart", 24), ("planted", 30)])
def test_eigvecs_residual_and_orthonormality(oracle_mod, kind, n):
    """A v_i = lam_i v_i (row i of vec) and V^T V = I: the definition of an
    orthonormal eigenbasis of a symmetric A."""
    A = (inputs.goe(n, 17) if kind == "goe" else inputs.wishart(n, 18) if kind == "wishart"
         else inputs.planted(n, 19, gap=1e-2).A)
    lam, vec = oracle_mod.eigvecs(A)
    norm = max(abs(lam[0]), abs(lam[-1]))
    resid = A @ vec.T - vec.T * lam[None, :]
    assert np.max(np.abs(resid)) < 1e-14 * n * norm
    assert np.max(np.abs(vec @ vec.T - np.eye(n))) < 1e-14 * n
    # the squared components are the oracle's |v_ij|^2 grid (both from one Jacobi run)
    _, vsq = oracle_mod.eig_vsq(A)
    assert np.max(np.abs(vec * vec - vsq)) < 1e-16 * n


@pytest.mark.parametrize("n", [3, 5, 8])
def test_eigvecs_inverse_iteration_brute_force(oracle_mod, n):
    A = inputs.goe(n, 40 + n)
    lam, vec = oracle_mod.eigvecs(A)
    for i in range(n):
        x = oracle_mod.inverse_iteration(A, lam[i] + 1e-9 * (1 + abs(lam[i])), iters=4)
        assert same_up_to_sign(vec[i:i + 1], x[None, :]) < 1e-14


def test_eigvecs_planted_q(oracle_mod):
    p = inputs.planted(40, 21, -1.0, 1.0, 1e-2)
    lam, vec = oracle_mod.eigvecs(p.A)
    assert np.max(np.abs(lam - p.lam)) < 1e-14
    assert same_up_to_sign(vec, p.Q.T) < 1e-12


def test_sign_convention():
    vec = np.array([[0.6, -0.8], [-0.8, -0.6], [0.0, 0.0]])
    import oracle
    out = oracle.sign_convention(vec)
    assert np.array_equal(out, [[-0.6, 0.8], [0.8, 0.6], [0.0, 0.0]])
    # ties: the first largest component decides
    t = oracle.sign_convention(np.array([[-0.5, 0.5, 0.5, -0.5]]))
    assert np.array_equal(t, [[0.5, -0.5, -0.5, 0.5]])


def test_eigvecs_pins_reject_planted_mistakes(oracle_mod):
    """A transposed result and a column permutation not applied to lam both fail."""
    A = inputs.goe(9, 33)
    lam, vec = oracle_mod.eigvecs(A)

    def residual(l, v):
        return float(np.max(np.abs(A @ v.T - v.T * l[None, :])))
    assert residual(lam, vec) < 1e-13
    assert residual(lam, vec.T.copy()) > 1e-3                 # transposed output
    perm = np.r_[1, 0, np.arange(2, 9)]
    assert residual(lam, vec[perm]) > 1e-3                    # vectors permuted, lam not


# ------------------------------------------------------------------ Hermitian A
# Sec. 2 states Eq. 1 for Hermitian matrices.  The oracle handles a complex Hermitian A
# through its real symmetric embedding; these pins do not use that construction.

def herm_goe(n, seed):
    g = np.random.default_rng(seed)
    G = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    return (G + G.conj().T) / 2


@pytest.mark.parametrize("seed", range(5))
def test_herm_2x2_closed_form(oracle_mod, seed):
    g = np.random.default_rng(400 + seed)
    a, c = g.standard_normal(2)
    b = complex(*g.standard_normal(2))
    A = np.array([[a, np.conj(b)], [b, c]])       # lower triangle holds b
    h = math.sqrt(((a - c) / 2) ** 2 + abs(b) ** 2)
    lp, lm = (a + c) / 2 + h, (a + c) / 2 - h
    # row 0 of (A - lam I) x = 0: (a - lam) x0 + conj(b) x1 = 0 -> x = (conj(b), lam - a)
    p0 = abs(b) ** 2 / (abs(b) ** 2 + (lp - a) ** 2)   # |x0|^2 / |x|^2 for lam_+
    expect = np.array([[1 - p0, p0], [p0, 1 - p0]])
    for method in (0, 2):
        out, lam = oracle_mod.components_herm(A, method=method, want_eigs=True)
        assert np.allclose(lam, [lm, lp], rtol=0, atol=1e-15 * (abs(lp) + abs(lm) + 1))
        assert np.max(np.abs(out - expect)) < 1e-14, method
    mu = oracle_mod.minor_eigvals_herm(A)
    assert mu[0, 0] == c and mu[1, 0] == a


@pytest.mark.parametrize("n,theta", [(5, 0.7), (16, -2.1), (33, 1.0)])
def test_herm_toeplitz_with_phase(oracle_mod, n, theta):
    """Off-diagonals e^{i theta} (below) and e^{-i theta} (above): the diagonal phase
    similarity D = diag(e^{i k theta}) makes it the real Toeplitz (0, 1), so the
    eigenvalues are 2 cos(k pi/(n+1)) and |v_ij|^2 the squared sine vectors."""
    A = np.zeros((n, n), dtype=complex)
    idx = np.arange(n - 1)
    A[idx + 1, idx] = np.exp(1j * theta)
    A[idx, idx + 1] = np.exp(-1j * theta)
    lam_c, vsq_c = toeplitz_closed(n, 0.0, 1.0)
    for method in (0, 2):
        out, lam = oracle_mod.components_herm(A, method=method, want_eigs=True)
        assert np.max(np.abs(lam - lam_c)) < 1e-14
        assert np.max(np.abs(out - vsq_c)) < 1e-13, method


def test_herm_real_input_matches_real_oracle(oracle_mod):
    A = inputs.goe(20, 5)
    a = oracle_mod.components(A, method=0)
    b = oracle_mod.components_herm(A.astype(complex), method=0)
    assert np.max(np.abs(a - b)) < 1e-15


@pytest.mark.parametrize("n", [7, 30])
def test_herm_against_lapack_and_invariants(oracle_mod, n):
    A = herm_goe(n, 500 + n)
    w, V = np.linalg.eigh(A)
    out, lam = oracle_mod.components_herm(A, method=0, want_eigs=True)
    assert np.max(np.abs(lam - w)) < 1e-13
    assert np.max(np.abs(out - (np.abs(V) ** 2).T)) < 1e-14 / np.min(np.diff(w))
    g = grid_errors(A.real, lam, out)        # the diagonal of a Hermitian A is real
    assert g["col_sum"] < 1e-13 and g["row_sum"] < 1e-13 and g["diag"] < 1e-13
    mu = oracle_mod.minor_eigvals_herm(A)
    lo = lam[:-1][None, :] - mu
    hi = mu - lam[1:][None, :]
    assert max(lo.max(), hi.max()) <= 1e-14                    # Cauchy interlacing
    assert np.max(np.abs(mu.sum(axis=1) - (np.trace(A).real - np.diag(A).real))) < 1e-12


def test_herm_planted_and_phase_invariance(oracle_mod):
    g = np.random.default_rng(9)
    n = 24
    Q, _ = np.linalg.qr(g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)))
    lam = np.sort(g.uniform(-1, 1, n))
    A = (Q * lam) @ Q.conj().T
    A = np.tril(A) + np.tril(A, -1).conj().T
    out = oracle_mod.components_herm(A, method=0)
    assert np.max(np.abs(out - (np.abs(Q) ** 2).T)) < 1e-12
    # a diagonal unitary similarity D A D^H multiplies each eigenvector's components by
    # phases only, so it changes no |v_ij|^2
    D = np.exp(1j * g.uniform(0, 2 * np.pi, n))
    B = (D[:, None] * A) * D.conj()[None, :]
    assert np.max(np.abs(oracle_mod.components_herm(B, method=0) - out)) < 1e-12
