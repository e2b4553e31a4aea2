/*
 * Oracle for the eigenvector-eigenvalue identity path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load or call this library.  The product path (the CUDA library and its
 * Python binding) never links, imports or executes anything in this directory,
 * and this file shares no code, header or constant table with it.
 *
 * Plain, slow, obviously-correct CPU implementation in `long double`
 * (x87 80-bit on x86-64, IEEE binary128 on aarch64).  Every function follows a
 * definition written out in the paper or a textbook method named in its comment:
 *
 *   oracle_eig / oracle_eigvals       cyclic-by-row Jacobi (Golub & Van Loan,
 *                                     "Matrix Computations", sec. 8.5) -- the
 *                                     plain definition of the spectrum and of the
 *                                     unit eigenvectors of a symmetric A (Sec. 2).
 *   oracle_eigvecs                    the same Jacobi run's unit eigenvectors
 *                                     themselves, signed (each is defined up to its
 *                                     sign; tests fix it by the convention that the
 *                                     largest-magnitude component is positive).
 *   oracle_minor_eigvals              the same Jacobi on the minor M_j, i.e. A with
 *                                     row and column j removed (Sec. 2, definition
 *                                     under Eq. 1).
 *   oracle_identity                   Eq. 1 itself, from given eigenvalues, two ways:
 *                                     mode 0 = numerator and denominator products
 *                                     exactly as printed, each renormalised with
 *                                     frexpl after every factor (this is the point of
 *                                     the paper's batching, Sec. 3: keep partial
 *                                     products out of overflow/underflow);
 *                                     mode 1 = the same quotient regrouped into
 *                                     factor-wise ratios (algebraically identical).
 *   oracle_components                 A -> |v_ij|^2 in long double end to end:
 *                                     method 0/1 = Jacobi eigenvalues of A and of
 *                                     every M_j, then Eq. 1 (mode 0/1);
 *                                     method 2 = the plain definition V o V from the
 *                                     Jacobi eigenvectors (no minors).
 *   oracle_secular_minor_eigvals      eigenvalues of M_j from a known
 *                                     eigendecomposition A = Q diag(lam) Q^T as the
 *                                     roots of sum_i Q_ji^2 / (mu - lam_i) = 0
 *                                     (Cramer's rule: ((mu I - A)^-1)_jj =
 *                                     det(mu I - M_j) / det(mu I - A); textbook, not
 *                                     the paper), one bisection per pole interval.
 *   oracle_components_herm,           the same for a complex Hermitian A (Sec. 2 states
 *   oracle_minor_eigvals_herm         Eq. 1 for Hermitian matrices), through the real
 *                                     symmetric 2n x 2n embedding [[Re, -Im], [Im, Re]],
 *                                     whose spectrum is A's with every eigenvalue doubled
 *                                     (textbook); Jacobi as above on the embedding.
 *   oracle_inverse_iteration          brute-force eigenvector by shifted inverse
 *                                     iteration with Gaussian elimination (partial
 *                                     pivoting); for tiny n only.
 *
 * Conventions: matrices are row-major double with leading dimension lda; only the
 * lower triangle (i >= j, element A[i*lda + j]) is read.  Eigenvalues are returned
 * ascending; indices are 0-based; out[r*ncols + c] = |v_{rows[r], cols[c]}|^2 where
 * i = rows[r] indexes the i-th smallest eigenvalue and j = cols[c] the component.
 * Return value: 0 on success, negative on bad arguments or allocation failure.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double real;

#define ORACLE_MAX_SWEEPS 100

/* ---------------------------------------------------------------- helpers */

/* Full symmetric long-double copy of A (lower triangle read), with row/column
 * `skip` removed when skip >= 0 (the minor M_skip).  Result is m x m, m = n or n-1. */
static void load_sym(int64_t n, const double* A, int64_t lda, int64_t skip, real* S) {
  int64_t m = (skip >= 0) ? n - 1 : n;
  for (int64_t r = 0; r < m; ++r) {
    int64_t i = (skip >= 0 && r >= skip) ? r + 1 : r;
    for (int64_t c = 0; c <= r; ++c) {
      int64_t j = (skip >= 0 && c >= skip) ? c + 1 : c;
      real v = (real)A[i * lda + j];
      S[r * m + c] = v;
      S[c * m + r] = v;
    }
  }
}

/* Cyclic-by-row Jacobi on the symmetric m x m matrix S (full storage, overwritten).
 * On return the diagonal of S holds the eigenvalues (unsorted).  If V != NULL it is
 * set to the accumulated rotations: column i of V is the unit eigenvector for S[i][i].
 *
 * Each rotation J(p,q,theta) is chosen so that (J^T S J)_pq = 0.  With
 * tau = (s_qq - s_pp) / (2 s_pq) the tangent t = tan(theta) is the root of
 * t^2 + 2 tau t - 1 = 0 of smaller magnitude; c = 1/sqrt(1+t^2), s = t c.  Then
 * s_pp <- s_pp - t s_pq, s_qq <- s_qq + t s_pq, s_pq <- 0 and, for k != p,q,
 * (s_kp, s_kq) <- (c s_kp - s s_kq, s s_kp + c s_kq).
 *
 * An off-diagonal entry is treated as zero when it is negligible next to the
 * geometric mean of its two diagonal entries (relative criterion) or below an
 * absolute floor far under working precision; a sweep with no rotation ends it. */
static int jacobi(int64_t m, real* S, real* V) {
  if (V) {
    for (int64_t i = 0; i < m * m; ++i) V[i] = 0;
    for (int64_t i = 0; i < m; ++i) V[i * m + i] = 1;
  }
  real fro = 0;
  for (int64_t i = 0; i < m * m; ++i) fro += S[i] * S[i];
  fro = sqrtl(fro);
  const real floor_abs = LDBL_EPSILON * LDBL_EPSILON * fro;
  for (int sweep = 0; sweep < ORACLE_MAX_SWEEPS; ++sweep) {
    int64_t rotations = 0;
    for (int64_t p = 0; p < m - 1; ++p) {
      for (int64_t q = p + 1; q < m; ++q) {
        real spq = S[p * m + q];
        real spp = S[p * m + p], sqq = S[q * m + q];
        if (fabsl(spq) <= floor_abs || fabsl(spq) <= LDBL_EPSILON * sqrtl(fabsl(spp * sqq)) * 0.5L) {
          S[p * m + q] = 0;
          S[q * m + p] = 0;
          continue;
        }
        ++rotations;
        real tau = (sqq - spp) / (2 * spq);
        real t = 1 / (fabsl(tau) + sqrtl(1 + tau * tau));
        if (tau < 0) t = -t;
        real c = 1 / sqrtl(1 + t * t);
        real s = t * c;
        for (int64_t k = 0; k < m; ++k) {
          if (k == p || k == q) continue;
          real skp = S[k * m + p], skq = S[k * m + q];
          real nkp = c * skp - s * skq;
          real nkq = s * skp + c * skq;
          S[k * m + p] = nkp; S[p * m + k] = nkp;
          S[k * m + q] = nkq; S[q * m + k] = nkq;
        }
        S[p * m + p] = spp - t * spq;
        S[q * m + q] = sqq + t * spq;
        S[p * m + q] = 0;
        S[q * m + p] = 0;
        if (V) {
          for (int64_t k = 0; k < m; ++k) {
            real vkp = V[k * m + p], vkq = V[k * m + q];
            V[k * m + p] = c * vkp - s * vkq;
            V[k * m + q] = s * vkp + c * vkq;
          }
        }
      }
    }
    if (rotations == 0) return 0;
  }
  return 1; /* did not converge within the sweep limit (not expected) */
}

/* Diagonal of S into lam (ascending); V's columns permuted alongside (may be NULL). */
static void sorted_eig(int64_t m, const real* S, real* V, real* lam) {
  for (int64_t i = 0; i < m; ++i) lam[i] = S[i * m + i];
  for (int64_t a = 0; a < m; ++a) { /* selection sort: plain and stable enough */
    int64_t best = a;
    for (int64_t b = a + 1; b < m; ++b)
      if (lam[b] < lam[best]) best = b;
    if (best != a) {
      real t = lam[a]; lam[a] = lam[best]; lam[best] = t;
      if (V)
        for (int64_t k = 0; k < m; ++k) {
          real u = V[k * m + a]; V[k * m + a] = V[k * m + best]; V[k * m + best] = u;
        }
    }
  }
}

/* Eigenvalues (ascending) of A (skip < 0) or of the minor M_skip, in long double. */
static int eigvals_ld(int64_t n, const double* A, int64_t lda, int64_t skip, real* lam) {
  int64_t m = (skip >= 0) ? n - 1 : n;
  if (m <= 0) return 0;
  real* S = (real*)malloc(sizeof(real) * m * m);
  if (!S) return -2;
  load_sym(n, A, lda, skip, S);
  jacobi(m, S, NULL);
  sorted_eig(m, S, NULL, lam);
  free(S);
  return 0;
}

/* Eq. 1 for one (i, j), given the n eigenvalues of A and the n-1 of M_j, both
 * ascending, in long double.
 *   mode 0: numerator prod_{k=1}^{n-1} (lam_i - mu_k) and denominator
 *           prod_{k != i} (lam_i - lam_k) accumulated separately, each kept as
 *           mantissa * 2^exponent with frexpl after every factor; then divided.
 *   mode 1: the quotient regrouped factor by factor,
 *           prod_{k<i} (lam_i - mu_k)/(lam_i - lam_k) *
 *           prod_{k>=i} (lam_i - mu_k)/(lam_i - lam_{k+1}),
 *           which is the same rational expression (the denominator's factors
 *           k = i+1..n-1 re-indexed as k+1); with interlaced spectra each ratio
 *           lies in [0, 1]. */
static real identity_one(int64_t n, const real* lam, const real* mu, int64_t i, int mode) {
  if (mode == 0) {
    real num = 1, den = 1;
    int en = 0, ed = 0, e;
    for (int64_t k = 0; k < n - 1; ++k) {
      num *= (lam[i] - mu[k]);
      num = frexpl(num, &e);
      en += e;
    }
    for (int64_t k = 0; k < n; ++k) {
      if (k == i) continue;
      den *= (lam[i] - lam[k]);
      den = frexpl(den, &e);
      ed += e;
    }
    return ldexpl(num / den, en - ed);
  } else {
    real prod = 1;
    for (int64_t k = 0; k < i; ++k) prod *= (lam[i] - mu[k]) / (lam[i] - lam[k]);
    for (int64_t k = i; k < n - 1; ++k) prod *= (lam[i] - mu[k]) / (lam[i] - lam[k + 1]);
    return prod;
  }
}

static int check_indices(int64_t n, const int64_t* idx, int64_t cnt) {
  for (int64_t a = 0; a < cnt; ++a)
    if (idx[a] < 0 || idx[a] >= n) return -1;
  return 0;
}

/* ---------------------------------------------------------------- exports */

/* Ascending eigenvalues of A (n values). */
int oracle_eigvals(int64_t n, const double* A, int64_t lda, double* lam) {
  if (n < 0 || (n > 0 && (!A || !lam || lda < n))) return -1;
  if (n == 0) return 0;
  real* l = (real*)malloc(sizeof(real) * n);
  if (!l) return -2;
  int rc = eigvals_ld(n, A, lda, -1, l);
  for (int64_t i = 0; i < n; ++i) lam[i] = (double)l[i];
  free(l);
  return rc;
}

/* Ascending eigenvalues and the squared components of the unit eigenvectors:
 * vsq[i*n + j] = V[j][i]^2 = |v_ij|^2 (row i = i-th smallest eigenvalue). */
int oracle_eig(int64_t n, const double* A, int64_t lda, double* lam, double* vsq) {
  if (n < 0 || (n > 0 && (!A || !lam || !vsq || lda < n))) return -1;
  if (n == 0) return 0;
  real* S = (real*)malloc(sizeof(real) * n * n);
  real* V = (real*)malloc(sizeof(real) * n * n);
  real* l = (real*)malloc(sizeof(real) * n);
  if (!S || !V || !l) { free(S); free(V); free(l); return -2; }
  load_sym(n, A, lda, -1, S);
  jacobi(n, S, V);
  sorted_eig(n, S, V, l);
  for (int64_t i = 0; i < n; ++i) {
    lam[i] = (double)l[i];
    for (int64_t j = 0; j < n; ++j) vsq[i * n + j] = (double)(V[j * n + i] * V[j * n + i]);
  }
  free(S); free(V); free(l);
  return 0;
}

/* Unit eigenvectors themselves (signed): vec[i*n + j] = V[j][i]. */
int oracle_eigvecs(int64_t n, const double* A, int64_t lda, double* lam, double* vec) {
  if (n < 0 || (n > 0 && (!A || !lam || !vec || lda < n))) return -1;
  if (n == 0) return 0;
  real* S = (real*)malloc(sizeof(real) * n * n);
  real* V = (real*)malloc(sizeof(real) * n * n);
  real* l = (real*)malloc(sizeof(real) * n);
  if (!S || !V || !l) { free(S); free(V); free(l); return -2; }
  load_sym(n, A, lda, -1, S);
  jacobi(n, S, V);
  sorted_eig(n, S, V, l);
  for (int64_t i = 0; i < n; ++i) {
    lam[i] = (double)l[i];
    for (int64_t j = 0; j < n; ++j) vec[i * n + j] = (double)V[j * n + i];
  }
  free(S); free(V); free(l);
  return 0;
}

/* Ascending eigenvalues of each minor M_j, j = cols[c]: mu[c*(n-1) + k]. */
int oracle_minor_eigvals(int64_t n, const double* A, int64_t lda, const int64_t* cols,
                         int64_t ncols, double* mu) {
  if (n < 1 || !A || lda < n || ncols < 0 || (ncols > 0 && (!cols || !mu))) return -1;
  if (check_indices(n, cols, ncols)) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t c = 0; c < ncols; ++c) {
    real* l = (real*)malloc(sizeof(real) * (n > 1 ? n - 1 : 1));
    if (!l) { bad |= 1; continue; }
    if (eigvals_ld(n, A, lda, cols[c], l)) bad |= 1;
    for (int64_t k = 0; k < n - 1; ++k) mu[c * (n - 1) + k] = (double)l[k];
    free(l);
  }
  return bad ? -2 : 0;
}

/* Eq. 1 from given eigenvalues: lam[n] (ascending) and mu[c*(n-1) + k] for the
 * minors of the requested columns.  out[r*ncols + c] for eigen-index rows[r]. */
int oracle_identity(int64_t n, const double* lam, const double* mu, const int64_t* rows,
                    int64_t nrows, int64_t ncols, int mode, double* out) {
  if (n < 1 || !lam || nrows < 0 || ncols < 0 || (mode != 0 && mode != 1)) return -1;
  if (nrows > 0 && ncols > 0 && (!rows || !out || (n > 1 && !mu))) return -1;
  if (check_indices(n, rows, nrows)) return -1;
  real* l = (real*)malloc(sizeof(real) * n);
  real* u = (real*)malloc(sizeof(real) * (n > 1 ? n - 1 : 1));
  if (!l || !u) { free(l); free(u); return -2; }
  for (int64_t k = 0; k < n; ++k) l[k] = lam[k];
  for (int64_t c = 0; c < ncols; ++c) {
    for (int64_t k = 0; k < n - 1; ++k) u[k] = mu[c * (n - 1) + k];
    for (int64_t r = 0; r < nrows; ++r)
      out[r * ncols + c] = (double)identity_one(n, l, u, rows[r], mode);
  }
  free(l); free(u);
  return 0;
}

/* A -> |v_ij|^2 entirely in long double.
 *   method 0: Jacobi eigenvalues of A and of each M_j, then Eq. 1 (mode 0).
 *   method 1: as method 0 with Eq. 1 in mode 1.
 *   method 2: V o V from the Jacobi eigenvectors of A (plain definition; lam_out
 *             is filled, mu_out is left untouched).
 * rows/cols may be NULL with nrows/ncols = n to mean "all".
 * lam_out[n] and mu_out[ncols*(n-1)] are optional outputs (NULL to skip). */
int oracle_components(int64_t n, const double* A, int64_t lda, const int64_t* rows,
                      int64_t nrows, const int64_t* cols, int64_t ncols, int method,
                      double* out, double* lam_out, double* mu_out) {
  if (n < 1 || !A || lda < n || nrows < 0 || ncols < 0 || method < 0 || method > 2) return -1;
  if ((rows && check_indices(n, rows, nrows)) || (cols && check_indices(n, cols, ncols))) return -1;
  if ((!rows && nrows != n) || (!cols && ncols != n)) return -1;
  if (nrows > 0 && ncols > 0 && !out) return -1;
  int rc = 0;
  if (method == 2) {
    real* S = (real*)malloc(sizeof(real) * n * n);
    real* V = (real*)malloc(sizeof(real) * n * n);
    real* l = (real*)malloc(sizeof(real) * n);
    if (!S || !V || !l) { free(S); free(V); free(l); return -2; }
    load_sym(n, A, lda, -1, S);
    jacobi(n, S, V);
    sorted_eig(n, S, V, l);
    for (int64_t r = 0; r < nrows; ++r)
      for (int64_t c = 0; c < ncols; ++c) {
        int64_t i = rows ? rows[r] : r, j = cols ? cols[c] : c;
        out[r * ncols + c] = (double)(V[j * n + i] * V[j * n + i]);
      }
    if (lam_out) for (int64_t k = 0; k < n; ++k) lam_out[k] = (double)l[k];
    free(S); free(V); free(l);
    return 0;
  }
  real* l = (real*)malloc(sizeof(real) * n);
  if (!l) return -2;
  rc = eigvals_ld(n, A, lda, -1, l);
  if (lam_out) for (int64_t k = 0; k < n; ++k) lam_out[k] = (double)l[k];
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t c = 0; c < ncols; ++c) {
    int64_t j = cols ? cols[c] : c;
    real* u = (real*)malloc(sizeof(real) * (n > 1 ? n - 1 : 1));
    if (!u) { bad |= 1; continue; }
    if (eigvals_ld(n, A, lda, j, u)) bad |= 1;
    if (mu_out) for (int64_t k = 0; k < n - 1; ++k) mu_out[c * (n - 1) + k] = (double)u[k];
    for (int64_t r = 0; r < nrows; ++r) {
      int64_t i = rows ? rows[r] : r;
      out[r * ncols + c] = (double)identity_one(n, l, u, i, method);
    }
    free(u);
  }
  free(l);
  return (rc || bad) ? -2 : 0;
}

/* Eigenvalues of the minors M_j of A = Q diag(lam) Q^T, from (lam, Q) alone.
 * lam[n] strictly ascending; Q row-major with Q[j*n + i] = component j of the unit
 * eigenvector for lam[i].  For each requested j, with weights w_i = Q_ji^2:
 *   det(mu I - M_j) / det(mu I - A) = sum_i w_i / (mu - lam_i),
 * so every pole lam_i with w_i > 0 is separated from the next such pole by exactly
 * one root (the sum falls from +inf to -inf between them), and every lam_i with
 * w_i == 0 is itself an eigenvalue of M_j.  Each root is found by bisection on its
 * pole interval until the bracket cannot be halved further in long double.
 * mu[c*(n-1) + k], ascending. */
int oracle_secular_minor_eigvals(int64_t n, const double* lam, const double* Q,
                                 const int64_t* cols, int64_t ncols, double* mu) {
  if (n < 1 || !lam || !Q || ncols < 0 || (ncols > 0 && (!cols || !mu))) return -1;
  if (check_indices(n, cols, ncols)) return -1;
  for (int64_t k = 0; k + 1 < n; ++k)
    if (!(lam[k] < lam[k + 1])) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t c = 0; c < ncols; ++c) {
    int64_t j = cols[c];
    real* pole = (real*)malloc(sizeof(real) * n);
    real* w = (real*)malloc(sizeof(real) * n);
    real* roots = (real*)malloc(sizeof(real) * n);
    if (!pole || !w || !roots) { free(pole); free(w); free(roots); bad |= 1; continue; }
    int64_t np = 0, nr = 0;
    for (int64_t i = 0; i < n; ++i) {
      real q = Q[j * n + i];
      if (q == 0) {
        roots[nr++] = lam[i]; /* deflated: lam_i is an eigenvalue of M_j */
      } else {
        pole[np] = lam[i];
        w[np] = q * q;
        ++np;
      }
    }
    for (int64_t k = 0; k + 1 < np; ++k) {
      real lo = pole[k], hi = pole[k + 1];
      for (;;) {
        real mid = lo + (hi - lo) / 2;
        if (!(mid > lo && mid < hi)) break;
        real f = 0;
        for (int64_t i = 0; i < np; ++i) f += w[i] / (mid - pole[i]);
        if (f > 0) lo = mid; else hi = mid;
      }
      roots[nr++] = lo + (hi - lo) / 2;
    }
    /* ascending order (deflated roots interleave with the secular ones) */
    for (int64_t a = 0; a < nr; ++a) {
      int64_t best = a;
      for (int64_t b = a + 1; b < nr; ++b)
        if (roots[b] < roots[best]) best = b;
      real t = roots[a]; roots[a] = roots[best]; roots[best] = t;
    }
    if (nr != n - 1) bad |= 1;
    for (int64_t k = 0; k < n - 1 && k < nr; ++k) mu[c * (n - 1) + k] = (double)roots[k];
    free(pole); free(w); free(roots);
  }
  return bad ? -2 : 0;
}

/* Brute-force unit eigenvector for the eigenvalue nearest `shift`:
 * `iters` steps of x <- (A - shift I)^{-1} x / ||.||, starting from x = (1,...,1)
 * plus a small index ramp, each solve by Gaussian elimination with partial
 * pivoting in long double.  x[n] out.  For tiny n (brute force) only. */
int oracle_inverse_iteration(int64_t n, const double* A, int64_t lda, double shift, int iters,
                             double* x) {
  if (n < 1 || !A || lda < n || !x || iters < 1) return -1;
  real* M = (real*)malloc(sizeof(real) * n * n);
  real* b = (real*)malloc(sizeof(real) * n);
  real* y = (real*)malloc(sizeof(real) * n);
  int64_t* piv = (int64_t*)malloc(sizeof(int64_t) * n);
  if (!M || !b || !y || !piv) { free(M); free(b); free(y); free(piv); return -2; }
  for (int64_t i = 0; i < n; ++i) b[i] = 1 + (real)i / (real)(7 * n);
  for (int it = 0; it < iters; ++it) {
    load_sym(n, A, lda, -1, M);
    for (int64_t i = 0; i < n; ++i) M[i * n + i] -= (real)shift;
    for (int64_t i = 0; i < n; ++i) { y[i] = b[i]; piv[i] = i; }
    /* LU with partial pivoting, applied to y as we go */
    for (int64_t k = 0; k < n; ++k) {
      int64_t p = k;
      for (int64_t r = k + 1; r < n; ++r)
        if (fabsl(M[r * n + k]) > fabsl(M[p * n + k])) p = r;
      if (p != k) {
        for (int64_t c = 0; c < n; ++c) { real t = M[k * n + c]; M[k * n + c] = M[p * n + c]; M[p * n + c] = t; }
        real t = y[k]; y[k] = y[p]; y[p] = t;
      }
      if (M[k * n + k] == 0) M[k * n + k] = LDBL_MIN; /* exactly singular: nudge */
      for (int64_t r = k + 1; r < n; ++r) {
        real f = M[r * n + k] / M[k * n + k];
        for (int64_t c = k; c < n; ++c) M[r * n + c] -= f * M[k * n + c];
        y[r] -= f * y[k];
      }
    }
    for (int64_t k = n - 1; k >= 0; --k) {
      real s = y[k];
      for (int64_t c = k + 1; c < n; ++c) s -= M[k * n + c] * b[c];
      b[k] = s / M[k * n + k];
    }
    real nrm = 0;
    for (int64_t i = 0; i < n; ++i) nrm += b[i] * b[i];
    nrm = sqrtl(nrm);
    for (int64_t i = 0; i < n; ++i) b[i] /= nrm;
  }
  for (int64_t i = 0; i < n; ++i) x[i] = (double)b[i];
  free(M); free(b); free(y); free(piv);
  return 0;
}

/* ---------------------------------------------------------------- Hermitian A */

/* Real symmetric embedding of a complex Hermitian matrix H (Sec. 2 states Eq. 1 for
 * Hermitian matrices).  H is row-major with interleaved (re, im) doubles, leading
 * dimension lda in complex elements, lower triangle read (H_cr = conj(H_rc)); row and
 * column `skip` are removed when skip >= 0.  With m = n or n - 1 the result is the
 * 2m x 2m matrix E = [[Re H, -Im H], [Im H, Re H]] (full storage).  H v = lam v with
 * v = a + i b is E (a; b) = lam (a; b), and E (-b; a) = lam (-b; a) as well, so every
 * eigenvalue of H is a double eigenvalue of E.  Textbook, not the paper. */
static void load_herm_embed(int64_t n, const double* H, int64_t lda, int64_t skip, real* E) {
  int64_t m = (skip >= 0) ? n - 1 : n;
  int64_t M = 2 * m;
  for (int64_t r = 0; r < m; ++r) {
    int64_t i = (skip >= 0 && r >= skip) ? r + 1 : r;
    for (int64_t c = 0; c <= r; ++c) {
      int64_t j = (skip >= 0 && c >= skip) ? c + 1 : c;
      real re = (real)H[2 * (i * lda + j)];
      real im = (r == c) ? 0 : (real)H[2 * (i * lda + j) + 1];  /* diagonal is real */
      /* H_rc = re + i im, H_cr = re - i im */
      E[r * M + c] = re;            E[c * M + r] = re;
      E[(m + r) * M + (m + c)] = re; E[(m + c) * M + (m + r)] = re;
      E[(m + r) * M + c] = im;      E[c * M + (m + r)] = im;      /* Im H_rc, and its transpose */
      E[(m + c) * M + r] = -im;     E[r * M + (m + c)] = -im;     /* Im H_cr = -im */
    }
  }
}

/* Ascending eigenvalues of H (skip < 0) or of its minor without row/col skip, from the
 * Jacobi eigenvalues of the embedding (each appears twice; the pair is averaged).  With
 * vsq != NULL (skip < 0 only) also the squared moduli of the unit eigenvectors:
 * vsq[i*n + j] = |v_ij|^2 = half the sum, over the two embedding eigenvectors of the
 * pair, of x_j^2 + x_{n+j}^2 (the diagonal of the projector onto the pair's plane). */
static int herm_eig_ld(int64_t n, const double* H, int64_t lda, int64_t skip, real* lam,
                       real* vsq) {
  int64_t m = (skip >= 0) ? n - 1 : n;
  if (m <= 0) return 0;
  int64_t M = 2 * m;
  real* E = (real*)malloc(sizeof(real) * M * M);
  real* V = vsq ? (real*)malloc(sizeof(real) * M * M) : NULL;
  real* l = (real*)malloc(sizeof(real) * M);
  if (!E || !l || (vsq && !V)) { free(E); free(V); free(l); return -2; }
  load_herm_embed(n, H, lda, skip, E);
  jacobi(M, E, V);
  sorted_eig(M, E, V, l);
  for (int64_t i = 0; i < m; ++i) {
    lam[i] = (l[2 * i] + l[2 * i + 1]) / 2;
    if (vsq)
      for (int64_t j = 0; j < m; ++j) {
        real s = 0;
        for (int64_t t = 2 * i; t <= 2 * i + 1; ++t)
          s += V[j * M + t] * V[j * M + t] + V[(m + j) * M + t] * V[(m + j) * M + t];
        vsq[i * m + j] = s / 2;
      }
  }
  free(E); free(V); free(l);
  return 0;
}

/* Hermitian A -> |v_ij|^2 in long double (same conventions as oracle_components; A is
 * interleaved complex with leading dimension lda in complex elements):
 *   method 0: eigenvalues of A and of each minor M_j from the embedding, then Eq. 1;
 *   method 2: |v_ij|^2 from the embedding's eigenvectors (plain definition). */
int oracle_components_herm(int64_t n, const double* A, int64_t lda, const int64_t* rows,
                           int64_t nrows, const int64_t* cols, int64_t ncols, int method,
                           double* out, double* lam_out) {
  if (n < 1 || !A || lda < n || nrows < 0 || ncols < 0 || (method != 0 && method != 2)) return -1;
  if ((rows && check_indices(n, rows, nrows)) || (cols && check_indices(n, cols, ncols))) return -1;
  if ((!rows && nrows != n) || (!cols && ncols != n)) return -1;
  if (nrows > 0 && ncols > 0 && !out) return -1;
  real* l = (real*)malloc(sizeof(real) * n);
  real* vsq = method == 2 ? (real*)malloc(sizeof(real) * n * n) : NULL;
  if (!l || (method == 2 && !vsq)) { free(l); free(vsq); return -2; }
  int rc = herm_eig_ld(n, A, lda, -1, l, vsq);
  if (lam_out) for (int64_t k = 0; k < n; ++k) lam_out[k] = (double)l[k];
  int bad = 0;
  if (method == 2) {
    for (int64_t r = 0; r < nrows; ++r)
      for (int64_t c = 0; c < ncols; ++c) {
        int64_t i = rows ? rows[r] : r, j = cols ? cols[c] : c;
        out[r * ncols + c] = (double)vsq[i * n + j];
      }
  } else {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int64_t c = 0; c < ncols; ++c) {
      int64_t j = cols ? cols[c] : c;
      real* u = (real*)malloc(sizeof(real) * (n > 1 ? n - 1 : 1));
      if (!u) { bad |= 1; continue; }
      if (herm_eig_ld(n, A, lda, j, u, NULL)) bad |= 1;
      for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        out[r * ncols + c] = (double)identity_one(n, l, u, i, 0);
      }
      free(u);
    }
  }
  free(l); free(vsq);
  return (rc || bad) ? -2 : 0;
}

/* Ascending eigenvalues of the minors M_j of Hermitian A: mu[c*(n-1) + k]. */
int oracle_minor_eigvals_herm(int64_t n, const double* A, int64_t lda, const int64_t* cols,
                              int64_t ncols, double* mu) {
  if (n < 1 || !A || lda < n || ncols < 0 || (ncols > 0 && (!cols || !mu))) return -1;
  if (check_indices(n, cols, ncols)) return -1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t c = 0; c < ncols; ++c) {
    real* u = (real*)malloc(sizeof(real) * (n > 1 ? n - 1 : 1));
    if (!u) { bad |= 1; continue; }
    if (herm_eig_ld(n, A, lda, cols[c], u, NULL)) bad |= 1;
    for (int64_t k = 0; k < n - 1; ++k) mu[c * (n - 1) + k] = (double)u[k];
    free(u);
  }
  return bad ? -2 : 0;
}

/* Number of bits of precision of `real` on this host (64 on x86 x87, 113 on
 * aarch64 binary128), so tests can state which oracle precision ran. */
int oracle_real_mant_dig(void) { return LDBL_MANT_DIG; }
