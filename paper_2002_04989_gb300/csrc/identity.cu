// K-c: the eigenvector-eigenvalue identity (Eq. 1, Sec. 2) from the eigenvalues of
// A (lam, ascending) and of the minors M_j (mu, ascending):
//
//     |v_ij|^2 = prod_{k=1}^{n-1} (lam_i - mu_k) / prod_{k != i} (lam_i - lam_k).
//
// The paper splits both products into batches and multiplies per-batch ratios to
// keep partial products out of overflow and underflow (Algorithm 1 and the
// discussion of matrices beyond ~150x150 in Sec. 3).  Here each product is kept
// instead as a mantissa and a separate binary exponent: after every factor an
// integer test of the exponent field renormalises the mantissa by an exact power
// of two when it leaves [2^-400, 2^400].  No logarithms, no per-factor division.
//
// Signs: with interlacing (lam_k <= mu_k <= lam_{k+1}) every factor k < i of the
// numerator is >= 0 and every factor k >= i is <= 0, and the denominator has the
// same sign pattern, so the quotient is a quotient of magnitudes:
//   N_ij = prod_{k<i} (lam_i - mu_k) * prod_{k>=i} (mu_k - lam_i),
//   D_i  = prod_{k<i} (lam_i - lam_k) * prod_{k>i} (lam_k - lam_i).
// A numerator factor of the wrong sign can only come from rounding when the true
// factor is ~0; it is clamped to 0 (the component is then 0).  D_i == 0 (two equal
// eigenvalues of A) makes Eq. 1 0/0: the component is NaN and a status bit is set.
//
// D_i is shared by every j, so it is computed once per requested row (k_denominators,
// one thread per row, the rows of large problems spread over several blocks);
// k_identity stages mu^(j) in shared memory and gives each thread one (i, j).
#include "internal.cuh"

#include <cmath>

namespace eeid {
namespace {

// x *= f, keeping x in [2^-400, 2^400] by moving powers of two into ex.
__device__ __forceinline__ void mul_renorm(double& x, int& ex, double f) {
  x *= f;
  const int h = __double2hiint(x);
  const int eb = (h >> 20) & 0x7ff;
  if ((unsigned)(eb - (1023 - 400)) > 800u) {
    if (eb == 0) {
      if (((h & 0x7fffffff) | __double2loint(x)) != 0) {  // subnormal: lift by 2^600
        x *= 0x1p600;
        ex -= 600;
      }
    } else {
      // bring the exponent to 1022, i.e. |x| in [0.5, 1)
      x *= __hiloint2double((2045 - eb) << 20, 0);
      ex += eb - 1022;
    }
  }
}

// -x when `neg`, else x: a sign-bit flip on the high word, no FP64 instruction.
__device__ __forceinline__ double flip_if(double x, bool neg) {
  const int h = __double2hiint(x) ^ (neg ? int(0x80000000u) : 0);
  return __hiloint2double(h, __double2loint(x));
}

__device__ __forceinline__ double clamp_nonneg(double x) {
  return (__double2hiint(x) < 0) ? 0.0 : x;
}

__global__ void __launch_bounds__(kDenomThreads)
k_denominators(const DenomTask* __restrict__ tasks, const DenomItem* __restrict__ items,
               unsigned* status) {
  extern __shared__ double lam[];
  const DenomItem it = items[blockIdx.x];
  const DenomTask T = tasks[it.task];
  const int n = T.n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) lam[k] = T.lam[k];
  __syncthreads();
  bool degenerate = false;
  const int r = it.r0 + threadIdx.x;
  if (r < T.nrows) {
    const int i = T.rows[r];
    const double li = lam[i];
    double x = 1.0;
    int ex = 0;
    for (int k = 0; k < n; ++k) {
      if (k == i) continue;
      mul_renorm(x, ex, flip_if(li - lam[k], k > i));
    }
    if (x == 0.0) degenerate = true;
    int e2 = 0;
    const double mnt = (x == 0.0) ? 0.0 : frexp(x, &e2);
    T.dm[i] = mnt;
    T.de[i] = ex + e2;
  }
  if (__any_sync(0xffffffffu, degenerate) && (threadIdx.x & 31) == 0)
    atomicOr(status, (unsigned)ST_DEGENERATE);
  if (it.r0 == 0 && threadIdx.x == 0 && n >= 2) {
    double g = INFINITY;
    for (int k = 0; k + 1 < n; ++k) g = fmin(g, lam[k + 1] - lam[k]);
    const double sc = fmax(fabs(lam[0]), fabs(lam[n - 1]));
    if (!(g >= 1e-4 * sc)) atomicOr(status, (unsigned)ST_SMALL_GAP);
  }
}

__global__ void __launch_bounds__(kIdentityThreads)
k_identity(const IdentityProblem* __restrict__ probs, const IdentityItem* __restrict__ items) {
  extern __shared__ double mu[];
  const IdentityItem it = items[blockIdx.x];
  const IdentityProblem P = probs[it.prob];
  const int n = P.n;
  const double* src = P.mu + (size_t)it.col * (n - 1);
  for (int k = threadIdx.x; k < n - 1; k += blockDim.x) mu[k] = src[k];
  __syncthreads();
  const int r = it.r0 + threadIdx.x;
  if (r >= P.nrows) return;
  const int i = P.rows[r];
  const double li = P.lam[i];
  double x = 1.0;
  int ex = 0;
  for (int k = 0; k < n - 1; ++k) {
    // k < i: lam_i - mu_k >= 0 ; k >= i: mu_k - lam_i >= 0 (interlacing)
    const double f = clamp_nonneg(flip_if(li - mu[k], k >= i));
    mul_renorm(x, ex, f);
  }
  const double dm = P.dm[i];
  double v;
  if (dm == 0.0) {
    v = NAN;
  } else {
    v = scalbn(x / dm, ex - P.de[i]);
  }
  P.out[(size_t)r * P.ncols + it.col] = v;
}

}  // namespace

static std::atomic<uint64_t> g_denom_limit_set{0}, g_identity_limit_set{0};

cudaError_t preload_identity() {
  cudaError_t e = raise_smem_limit_once((const void*)k_denominators, g_denom_limit_set);
  if (e == cudaSuccess) e = raise_smem_limit_once((const void*)k_identity, g_identity_limit_set);
  return e;
}

cudaError_t launch_denominators(const DenomTask* tasks, const DenomItem* items, int nitems,
                                int max_n, unsigned* status, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_n * sizeof(double);
  cudaError_t e = raise_smem_limit_once((const void*)k_denominators, g_denom_limit_set);
  if (e != cudaSuccess) return e;
  k_denominators<<<nitems, kDenomThreads, smem, s>>>(tasks, items, status);
  return cudaGetLastError();
}

cudaError_t launch_identity(const IdentityProblem* probs, const IdentityItem* items, int nitems,
                            int max_n, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)(max_n > 1 ? max_n - 1 : 1) * sizeof(double);
  cudaError_t e = raise_smem_limit_once((const void*)k_identity, g_identity_limit_set);
  if (e != cudaSuccess) return e;
  k_identity<<<nitems, kIdentityThreads, smem, s>>>(probs, items);
  return cudaGetLastError();
}

}  // namespace eeid
