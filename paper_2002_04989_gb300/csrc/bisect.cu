// K-b: eigenvalues of symmetric tridiagonal matrices by Sturm-sequence bisection,
// one lane per eigenvalue.
//
// Why: Eq. 1 (Sec. 2) consumes the eigenvalues of A and of each minor M_j; after
// K-a both are symmetric tridiagonals T (diagonal d, off-diagonal e).  The number
// of eigenvalues of T below x equals the number of sign changes in the sequence of
// leading principal minors p_0 = 1, p_1, ..., p_m of T - xI, which obey
//     p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1}.
// Bisection on that count brackets each eigenvalue independently.
//
// GB300 choices:
//  * Division-free recurrence.  FP64 divide costs about ten FP64-pipe slots on this
//    part (measured), the ratio form of the count needs one per step; the
//    three-term form above needs one subtract, one multiply and one FMA.  The
//    computed signs are those of an exact recurrence for a tridiagonal whose
//    diagonal is perturbed by O(eps (|d|+|x|)) and whose e^2 by O(eps) relative, the
//    same backward error as the ratio form.  The pair (p_{i-1}, p_i) is rescaled by
//    an exact power of two whenever its larger exponent leaves [2^-400, 2^400]; a
//    zero p_i is replaced by 2^-900 with the sign opposite to p_{i-1} (the
//    eigenvalue at x is counted below x).  Exponent tests and sign counting are
//    integer operations on the high word, off the FP64 pipe.
//  * T is scaled by an exact power of two so that its Gershgorin bound lies in
//    [0.5, 1): no rounding, and growth per step is at most a factor 4.
//  * Minor eigenvalues are seeded by interlacing: lam_k(A) <= mu_k(M_j) <= lam_{k+1}(A)
//    (Cauchy), widened by 2^-40 ||T|| and verified with two Sturm counts; a failed
//    check falls back to the Gershgorin bracket.
//  * (d_i, e_{i-1}^2) are staged in shared memory as one 16-byte pair per step and
//    read as a warp-wide broadcast; each warp loops until a warp vote finds every
//    lane converged.
#include "internal.cuh"

namespace eeid {
namespace {

constexpr int kTinyBiasedExp = 1023 - 900;  // 2^-900
constexpr int kMaxIter = 120;

__device__ __forceinline__ int hi_of(double x) { return __double2hiint(x); }
__device__ __forceinline__ int bexp(int hi) { return (hi >> 20) & 0x7ff; }

// Number of eigenvalues of the (scaled) tridiagonal below x.
__device__ __forceinline__ int sturm_count(const double2* __restrict__ de, int m, double x) {
  double pm = 1.0;
  double pc = de[0].x - x;
  int hc = hi_of(pc);
  if (bexp(hc) == 0) {  // p_1 zero or subnormal
    const bool zero = ((hc & 0x7fffffff) | __double2loint(pc)) == 0;
    const int sgn = zero ? int(0x80000000u) : (hc & int(0x80000000u));  // zero counts below
    pc = __hiloint2double(sgn | (kTinyBiasedExp << 20), 0);
    hc = hi_of(pc);
  }
  int cnt = (hc >> 31) & 1;
  for (int i = 1; i < m; ++i) {
    const double2 q = de[i];
    double pn = (q.x - x) * pc;
    pn = fma(-q.y, pm, pn);
    int hn = hi_of(pn);
    int en = bexp(hn);
    const int ec = bexp(hc);
    const int emax = max(en, ec);
    if (en == 0 || (unsigned)(emax - (1023 - 400)) > 800u) {
      if (en == 0) {
        const bool zero = ((hn & 0x7fffffff) | __double2loint(pn)) == 0;
        const int sgn = zero ? ((~hc) & int(0x80000000u)) : (hn & int(0x80000000u));
        pn = __hiloint2double(sgn | (kTinyBiasedExp << 20), 0);
        hn = hi_of(pn);
        en = bexp(hn);
      }
      const int em = max(en, ec);
      if ((unsigned)(em - (1023 - 400)) > 800u) {
        const double f = __hiloint2double((2046 - em) << 20, 0);  // 2^(1023 - em)
        pn *= f;
        pc *= f;
        hn = hi_of(pn);
      }
    }
    cnt += ((hn ^ hc) >> 31) & 1;
    pm = pc;
    pc = pn;
    hc = hn;
  }
  return cnt;
}

__global__ void __launch_bounds__(kBisectThreads)
k_bisect(const BisectTask* __restrict__ tasks, const BisectItem* __restrict__ items,
         unsigned* status) {
  extern __shared__ __align__(16) double2 de[];
  __shared__ double red[3][kBisectThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const BisectItem it = items[blockIdx.x];
  const BisectTask T = tasks[it.task];
  const int m = T.m;
  if (m == 1) {  // a 1x1 tridiagonal is its own eigenvalue
    if (it.k0 + tid == 0) T.eig[0] = T.d[0];
    return;
  }

  // Gershgorin bounds and the spectral scale, from the unscaled entries.
  double gl = 1e308, gu = -1e308, tn = 0.0;
  for (int i = tid; i < m; i += blockDim.x) {
    const double d = T.d[i];
    const double el = (i > 0) ? fabs(T.e[i - 1]) : 0.0;
    const double er = (i + 1 < m) ? fabs(T.e[i]) : 0.0;
    const double r = el + er;
    gl = fmin(gl, d - r);
    gu = fmax(gu, d + r);
    tn = fmax(tn, fabs(d) + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
    tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  }
  if (lane == 0) { red[0][warp] = gl; red[1][warp] = gu; red[2][warp] = tn; }
  __syncthreads();
  gl = red[0][0]; gu = red[1][0]; tn = red[2][0];
  for (int w = 1; w < kBisectThreads / 32; ++w) {
    gl = fmin(gl, red[0][w]);
    gu = fmax(gu, red[1][w]);
    tn = fmax(tn, red[2][w]);
  }
  const int k = it.k0 + tid;
  if (tn == 0.0) {  // zero matrix: every eigenvalue is 0
    if (k < m) T.eig[k] = 0.0;
    return;
  }
  int ex;
  frexp(tn, &ex);                   // tn * 2^-ex in [0.5, 1)
  const double sc = ldexp(1.0, -ex);
  const double isc = ldexp(1.0, ex);
  for (int i = tid; i < m; i += blockDim.x) {
    const double d = T.d[i] * sc;
    const double e = (i > 0) ? T.e[i - 1] * sc : 0.0;
    de[i] = make_double2(d, e * e);
  }
  __syncthreads();

  // Scaled Gershgorin bracket, widened by a few ulps of the scale.
  const double glo = gl * sc - 0x1p-45, ghi = gu * sc + 0x1p-45;
  bool active = k < m;
  double lo = glo, hi = ghi;
  if (active && T.parent != nullptr) {
    lo = T.parent[k] * sc - 0x1p-40;
    hi = T.parent[k + 1] * sc + 0x1p-40;
    lo = fmax(lo, glo);
    hi = fmin(hi, ghi);
  }
  // Verify interlacing brackets (count(lo) <= k < count(hi)); fall back if not.
  if (T.parent != nullptr) {
    bool fell = false;
    if (active) {
      if (sturm_count(de, m, lo) > k) { lo = glo; fell = true; }
      if (sturm_count(de, m, hi) <= k) { hi = ghi; fell = true; }
    }
    if (__any_sync(0xffffffffu, fell) && lane == 0) atomicOr(status, (unsigned)ST_BRACKET_FALLBACK);
  }
  int iter = 0;
  while (__any_sync(0xffffffffu, active)) {
    if (active) {
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(de, m, mid) > k) hi = mid; else lo = mid;
      const double tol = fmax(ldexp(fmax(fabs(lo), fabs(hi)), -50), 0x1p-53);
      active = (hi - lo > tol) && (++iter < kMaxIter);
    }
  }
  if (k < m) T.eig[k] = 0.5 * (lo + hi) * isc;
}

}  // namespace

cudaError_t launch_bisect(const BisectTask* tasks, const BisectItem* items, int nitems, int max_m,
                          unsigned* status, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)max_m * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bisect<<<nitems, kBisectThreads, smem, s>>>(tasks, items, status);
  return cudaGetLastError();
}

}  // namespace eeid
