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
//  * Two phases.  FP32 runs at ~60x the FP64 rate on this part, so the bracket is
//    first narrowed to ~2^-36 ||T|| with Sturm counts in double-float arithmetic
//    (pairs of FP32 values, ~2^-44 relative per operation).  The FP64 phase then
//    widens that bracket by 2^-40 ||T|| (more than the double-float counts' error),
//    re-verifies it with two exact-FP64 Sturm counts and finishes in FP64.  A bracket that fails the check
//    (the cheap phase misjudged, or the interlacing seed was wrong) falls back to
//    the Gershgorin bracket, so the result never depends on the FP32 phase.
//  * The two verifying counts also return det(T - xI) at the bracket ends; one
//    secant step and two counts around it cut the FP64 finish from about 13
//    halvings to none: when the counts put eigenvalue k inside the window
//    x1 +- h, h = max(2^-50 |x1|, 2^-51 ||T||), the lane returns x1, verified to h
//    (bisection from the narrowed bracket is the fallback).
#include "internal.cuh"

namespace eeid {
namespace {

constexpr int kTinyBiasedExp = 1023 - 900;  // 2^-900
constexpr int kMaxIter = 120;

__device__ __forceinline__ int hi_of(double x) { return __double2hiint(x); }
__device__ __forceinline__ int bexp(int hi) { return (hi >> 20) & 0x7ff; }

// Number of eigenvalues of the (scaled) tridiagonal below x.  With VAL the value of
// the last minor, p_m(x) = det(T - xI), is returned as *val * 2^(*vexp) (the power of
// two undoes the rescalings; a p_i that came out exactly zero is the 2^-900 stand-in).
template <bool VAL = false>
__device__ __forceinline__ int sturm_count(const double2* __restrict__ de, int m, double x,
                                           double* val = nullptr, int* vexp = nullptr) {
  int sexp = 0;
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
        if (VAL) sexp += em - 1023;
      }
    }
    cnt += ((hn ^ hc) >> 31) & 1;
    pm = pc;
    pc = pn;
    hc = hn;
  }
  if (VAL) {
    *val = pc;
    *vexp = sexp;
  }
  return cnt;
}

// ---- double-float arithmetic: a value is hi + lo with two FP32 numbers, built from
// the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2):
// two_sum and two_prod return a rounded result and its exact rounding error.
struct dflt {
  float h, l;
};
__device__ __forceinline__ dflt df_quick(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb) + (a.l + b.l);
  return df_quick(s, e);
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_quick(p, e);
}
__device__ __forceinline__ dflt df_of(double v) {   // round to the nearest double-float
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_val(dflt a) { return (double)a.h + (double)a.l; }

constexpr int kTinyF = 127 - 100;  // 2^-100 as an FP32 biased exponent

// Number of eigenvalues below x of the scaled tridiagonal, with the three-term
// recurrence evaluated in double-float (q[i] = (d_i hi, d_i lo, e_{i-1}^2 hi, lo)).
// Same conventions as the FP64 count; the pair is rescaled by powers of two to keep
// its larger exponent in [2^-40, 2^40] (FP32 range).
__device__ __forceinline__ int sturm_count_df(const float4* __restrict__ q, int m, dflt x) {
  const dflt nx = {-x.h, -x.l};
  dflt pm = {1.0f, 0.0f};
  float4 q0 = q[0];
  dflt pc = df_add({q0.x, q0.y}, nx);
  int hc = __float_as_int(pc.h);
  if (((hc >> 23) & 0xff) == 0) {
    const int sgn = ((hc & 0x7fffffff) == 0) ? int(0x80000000u) : (hc & int(0x80000000u));
    pc = {__int_as_float(sgn | (kTinyF << 23)), 0.0f};
    hc = __float_as_int(pc.h);
  }
  int cnt = (hc >> 31) & 1;
  for (int i = 1; i < m; ++i) {
    const float4 qi = q[i];
    const dflt t = df_add({qi.x, qi.y}, nx);
    const dflt a = df_mul(t, pc);
    const dflt b = df_mul({qi.z, qi.w}, pm);
    dflt pn = df_add(a, {-b.h, -b.l});
    int hn = __float_as_int(pn.h);
    int en = (hn >> 23) & 0xff;
    const int ec = (hc >> 23) & 0xff;
    if (en == 0 || (unsigned)(max(en, ec) - (127 - 40)) > 80u) {
      if (en == 0) {
        const bool zero = (hn & 0x7fffffff) == 0;
        const int sgn = zero ? ((~hc) & int(0x80000000u)) : (hn & int(0x80000000u));
        pn = {__int_as_float(sgn | (kTinyF << 23)), 0.0f};
        hn = __float_as_int(pn.h);
        en = (hn >> 23) & 0xff;
      }
      const int em = max(en, ec);
      if ((unsigned)(em - (127 - 40)) > 80u) {
        const float f = __int_as_float((254 - em) << 23);  // 2^(127 - em)
        pn.h *= f; pn.l *= f;
        pc.h *= f; pc.l *= f;
        hn = __float_as_int(pn.h);
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
  extern __shared__ __align__(16) double2 de_all[];
  __shared__ double red[3][kBisectThreads / 32];
  __shared__ double s_g[3][kBisectMaxPack];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const BisectItem it = items[blockIdx.x];
  const int npack = it.ntask;          // > 1: npack consecutive tasks of one size m
  const int m = tasks[it.task].m;
  // this lane's task (local index lt) and eigenvalue index k
  const int lt = npack > 1 ? tid / m : 0;
  const bool in_task = lt < npack;
  const BisectTask T = tasks[it.task + (in_task ? lt : 0)];
  const int k = npack > 1 ? tid - lt * m : it.k0 + tid;
  if (m == 1) {  // a 1x1 tridiagonal is its own eigenvalue
    if (in_task && k == 0) T.eig[0] = T.d[0];
    return;
  }

  // Gershgorin bounds and the spectral scale of each task, from the unscaled entries:
  // one task per block reduced by the whole block, packed tasks one per warp at a time.
  if (npack == 1) {
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
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        gl = fmin(gl, red[0][w]);
        gu = fmax(gu, red[1][w]);
        tn = fmax(tn, red[2][w]);
      }
      s_g[0][0] = gl; s_g[1][0] = gu; s_g[2][0] = tn;
    }
  } else {
    for (int q = warp; q < npack; q += (int)(blockDim.x >> 5)) {
      const BisectTask Q = tasks[it.task + q];
      double gl = 1e308, gu = -1e308, tn = 0.0;
      for (int i = lane; i < m; i += 32) {
        const double d = Q.d[i];
        const double el = (i > 0) ? fabs(Q.e[i - 1]) : 0.0;
        const double er = (i + 1 < m) ? fabs(Q.e[i]) : 0.0;
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
      if (lane == 0) { s_g[0][q] = gl; s_g[1][q] = gu; s_g[2][q] = tn; }
    }
  }
  __syncthreads();
  // every task's table scaled by an exact power of two to a Gershgorin bound in [0.5, 1);
  // the tables of packed tasks lie one after the other
  const int rows = npack * m;
  float4* dq_all = (float4*)(de_all + (rows > m ? rows : m));   // double-float copies
  for (int i = tid; i < rows; i += blockDim.x) {
    const int q = i / m, r = i - q * m;
    const BisectTask Q = npack > 1 ? tasks[it.task + q] : T;
    const double tq = s_g[2][q];
    int exq = 0;
    if (tq != 0.0) frexp(tq, &exq);
    const double scq = ldexp(1.0, -exq);
    const double d = Q.d[r] * scq;
    const double e = (r > 0) ? Q.e[r - 1] * scq : 0.0;
    const double e2 = e * e;
    de_all[i] = make_double2(d, e2);
    const dflt dd = df_of(d), ee = df_of(e2);
    dq_all[i] = make_float4(dd.h, dd.l, ee.h, ee.l);
  }
  __syncthreads();
  const double2* de = de_all + lt * m;
  const float4* dq = dq_all + lt * m;
  const double gl = s_g[0][in_task ? lt : 0], gu = s_g[1][in_task ? lt : 0];
  const double tn = s_g[2][in_task ? lt : 0];
  // a zero matrix has every eigenvalue 0 (its lanes stay in the warp, inactive)
  const bool zero = tn == 0.0;
  int ex = 0;
  if (!zero) frexp(tn, &ex);        // tn * 2^-ex in [0.5, 1)
  const double sc = ldexp(1.0, -ex);
  const double isc = ldexp(1.0, ex);

  // Scaled Gershgorin bracket, widened by a few ulps of the scale.
  const double glo = gl * sc - 0x1p-45, ghi = gu * sc + 0x1p-45;
  bool active = in_task && k < m && !zero;
  double lo = glo, hi = ghi;
  if (active && T.parent != nullptr) {
    lo = T.parent[k] * sc - 0x1p-40;
    hi = T.parent[k + 1] * sc + 0x1p-40;
    lo = fmax(lo, glo);
    hi = fmin(hi, ghi);
  }
  // Phase 1 (double-float): bisect until the bracket is below 2^-36 of the scale.  The
  // FP64 phase starts with a secant step, whose error from the curvature of det(T - xI)
  // is about width^2 / gap; at 2^-36 that stays far below the tolerance for relative
  // gaps down to 1e-5 (a CPU emulation on n = 1024 minors and the batch families put
  // every secant estimate inside its verification window), so narrowing further here
  // would only add passes.
  {
    dflt dlo = df_of(lo), dhi = df_of(hi);
    bool act = active;
    int it1 = 0;
    while (__any_sync(0xffffffffu, act)) {
      if (act) {
        dflt mid = df_add(dlo, dhi);
        mid.h *= 0.5f;
        mid.l *= 0.5f;
        if (sturm_count_df(dq, m, mid) > k) dhi = mid; else dlo = mid;
        const dflt w = df_add(dhi, {-dlo.h, -dlo.l});
        act = (w.h > 0x1p-36f) && (++it1 < 64);
      }
    }
    if (active) {
      lo = fmax(df_val(dlo) - 0x1p-40, glo);
      hi = fmin(df_val(dhi) + 0x1p-40, ghi);
    }
  }
  // Phase 2 (FP64): verify the narrowed bracket (count(lo) <= k < count(hi)) with
  // exact FP64 counts; fall back to the Gershgorin bracket if it fails.
  {
    bool fell = false;
    double vlo = 1.0, vhi = 1.0;
    int slo = 0, shi = 0, clo = 0, chi = 0;
    if (active) {
      clo = sturm_count<true>(de, m, lo, &vlo, &slo);
      chi = sturm_count<true>(de, m, hi, &vhi, &shi);
      if (clo > k) { lo = glo; fell = true; }
      if (chi <= k) { hi = ghi; fell = true; }
    }
    if (__any_sync(0xffffffffu, fell) && lane == 0) atomicOr(status, (unsigned)ST_BRACKET_FALLBACK);
    // Secant step.  With exactly one eigenvalue in (lo, hi] and the bracket a few
    // 2^-40 wide, det(T - xI) is linear across it to far below the tolerance, so the
    // secant through the two end values lands within rounding of the eigenvalue.  A
    // window of +-max(tol, 2^-51) around it (2^-51 stays clear of the counts' own
    // rounding, a few 2^-53) is verified with two counts; bisection then finishes
    // from the window.  A window that misses only narrows the bracket, and bisection
    // goes on from there, so the result never rests on the secant.
    if (active && !fell && chi - clo == 1) {
      const double rho = ldexp(vhi / vlo, max(-2000, min(2000, shi - slo)));  // p(hi)/p(lo) < 0
      const double x1 = lo + (hi - lo) / (1.0 - rho);
      const double h = fmax(fmax(ldexp(fabs(x1), -50), 0x1p-53), 0x1p-51);
      const double a = x1 - h, b = x1 + h;
      if (a > lo && b < hi) {
        if (sturm_count(de, m, a) > k) hi = a; else lo = a;
        if (hi > b) {
          if (sturm_count(de, m, b) > k) hi = b; else lo = b;
        }
        // both window counts held: eigenvalue k is in (a, b], and its midpoint is the
        // secant estimate, accurate to the FP64 values' rounding; no halving refines it
        // further in any useful way, so the lane is done (verified to +-h)
        if (lo == a && hi == b) active = false;
      }
    }
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
  if (in_task && k < m) T.eig[k] = zero ? 0.0 : 0.5 * (lo + hi) * isc;
}

}  // namespace

static std::atomic<uint64_t> g_bisect_limit_set{0};

cudaError_t preload_bisect() { return raise_smem_limit_once((const void*)k_bisect, g_bisect_limit_set); }

cudaError_t launch_bisect(const BisectTask* tasks, const BisectItem* items, int nitems, int max_m,
                          unsigned* status, cudaStream_t s, int threads) {
  if (threads < 32 || threads > kBisectThreads || threads % 32) return cudaErrorInvalidValue;
  if (nitems <= 0) return cudaSuccess;
  // room for one task of max_m rows or for packed tasks of up to kBisectThreads rows
  const size_t rows = (size_t)(max_m > kBisectThreads ? max_m : kBisectThreads);
  const size_t smem = rows * (sizeof(double2) + sizeof(float4));
  cudaError_t e = raise_smem_limit_once((const void*)k_bisect, g_bisect_limit_set);
  if (e != cudaSuccess) return e;
  k_bisect<<<nitems, threads, smem, s>>>(tasks, items, status);
  return cudaGetLastError();
}

}  // namespace eeid
