// Signed eigenvectors from Eq. 1 applied in a second basis (the sign-recovery step).
//
// Why: Eq. 1 (Sec. 2) yields only |v_ij|^2; the paper notes that applying the identity
// in other bases recovers the direction.  Rotate coordinates r and j by 45 degrees,
// u = (e_r + e_j)/sqrt2: the unit eigenvectors of A in the new basis have u-component
// (v_ir + v_ij)/sqrt2, and Eq. 1 on the minor that removes u (the "rotated minor",
// built by K-a's copy step) gives q_ij = (v_ir + v_ij)^2 / 2 for every i at once.  So
//     v_ir v_ij = q_ij - (|v_ir|^2 + |v_ij|^2) / 2,
// and with v_ir = +sqrt(|v_ir|^2) fixing the eigenvector's sign,
//     v_ij = (q_ij - (|v_ir|^2 + |v_ij|^2) / 2) / |v_ir|.
// Each of q, |v_ir|^2, |v_ij|^2 carries the identity's absolute error delta, so v_ij
// carries about 2 delta / |v_ir|: the reference component r must be large.
//
// k_pick_refs chooses, for the requested eigenvectors, a small set of reference
// components by greedy set cover: eigenvector i accepts r when
// |v_ir|^2 >= max_j |v_ij|^2 / 16, i.e. |v_ir| >= max_j |v_ij| / 4 >= 1/(4 sqrt n).  Each
// chosen reference costs one rotated minor per component j != r; the eigenvectors that
// share a reference share those minors.
//
// k_signed assembles each eigenvector and applies the sign convention: the component
// of largest |v_ij|^2 (the first on exact ties) is made positive.
#include "internal.cuh"

namespace eeid {
namespace {

constexpr int kPickThreads = 1024;
constexpr double kRefRatio = 1.0 / 16.0;

// One CTA.  g: nrows x n (row r = |v_{i_r, j}|^2 for all j).  Outputs: refs[0 .. *nref)
// (component indices), row_ref[r] (index into refs; -1 for a row with no usable
// magnitude: all zero or NaN, i.e. a degenerate eigenvalue), and need[q*n + j] = 1 when
// some row of reference q has |v_ij|^2 != 0 (a column whose magnitudes are exactly zero
// for all of them needs no rotated minor: those components are exactly 0).  Scratch in
// shared memory: thr (nrows doubles), covered (nrows bytes), count (n ints).
__global__ void __launch_bounds__(kPickThreads)
k_pick_refs(const double* __restrict__ g, int nrows, int n, int* __restrict__ refs,
            int* __restrict__ row_ref, int* __restrict__ nref, unsigned char* __restrict__ need) {
  extern __shared__ __align__(16) double thr[];
  int* count = (int*)(thr + nrows);
  unsigned char* covered = (unsigned char*)(count + n);
  __shared__ int s_best, s_bestc;
  __shared__ int s_wbest[kPickThreads / 32], s_wbestc[kPickThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // per-row acceptance threshold (a warp per row)
  for (int r = warp; r < nrows; r += kPickThreads / 32) {
    const double* row = g + (size_t)r * n;
    double mx = 0.0;
    bool bad = false;
    for (int j = lane; j < n; j += 32) {
      const double x = row[j];
      bad |= !(x == x);
      mx = fmax(mx, x);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      const bool usable = !bad && mx > 0.0;
      thr[r] = mx * kRefRatio;
      covered[r] = usable ? 0 : 1;
      row_ref[r] = -1;
    }
  }
  __syncthreads();

  int R = 0;
  for (int it = 0; it < nrows; ++it) {   // each pick covers at least one row
    // rows of each column that would accept it as their reference
    for (int j = tid; j < n; j += kPickThreads) {
      int c = 0;
      for (int r = 0; r < nrows; ++r)
        if (!covered[r] && g[(size_t)r * n + j] >= thr[r]) ++c;
      count[j] = c;
    }
    __syncthreads();
    // the column covering most rows (the smallest index on ties)
    int best = -1, bestc = 0;
    for (int j = tid; j < n; j += kPickThreads)
      if (count[j] > bestc) { bestc = count[j]; best = j; }
    for (int o = 16; o > 0; o >>= 1) {
      const int oc = __shfl_xor_sync(0xffffffffu, bestc, o);
      const int ob = __shfl_xor_sync(0xffffffffu, best, o);
      if (oc > bestc || (oc == bestc && oc > 0 && (unsigned)ob < (unsigned)best)) {
        bestc = oc;
        best = ob;
      }
    }
    if (lane == 0) { s_wbest[warp] = best; s_wbestc[warp] = bestc; }
    __syncthreads();
    if (tid == 0) {
      int b = -1, bc = 0;
      for (int w = 0; w < kPickThreads / 32; ++w)
        if (s_wbestc[w] > bc || (s_wbestc[w] == bc && bc > 0 && (unsigned)s_wbest[w] < (unsigned)b)) {
          bc = s_wbestc[w];
          b = s_wbest[w];
        }
      s_best = b;
      s_bestc = bc;
    }
    __syncthreads();
    const int jb = s_best;
    if (s_bestc == 0) break;
    for (int r = tid; r < nrows; r += kPickThreads)
      if (!covered[r] && g[(size_t)r * n + jb] >= thr[r]) {
        covered[r] = 1;
        row_ref[r] = R;
      }
    if (tid == 0) refs[R] = jb;
    ++R;
    __syncthreads();
  }
  if (tid == 0) *nref = R;
  // columns each reference's rows need (row_ref complete after the last barrier)
  for (int j = tid; j < n; j += kPickThreads) {
    for (int q = 0; q < R; ++q) need[(size_t)q * n + j] = 0;
    for (int r = 0; r < nrows; ++r) {
      const int q = row_ref[r];
      if (q >= 0 && g[(size_t)r * n + j] != 0.0) need[(size_t)q * n + j] = 1;
    }
  }
}

// One CTA per requested eigenvector.  g: its |v_ij|^2 row (n); q: its row of rotated
// components; pos[j]: the place of q_ij in that row, or -1 where no rotated minor was
// needed (|v_ij|^2 exactly 0 for every row of this reference); out: the signed vector.
struct SignedRow {
  const double* g;
  const double* q;
  const int* pos;
  double* out;
  int ref;   // reference component, -1 if the row had no usable magnitude
};
constexpr int kSignedThreads = 256;

__global__ void __launch_bounds__(kSignedThreads)
k_signed(const SignedRow* __restrict__ rows, int n) {
  __shared__ double s_max[kSignedThreads / 32];
  __shared__ int s_arg[kSignedThreads / 32];
  const SignedRow R = rows[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (R.ref < 0) {
    for (int j = tid; j < n; j += kSignedThreads) R.out[j] = NAN;
    return;
  }
  // the sign convention's component: largest |v_ij|^2, first on ties
  double mx = -1.0;
  int arg = 0x7fffffff;
  for (int j = tid; j < n; j += kSignedThreads) {
    const double x = R.g[j];
    if (x > mx) { mx = x; arg = j; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double om = __shfl_xor_sync(0xffffffffu, mx, o);
    const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (om > mx || (om == mx && oa < arg)) { mx = om; arg = oa; }
  }
  if (lane == 0) { s_max[warp] = mx; s_arg[warp] = arg; }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kSignedThreads / 32; ++w)
      if (s_max[w] > s_max[0] || (s_max[w] == s_max[0] && s_arg[w] < s_arg[0])) {
        s_max[0] = s_max[w];
        s_arg[0] = s_arg[w];
      }
  }
  __syncthreads();
  const int jstar = s_arg[0];
  const int r = R.ref;
  const double gr = R.g[r];
  const double vr = sqrt(gr);
  // sign of the convention's component relative to the reference (v_ir > 0)
  double vstar;
  if (jstar == r) {
    vstar = vr;
  } else {
    const double qs = R.q[R.pos[jstar]];   // |v_ij*|^2 > 0, so its minor was computed
    vstar = (qs - 0.5 * (gr + R.g[jstar])) / vr;
  }
  const double flip = vstar < 0.0 ? -1.0 : 1.0;
  for (int j = tid; j < n; j += kSignedThreads) {
    double v;
    const int pj = R.pos[j];
    if (j == r) {
      v = vr;
    } else if (pj < 0) {
      v = 0.0;
    } else {
      v = (R.q[pj] - 0.5 * (gr + R.g[j])) / vr;
    }
    R.out[j] = flip * v;
  }
}

}  // namespace

size_t pick_refs_smem_bytes(int nrows, int n) {
  return sizeof(double) * (size_t)nrows + sizeof(int) * (size_t)n + (size_t)nrows + 16;
}

static std::atomic<uint64_t> g_pick_limit_set{0};

cudaError_t preload_vectors() {
  return raise_smem_limit_once((const void*)k_pick_refs, g_pick_limit_set);
}

cudaError_t launch_pick_refs(const double* g, int nrows, int n, int* refs, int* row_ref,
                             int* nref, unsigned char* need, cudaStream_t s) {
  cudaError_t e = raise_smem_limit_once((const void*)k_pick_refs, g_pick_limit_set);
  if (e != cudaSuccess) return e;
  k_pick_refs<<<1, kPickThreads, pick_refs_smem_bytes(nrows, n), s>>>(g, nrows, n, refs, row_ref,
                                                                      nref, need);
  return cudaGetLastError();
}

cudaError_t launch_signed(const void* rows, int nrows, int n, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  k_signed<<<nrows, kSignedThreads, 0, s>>>((const SignedRow*)rows, n);
  return cudaGetLastError();
}

size_t signed_row_bytes() { return sizeof(SignedRow); }

void fill_signed_row(void* dst, const double* g, const double* q, const int* pos, double* out,
                     int ref) {
  SignedRow r{g, q, pos, out, ref};
  *(SignedRow*)dst = r;
}

}  // namespace eeid
