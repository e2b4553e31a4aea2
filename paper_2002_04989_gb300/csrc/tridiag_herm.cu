// K-a for a complex Hermitian A: Householder reduction of A and of its minors M_j to a
// real symmetric tridiagonal (d, e), FP64, one CTA per matrix, persistent over a
// cost-sorted task list.
//
// Why: Sec. 2 states Eq. 1 for Hermitian matrices; the identity needs the eigenvalues
// of A and of each minor, and both keep their spectrum under unitary similarity.  The
// reduction here uses Hermitian reflectors H = I - tau v v^H with real tau, so every
// step is the real algorithm with complex data:
//   x = A[k+1:, k], alpha = x_0, sigma = sum_{i>0} |x_i|^2, nrm = sqrt(|alpha|^2 + sigma),
//   phase = alpha/|alpha| (1 if alpha = 0), v_0 = 1, v_i = x_i conj(phase)/(|alpha| + nrm),
//   tau = 1 + |alpha|/nrm, so that H x = -phase nrm e_1;
//   p = tau A22 v, gamma = tau/2 Re(v^H p), w = p - gamma v, A22 <- A22 - v w^H - w v^H.
// The sub-diagonal entry -phase nrm has modulus nrm; a diagonal unitary similarity makes
// every sub-diagonal entry real and positive without changing the spectrum, so the
// tridiagonal handed to K-b is (Re of the diagonal, moduli of the sub-diagonal).
// K-b and K-c are then unchanged.
//
// Per element of the trailing lower triangle the fused pass costs 16 FP64 FMA (rank-2
// update 8, both halves of the Hermitian matrix-vector product 8) for 16 bytes read and
// written, so like the real kernel it is bound by FP64 issue.  The layout follows the
// real global-slot kernel: 32 x 32 tiles split over the warps in contiguous ranges,
// every tile keeping its own column partial (the strictly upper part, conj(a_ic) v_i)
// and row partial (a_ic v_c, c <= i) in the CTA's global slot, summed in tile order, so
// a matrix's (d, e) do not depend on the warp count.  Diagonal tiles are packed (their
// lower triangle in 17 full warp-rows, mirrored into the shared tile for the product).
#include "internal.cuh"

namespace eeid {
namespace {

constexpr int kT = 32, kTP = 33;

__host__ __device__ inline int hround_up(int x, int a) { return (x + a - 1) / a * a; }

struct HLayout {
  int VM;
  int nbmax;
  int64_t ld;   // complex elements per row of the working matrix
};

__host__ __device__ inline HLayout herm_layout(int max_m) {
  HLayout L;
  L.VM = hround_up(max_m, 32) + 32;
  L.nbmax = (max_m + 31) / 32;
  L.ld = hround_up(max_m, 2);
  return L;
}

// t += conj(a) v
__device__ __forceinline__ void mac_conj(double2& t, double2 a, double2 v) {
  t.x = fma(a.x, v.x, fma(a.y, v.y, t.x));
  t.y = fma(a.x, v.y, fma(-a.y, v.x, t.y));
}
// u += a v
__device__ __forceinline__ void mac(double2& u, double2 a, double2 v) {
  u.x = fma(a.x, v.x, fma(-a.y, v.y, u.x));
  u.y = fma(a.x, v.y, fma(a.y, v.x, u.y));
}
// a - x conj(y) - z conj(q), as one chain of four FMA per component
__device__ __forceinline__ double2 rank2(double2 a, double2 x, double2 y, double2 z, double2 q) {
  double2 r;
  r.x = fma(-x.x, y.x, fma(-x.y, y.y, fma(-z.x, q.x, fma(-z.y, q.y, a.x))));
  r.y = fma(-x.y, y.x, fma(x.x, y.y, fma(-z.y, q.x, fma(z.x, q.y, a.y))));
  return r;
}

__device__ __forceinline__ double warp_sum_h(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One tile (rows [R0, R0+32), columns [C0, C0+32)) of the fused pass.  Lane l owns column
// C0+l in the column half and row R0+l in the row half.  EDGE tiles (diagonal, or rows
// past m) predicate every element on i < m and c <= i; diagonal entries are kept real.
template <bool EDGE, bool UPD>
__device__ __forceinline__ void htile(double2* S, int64_t ld, int m, int R0, int C0, int lane,
                                      const double2* vP, const double2* wP, const double2* vC,
                                      double2* tile, double2* tslot, double2* uslot) {
  const int c = C0 + lane;
  const bool cv = !EDGE || c < m;
  const double2 z = make_double2(0.0, 0.0);
  const double2 vPc = UPD ? vP[c] : z, wPc = UPD ? wP[c] : z;
  const int nrows = EDGE ? min(kT, m - R0) : kT;
  double2 t = z;
#pragma unroll 1
  for (int h = 0; h < nrows; h += 8) {
    double2 a[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      const int i = R0 + h + rr;
      const bool ok = (!EDGE || (h + rr < nrows && cv && i >= c));
      a[rr] = ok ? S[(size_t)i * ld + c] : z;
    }
    if (UPD) {
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int i = R0 + h + rr;
        const bool ok = (!EDGE || (h + rr < nrows && cv && i >= c));
        double2 x = rank2(a[rr], vP[i], wPc, wP[i], vPc);
        if (EDGE && i == c) x.y = 0.0;
        a[rr] = ok ? x : z;
        if (ok) S[(size_t)i * ld + c] = x;
      }
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      const int i = R0 + h + rr;
      if (!EDGE || i > c) mac_conj(t, a[rr], vC[i]);
      tile[(h + rr) * kTP + lane] = a[rr];
    }
  }
  *tslot = t;
  __syncwarp();
  const int i = R0 + lane;
  double2 u = z;
#pragma unroll 8
  for (int cc = 0; cc < kT; ++cc) {
    const bool ok = !EDGE || (lane < nrows && C0 + cc <= i);
    const double2 x = ok ? tile[lane * kTP + cc] : z;
    mac(u, x, vC[C0 + cc]);
  }
  *uslot = u;
  __syncwarp();
}

// Diagonal tile: its lower triangle is 528 of 1024 entries, so the lane-per-column
// mapping of htile would issue with half the lanes masked.  The update is packed instead:
// warp-row r < 15 holds row r (lanes 0..r) and row 30-r (lanes r+1..31), then row 15 and
// row 31, 17 warp-rows in all.  Each updated entry a_ic goes to the shared tile at (i, c)
// and its conjugate at (c, i); one pass over the full Hermitian tile then gives the whole
// product row by row (row partials only; the tile's column partial is 0).
template <bool UPD>
__device__ __forceinline__ void hdiag(double2* S, int64_t ld, int m, int R0, int lane,
                                      const double2* vP, const double2* wP, const double2* vC,
                                      double2* tile, double2* tslot, double2* uslot) {
  const double2 z = make_double2(0.0, 0.0);
  const int nrows = min(kT, m - R0);
#pragma unroll
  for (int it = 0; it < 17; ++it) {
    int i, c;
    bool valid;
    if (it < 15) {
      const bool first = lane <= it;
      i = first ? it : 30 - it;
      c = first ? lane : lane - it - 1;
      valid = true;
    } else if (it == 15) {
      i = 15;
      c = lane;
      valid = lane <= 15;
    } else {
      i = 31;
      c = lane;
      valid = true;
    }
    valid = valid && i < nrows;
    double2* ptr = S + (size_t)(R0 + i) * ld + (R0 + c);
    double2 a = valid ? *ptr : z;
    if (UPD) {
      double2 x = rank2(a, vP[R0 + i], wP[R0 + c], wP[R0 + i], vP[R0 + c]);
      if (i == c) x.y = 0.0;
      a = valid ? x : z;
      if (valid) *ptr = a;
    }
    if (valid) {
      tile[i * kTP + c] = a;
      tile[c * kTP + i] = make_double2(a.x, -a.y);
    }
  }
  *tslot = z;
  __syncwarp();
  double2 u = z;
#pragma unroll 8
  for (int cc = 0; cc < kT; ++cc) {
    const bool ok = lane < nrows && cc < nrows;
    const double2 x = ok ? tile[lane * kTP + cc] : z;
    mac(u, x, vC[R0 + cc]);
  }
  *uslot = u;
  __syncwarp();
}

__device__ __forceinline__ int htile_start(int w, int T, int W) { return (int)(((int64_t)w * T) / W); }

template <int W>
__global__ void __launch_bounds__(W * 32, 1) k_tridiag_herm(TridiagLaunch P) {
  extern __shared__ __align__(16) double2 hsm[];
  constexpr int NT = W * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const HLayout Ly = herm_layout(P.max_m);
  const int64_t ld = Ly.ld;
  const int nbmax = Ly.nbmax;
  double2* vP = hsm;
  double2* wP = vP + Ly.VM;
  double2* vC = wP + Ly.VM;
  double2* const wC = wP;
  double* scal = (double*)(vC + Ly.VM);   // 8 doubles
  double2* tile = (double2*)(scal + 8) + warp * (kT * kTP);
  double2* S = (double2*)(P.work + (size_t)blockIdx.x * P.work_stride);
  double2* tpart = S + (size_t)P.max_m * ld;
  double2* upart = tpart + (size_t)nbmax * nbmax * 32;
  __shared__ int s_task;
  const double2 z = make_double2(0.0, 0.0);

  for (;;) {
    if (tid == 0) s_task = atomicAdd(P.counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= P.ntasks) break;
    const TridiagTask task = P.tasks[t];
    const int skip = task.skip;
    const int m = task.n - (skip >= 0 ? 1 : 0);
    if (m < 1 || m > P.max_m) {
      if (tid == 0) atomicOr(P.status, (unsigned)ST_BAD_TASK);
      continue;
    }
    double* __restrict__ dout = task.d;
    double* __restrict__ eout = task.e;
    for (int i = m + tid; i < Ly.VM; i += NT) {
      vP[i] = z;
      wP[i] = z;
      vC[i] = z;
    }
    // a1: the minor view of the interleaved complex A (lower triangle, real diagonal)
    const double2* A = (const double2*)task.A;
    for (int r = warp; r < m; r += W) {
      const int i = (skip >= 0 && r >= skip) ? r + 1 : r;
      for (int c = lane; c <= r; c += 32) {
        const int j = (skip >= 0 && c >= skip) ? c + 1 : c;
        double2 x = A[(size_t)i * task.lda + j];
        if (c == r) x.y = 0.0;
        S[(size_t)r * ld + c] = x;
      }
    }
    __syncthreads();

    for (int k = 0; k + 2 < m; ++k) {
      const int base = k + 1;
      const bool upd = (k > 0);
      // ---- Phase A: update k-1 applied to column k; x = the column below the diagonal
      const double2 vPk = upd ? vP[k] : z, wPk = upd ? wP[k] : z;
      for (int i = k + tid; i < m; i += NT) {
        double2 a = S[(size_t)i * ld + k];
        if (upd) a = rank2(a, vP[i], wPk, wP[i], vPk);
        if (i == k) {
          dout[k] = a.x;
        } else if (i == k + 1) {
          scal[0] = a.x;
          scal[1] = a.y;
          vC[i] = make_double2(1.0, 0.0);
        } else {
          vC[i] = a;
        }
      }
      __syncthreads();
      // ---- Phase B: sigma and the reflector (warp 0, fixed order)
      if (warp == 0) {
        double q0 = 0.0, q1 = 0.0;
        for (int i = k + 2 + lane; i < m; i += 32) {
          q0 = fma(vC[i].x, vC[i].x, q0);
          q1 = fma(vC[i].y, vC[i].y, q1);
        }
        const double sig = warp_sum_h(q0 + q1);
        if (lane == 0) {
          const double ar = scal[0], ai = scal[1];
          const double aabs = hypot(ar, ai);
          double tau = 0.0, sr = 0.0, si = 0.0, enorm = aabs;
          if (sig != 0.0) {
            const double nrm = sqrt(fma(aabs, aabs, sig));
            tau = 1.0 + aabs / nrm;
            const double pr = aabs > 0.0 ? ar / aabs : 1.0, pi = aabs > 0.0 ? ai / aabs : 0.0;
            const double den = 1.0 / (aabs + nrm);
            sr = pr * den;     // scale = conj(phase) / (|alpha| + nrm)
            si = -pi * den;
            enorm = nrm;
          }
          scal[2] = tau;
          scal[3] = sr;
          scal[4] = si;
          eout[k] = enorm;
        }
      }
      __syncthreads();
      const double tau = scal[2];
      // ---- Phase C: v = x * scale, v[k+1] = 1
      {
        const double sr = scal[3], si = scal[4];
        for (int i = k + 2 + tid; i < m; i += NT) {
          const double2 x = vC[i];
          vC[i] = make_double2(fma(x.x, sr, -x.y * si), fma(x.x, si, x.y * sr));
        }
      }
      __syncthreads();
      // ---- Phase D: fused pass over the trailing lower triangle
      const int s = m - base;
      const int nb = (s + 31) >> 5;
      {
        const int T = nb * (nb + 1) / 2;
        const int t0 = htile_start(warp, T, W), t1 = htile_start(warp + 1, T, W);
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= t0) ++I;
        int J = t0 - I * (I + 1) / 2;
        for (int tt = t0; tt < t1; ++tt) {
          const int R0 = base + kT * I, C0 = base + kT * J;
          double2* tslot = tpart + ((size_t)I * nbmax + J) * 32 + lane;
          double2* uslot = upart + ((size_t)I * nbmax + J) * 32 + lane;
          if (J < I && R0 + kT <= m) {
            if (upd) htile<false, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, uslot);
            else     htile<false, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, uslot);
          } else if (J == I) {
            if (upd) hdiag<true>(S, ld, m, R0, lane, vP, wP, vC, tile, tslot, uslot);
            else     hdiag<false>(S, ld, m, R0, lane, vP, wP, vC, tile, tslot, uslot);
          } else {
            if (upd) htile<true, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, uslot);
            else     htile<true, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, uslot);
          }
          if (++J > I) { ++I; J = 0; }
        }
      }
      __syncthreads();
      // ---- Phase E: p = tau (row partials + column partials), in tile order
      for (int i = base + tid; i < m; i += NT) {
        const int r = i - base, I = r >> 5, l = r & 31;
        const double2* up = upart + (size_t)I * nbmax * 32 + l;
        double2 p = up[0];
        for (int J = 1; J <= I; ++J) {
          p.x += up[(size_t)J * 32].x;
          p.y += up[(size_t)J * 32].y;
        }
        for (int I2 = I; I2 < nb; ++I2) {
          const double2 q = tpart[((size_t)I2 * nbmax + I) * 32 + l];
          p.x += q.x;
          p.y += q.y;
        }
        wC[i] = make_double2(p.x * tau, p.y * tau);
      }
      __syncthreads();
      // gamma = tau/2 Re(v^H p) (warp 0, fixed order)
      if (warp == 0) {
        double q0 = 0.0, q1 = 0.0;
        for (int i = base + lane; i < m; i += 32) {
          q0 = fma(vC[i].x, wC[i].x, q0);
          q1 = fma(vC[i].y, wC[i].y, q1);
        }
        const double dot = warp_sum_h(q0 + q1);
        if (lane == 0) scal[5] = 0.5 * tau * dot;
      }
      __syncthreads();
      // ---- Phase F: w = p - gamma v
      {
        const double gamma = scal[5];
        for (int i = base + tid; i < m; i += NT) {
          const double2 v = vC[i], p = wC[i];
          wC[i] = make_double2(fma(-gamma, v.x, p.x), fma(-gamma, v.y, p.y));
        }
      }
      __syncthreads();
      double2* tv = vP; vP = vC; vC = tv;
    }
    // last 2 x 2 block (or 1 x 1)
    if (tid == 0) {
      if (m == 1) {
        dout[0] = S[0].x;
      } else {
        const int a0 = m - 2, a1 = m - 1;
        double2 s00 = S[(size_t)a0 * ld + a0], s10 = S[(size_t)a1 * ld + a0];
        double2 s11 = S[(size_t)a1 * ld + a1];
        if (m >= 3) {
          s00 = rank2(s00, vP[a0], wP[a0], wP[a0], vP[a0]);
          s10 = rank2(s10, vP[a1], wP[a0], wP[a1], vP[a0]);
          s11 = rank2(s11, vP[a1], wP[a1], wP[a1], vP[a1]);
        }
        dout[a0] = s00.x;
        dout[a1] = s11.x;
        eout[a0] = hypot(s10.x, s10.y);
      }
    }
    __syncthreads();
    vP = hsm;
    vC = hsm + 2 * (size_t)Ly.VM;
  }
}

}  // namespace

size_t tridiag_herm_slot_doubles(int max_m) {
  const HLayout L = herm_layout(max_m);
  return 2 * ((size_t)max_m * L.ld + 2 * (size_t)L.nbmax * L.nbmax * 32) + 64;
}

size_t tridiag_herm_smem_bytes(int max_m, int warps) {
  const HLayout L = herm_layout(max_m);
  return 3 * (size_t)L.VM * sizeof(double2) + 8 * sizeof(double) +
         (size_t)warps * kT * kTP * sizeof(double2);
}

template <int W>
std::atomic<uint64_t>& herm_limit_set() {
  static std::atomic<uint64_t> done{0};
  return done;
}

template <int W>
static cudaError_t herm_launch_one(int grid, const TridiagLaunch& L, cudaStream_t s) {
  cudaError_t e = raise_smem_limit_once((const void*)k_tridiag_herm<W>, herm_limit_set<W>());
  if (e != cudaSuccess) return e;
  k_tridiag_herm<W><<<grid, W * 32, tridiag_herm_smem_bytes(L.max_m, W), s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_tridiag_herm(int warps, int grid, const TridiagLaunch& L, cudaStream_t s) {
  switch (warps) {
    case 4: return herm_launch_one<4>(grid, L, s);
    case 8: return herm_launch_one<8>(grid, L, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t preload_tridiag_herm() {
  cudaError_t e = raise_smem_limit_once((const void*)k_tridiag_herm<4>, herm_limit_set<4>());
  if (e == cudaSuccess) e = raise_smem_limit_once((const void*)k_tridiag_herm<8>, herm_limit_set<8>());
  return e;
}

int tridiag_herm_blocks_per_sm(int warps, int max_m) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const size_t smem = tridiag_herm_smem_bytes(max_m, warps);
  if (warps == 4) {
    e = raise_smem_limit_once((const void*)k_tridiag_herm<4>, herm_limit_set<4>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag_herm<4>, 128, smem);
  } else if (warps == 8) {
    e = raise_smem_limit_once((const void*)k_tridiag_herm<8>, herm_limit_set<8>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag_herm<8>, 256, smem);
  }
  return e == cudaSuccess ? nb : 0;
}

}  // namespace eeid
