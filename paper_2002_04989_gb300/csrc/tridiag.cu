// K-a: Householder reduction of A and of its minors M_j to symmetric tridiagonal
// form (d, e), FP64, one CTA per matrix, persistent over a cost-sorted task list.
//
// Why: Eq. 1 (Sec. 2) needs the eigenvalues of A and of every requested minor;
// the paper obtains them from LAPACK (Sec. 2-3), whose symmetric solvers start by
// this same orthogonal reduction.  The reduction preserves the spectrum exactly in
// exact arithmetic and costs 4/3 m^3 flops per m x m matrix.
//
// Per column k (trailing size s = m-k-1): the reflector H = I - tau v v^T that
// zeroes A[k+2:, k] is formed from the column; then p = tau A22 v,
// w = p - (tau/2)(p^T v) v, and A22 <- A22 - v w^T - w v^T.  The update of step k-1
// and the symmetric matrix-vector product of step k are fused into ONE pass over
// the lower triangle of the trailing block: every element is loaded once, gets the
// rank-2 update (2 FMA), and feeds both halves of the symmetric product (2 FMA),
// then is stored once.  On GB300 the FP64 FMA rate (about 2 lane-FMA/clk/SM) and
// not HBM bandwidth bounds this pass (16 bytes per 4 FMA is ~2.3 TB/s at the FP64
// peak), so the design minimises FP64 instructions: no FP64 atomics, no shuffle
// reductions inside tiles, and each 32x32 tile of the product is reduced along rows
// from a conflict-free shared-memory copy and along columns in registers.
//
// Determinism: every partial sum has one owner and a fixed summation order, so a
// matrix's (d, e) do not depend on which CTA, batch or launch processed it.  In the
// global-slot variant every tile keeps its own row and column partials, which are
// summed in tile order, so the result does not depend on the warp count either: the
// 2-16-warp instantiations give bitwise the same (d, e).
//
// Two storage variants share the code:
//   SMEM = true   the whole working matrix lives in shared memory (m <= 160);
//   SMEM = false  it lives in a per-CTA slot of global memory (L2-resident for
//                 small m), tiles are staged through a per-warp shared buffer.
#include "internal.cuh"
#include "tile_split.h"

#include <cooperative_groups.h>
#include <cstdio>

namespace cg = cooperative_groups;

namespace eeid {
namespace {

constexpr int kTile = 32;
constexpr int kTilePad = 33;

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum_{i in [i0, m)} x_i y_i by one warp, in an order fixed by (i0, m) alone: lane l
// takes i = i0 + l, i0 + l + 32, ... in four interleaved chains, then a shuffle tree.
// Only warp 0 calls it, so the reductions of a step do not depend on the CTA's warp
// count (and cost the FP64 issue of (m - i0)/32 + 8 warp instructions).
__device__ __forceinline__ double warp_dot(const double* x, const double* y, int i0, int m,
                                           int lane) {
  double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
  int i = i0 + lane;
  for (; i + 96 < m; i += 128) {
    q0 = fma(x[i], y[i], q0);
    q1 = fma(x[i + 32], y[i + 32], q1);
    q2 = fma(x[i + 64], y[i + 64], q2);
    q3 = fma(x[i + 96], y[i + 96], q3);
  }
  for (; i < m; i += 32) q0 = fma(x[i], y[i], q0);
  return warp_sum((q0 + q1) + (q2 + q3));
}

// Row half of a ragged off-diagonal tile with nrows <= 32/P rows inside the matrix (global
// variants; the tile is in the warp's shared copy, every column valid): lane l takes row
// l mod (32/P) and the P-th part (l / (32/P)) of the columns, one chain each, and the
// parts are added by shuffles in a fixed order; lane r < 32/P ends with row r's partial
// (the other lanes with 0).
template <int P>
__device__ __forceinline__ void row_half_split(const double* tile, const double* vC, int C0,
                                               int lane, int nrows, double (&u)[4]) {
  constexpr int TP = 33, R = 32 / P, CW = 32 / P;
  const int r = lane & (R - 1), part = lane / R;
  const double* rowp = tile + r * TP + part * CW;
  const double* vp = vC + C0 + part * CW;
  double acc = 0.0;
#pragma unroll
  for (int cc = 0; cc < CW; ++cc) {
    const double x = r < nrows ? rowp[cc] : 0.0;
    acc = fma(x, vp[cc], acc);
  }
#pragma unroll
  for (int o = 16; o >= R; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  u[0] += lane < R ? acc : 0.0;
}

// One 32x32 tile of the fused pass: rows [R0, R0+32), columns [C0, C0+32) of the
// working matrix.  Lane l owns column C0+l in the column half and row R0+l in the
// row half.  EDGE tiles (on the diagonal, or with rows beyond m) use predicated
// loads and selects instead of branches, so every tile is fully unrolled;
// positions outside the lower triangle contribute exact zeros.  UPD applies the
// previous step's rank-2 update (absent at the first step).
template <bool SMEM, bool EDGE, bool UPD>
__device__ __forceinline__ void tile_step(double* S, int64_t ld, int m, int R0, int C0, int lane,
                                          const double* vP, const double* wP, const double* vC,
                                          double* tile, double* tslot, double (&u)[4]) {
  // No __restrict__ here: S is written by this warp and read by other warps of the
  // CTA in later steps, so its loads must stay on the coherent path.
  constexpr int T = 32, TP = 33;
  const int c = C0 + lane;
  const bool cv = !EDGE || c < m;
  const double vPc = UPD ? vP[c] : 0.0, wPc = UPD ? wP[c] : 0.0;
  // rows of this tile inside the matrix: a warp-uniform bound, so a ragged tile
  // issues no FP64 instructions for the rows past m (full 16-row slabs unrolled,
  // the remaining rows one at a time)
  const int nrows = EDGE ? min(T, m - R0) : T;
  double t0 = 0.0, t1 = 0.0;
  int h = 0;
#pragma unroll 1
  for (; h + 16 <= nrows; h += 16) {
    double a[16];
    const double* src = S + (size_t)(R0 + h) * ld + c;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int i = R0 + h + rr;
      const bool ok = !EDGE || (cv && i >= c);
      a[rr] = ok ? src[(size_t)rr * ld] : 0.0;
    }
    if (UPD) {
      double* dst = S + (size_t)(R0 + h) * ld + c;
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const int i = R0 + h + rr;
        const double x = fma(-vP[i], wPc, fma(-wP[i], vPc, a[rr]));
        const bool ok = !EDGE || (cv && i >= c);
        a[rr] = ok ? x : 0.0;
        if (ok) dst[(size_t)rr * ld] = a[rr];
      }
    }
    // t_c = sum_{i > c} a_ic v_i (shared-memory variant: two chains; global variant:
    // one, for the reason given at the row half below)
#pragma unroll
    for (int rr = 0; rr < 16; rr += 2) {
      const int i = R0 + h + rr;
      const double x0 = (!EDGE || i > c) ? a[rr] : 0.0;
      const double x1 = (!EDGE || i + 1 > c) ? a[rr + 1] : 0.0;
      t0 = fma(x0, vC[i], t0);
      if (SMEM) t1 = fma(x1, vC[i + 1], t1);
      else      t0 = fma(x1, vC[i + 1], t0);
    }
    if (!SMEM) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) tile[(h + rr) * TP + lane] = a[rr];
    }
  }
  if (EDGE) {
    for (int rr = h; rr < nrows; ++rr) {
      const int i = R0 + rr;
      const bool ok = cv && i >= c;
      double a = ok ? S[(size_t)i * ld + c] : 0.0;
      if (UPD) {
        const double x = fma(-vP[i], wPc, fma(-wP[i], vPc, a));
        a = ok ? x : 0.0;
        if (ok) S[(size_t)i * ld + c] = a;
      }
      t0 = fma((i > c) ? a : 0.0, vC[i], t0);
      if (!SMEM) tile[rr * TP + lane] = a;
    }
  }
  *tslot = SMEM ? t0 + t1 : t0;
  __syncwarp();
  // row half: u_i += sum_{c <= i} a_ic v_c.  Shared-memory variant: four chains carried
  // across the block-row.  Global variant: one chain per tile (u[0], stored per tile);
  // with 16 warps on the SM a warp gets an FP64 issue slot only every few hundred
  // cycles, so the chain's latency is hidden and no per-tile combine is needed.
  constexpr int NCH = SMEM ? 4 : 1;
  if constexpr (!SMEM && EDGE) {
    // A ragged tile of the global variants (J < I, rows past m): with at most 16 (8)
    // rows left, 2 (4) lanes share each row and take a half (quarter) of the columns
    // each, so no FP64 instruction runs with most lanes masked; shuffles add the parts.
    if (nrows <= 8) {
      row_half_split<4>(tile, vC, C0, lane, nrows, u);
      __syncwarp();
      return;
    }
    if (nrows <= 16) {
      row_half_split<2>(tile, vC, C0, lane, nrows, u);
      __syncwarp();
      return;
    }
  }
  const int i = R0 + lane;
  const int ir = EDGE ? min(i, m - 1) : i;   // clamped row address for the shared copy
  const double* rowp = SMEM ? (S + (size_t)ir * ld + C0) : (tile + lane * TP);
#pragma unroll
  for (int cc = 0; cc < T; ++cc) {
    const bool ok = !EDGE || (i < m && C0 + cc <= i);
    const double x = ok ? rowp[cc] : 0.0;
    u[cc & (NCH - 1)] = fma(x, vC[C0 + cc], u[cc & (NCH - 1)]);
  }
  __syncwarp();
}

// Diagonal tile (global-slot variant): its lower triangle holds 528 of 1024 slots, so
// the lane-per-column mapping of tile_step would issue every FP64 instruction with half
// the lanes masked.  Here the update is packed: warp-row r < 15 holds row r (lanes
// 0..r) and row 30-r (lanes r+1..31), then row 15 and row 31, 17 warp-rows in all.  The
// updated values are mirrored into the shared tile, and one unmasked pass over the
// full symmetric tile gives both halves of the product (row partials only; the tile's
// column partial is 0).  FP64 issue: 2 x 17 + 32 = 66 instructions instead of 128.
template <bool UPD>
__device__ __forceinline__ void diag_tile(double* S, int64_t ld, int m, int R0, int lane,
                                          const double* vP, const double* wP, const double* vC,
                                          double* tile, double* tslot, double (&u)[4]) {
  constexpr int TP = 33;
  const int nrows = min(32, m - R0);   // rows (= columns) of the tile inside the matrix
#pragma unroll
  for (int it = 0; it < 17; ++it) {
    // a ragged tile skips the warp-rows whose rows all lie past m (warp-uniform): the
    // first row of warp-row it is it (it < 16) or 31
    if ((it < 16 ? it : 31) >= nrows) continue;
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
    double* ptr = S + (size_t)(R0 + i) * ld + (R0 + c);
    double a = valid ? *ptr : 0.0;
    if (UPD) {
      const double x = fma(-vP[R0 + i], wP[R0 + c], fma(-wP[R0 + i], vP[R0 + c], a));
      a = valid ? x : 0.0;
      if (valid) *ptr = a;
    }
    if (valid) {
      tile[i * TP + c] = a;
      tile[c * TP + i] = a;
    }
  }
  *tslot = 0.0;
  __syncwarp();
  const int i = lane;
#pragma unroll
  for (int cc = 0; cc < 32; ++cc) {
    if (cc >= nrows) break;   // columns past m add nothing (warp-uniform)
    const bool ok = i < nrows;
    const double x = ok ? tile[i * TP + cc] : 0.0;
    u[0] = fma(x, vC[R0 + cc], u[0]);   // one chain (global variant, see tile_step)
  }
  __syncwarp();
}


__device__ __forceinline__ int snake_owner(int I, int W) {
  const int q = I / W, r = I % W;
  return (q & 1) ? (W - 1 - r) : r;
}

struct Layout {
  int VM;         // padded vector length
  int nbmax;      // max tile blocks along the trailing block
  int64_t ld;     // working-matrix leading dimension
};

__host__ __device__ inline Layout make_layout(bool smem, int max_m) {
  Layout L;
  L.VM = round_up(max_m, 32) + 32;
  L.nbmax = (max_m + 31) / 32;
  L.ld = smem ? (int64_t)(max_m | 1) : (int64_t)round_up(max_m, 4);
  return L;
}

// Barrier of the CTA, or of the whole cluster with its global-memory writes (the
// working slot's tiles and partial sums) made visible to the other CTAs first.
template <bool CL>
__device__ __forceinline__ void block_or_cluster_sync() {
  if constexpr (CL) {
    __threadfence();
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
}

// Barrier of a group of G CTAs that reduce one matrix together (the group variant), in
// global memory: each arrival adds 1 to the group's counter, and the k-th barrier is
// passed once the counter reaches k*G (the counter only grows within a launch, so there is
// no reset to race with).  Writes before the barrier are made visible by the fences on
// both sides (release before the arrival, acquire after the wait; the CTA barriers order
// the other threads' accesses around thread 0's).  The wait is bounded: after
// kGroupWaitNs of the global timer (or kGroupSpinLimit polls, whichever comes first) the
// CTA raises the group's abort flag and ST_TIMEOUT; a CTA that sees the flag stops
// waiting too.  Returns false when the group gave up (the caller then returns without
// writing its outputs).
constexpr unsigned long long kGroupWaitNs = 1000000000ull;   // 1 s
constexpr unsigned kGroupSpinLimit = 1u << 24;               // >= 1 s at >= 64 ns a poll
struct GroupSync {
  unsigned* cnt;
  unsigned* abort_flag;
  unsigned target;
  unsigned G;
};
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __noinline__ bool group_sync(GroupSync& gs, unsigned* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    gs.target += gs.G;
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // release
    atomicAdd(gs.cnt, 1u);
    const volatile unsigned* c = gs.cnt;
    const volatile unsigned* ab = gs.abort_flag;
    const unsigned long long t0 = global_ns();
    unsigned polls = 0;
    while (*c < gs.target) {
      if (*ab) { ok = 0; break; }
      if (++polls > kGroupSpinLimit || global_ns() - t0 > kGroupWaitNs) {
        atomicExch(gs.abort_flag, 1u);
        atomicOr(status, (unsigned)ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");   // acquire
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Loads in flight per thread while the split variants stage Phase E's partials.
constexpr int kEStage = 8;

// Minimum resident CTAs per SM the register allocation must allow.
// HI: the high-occupancy build of the global-slot variant (at most 80 registers a thread:
// three 8-warp or six 4-warp CTAs per SM, a little register spilling), for small matrices
// whose per-step serial phases leave the FP64 pipe idle unless more CTAs share the SM.
template <bool SMEM, int W, bool HI = false>
struct MinBlocks {
  static constexpr int value = HI ? ((W >= 8) ? 3 : 6)
                                  : (W >= 12) ? 1 : (W >= 8) ? 2 : (SMEM && W <= 2) ? 8
                                  : (!SMEM && W == 1) ? 16 : (!SMEM && W == 2) ? 8 : 4;
};

// CL = true: the cluster variant (global-slot path only).  One thread-block cluster of C
// CTAs reduces one matrix: the tiles of each step's fused pass are split over the C*W
// warps of the cluster, every tile keeps its partial sums in the cluster's global slot
// as in the one-CTA variant, and each CTA sums its share of the elements in Phase E in
// the same tile order and writes them into every CTA's shared copy of w (distributed
// shared memory).  The serial phases (A-C, gamma, F) run redundantly in every CTA on
// identical data.  So the results are bitwise those of the one-CTA global variant.
// GR = true: the group variant (global-slot path only).  P.group CTAs, resident together
// (cooperative launch), reduce one matrix exactly as a cluster does, but exchange w through
// a vector in global memory and meet at global-memory barriers (group_sync), so a group
// can span any number of SMs.  Each group takes one task (blockIdx.x / P.group).
template <bool SMEM, int W, bool CL = false, bool HI = false, bool GR = false>
__global__ void __launch_bounds__(W * 32, (MinBlocks<SMEM, W, HI>::value)) k_tridiag(TridiagLaunch P) {
  extern __shared__ __align__(16) double sm[];
  constexpr int NT = W * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // cluster geometry (1 CTA and rank 0 without clusters)
  int crank = 0, csize = 1;
  if constexpr (CL) {
    cg::cluster_group cluster = cg::this_cluster();
    crank = (int)cluster.block_rank();
    csize = (int)cluster.num_blocks();
  }
  GroupSync gs{nullptr, nullptr, 0u, 1u};
  double* gw = nullptr;
  if constexpr (GR) {
    csize = P.group;
    crank = (int)blockIdx.x % csize;
    const int gid = (int)blockIdx.x / csize;
    gs.cnt = P.gsync + (size_t)gid * kGroupSyncWords;
    gs.abort_flag = gs.cnt + 1;
    gs.G = (unsigned)csize;
    gw = P.gw + (size_t)gid * make_layout(false, P.max_m).VM;
  }
  int rounds_done = 0;
  const int gwarp = crank * W + warp, GW = csize * W;   // warp index within the cluster
  const Layout Ly = make_layout(SMEM, P.max_m);
  const int64_t ld = Ly.ld;
  const int nbmax = Ly.nbmax;

  // Three vectors: v of the previous step (vP), v of this step (vC), and w.  The
  // fused pass reads the previous w; once it is done that w is dead, so this step's
  // w (first p) is written into the same buffer (wC aliases wP).
  double* vP = sm;
  double* wP = vP + Ly.VM;
  double* vC = wP + Ly.VM;
  double* const wC = wP;
  double* scal = vC + Ly.VM;      // 8 scalars
  double* S;
  double* tpart;
  double* upart;
  double* tile = nullptr;
  if (SMEM) {
    S = scal + 8;
    tpart = S + (size_t)P.max_m * ld;
    upart = tpart + (size_t)nbmax * nbmax * 32;
  } else {
    double* slot = P.work + (size_t)(blockIdx.x / csize) * P.work_stride;
    S = slot;
    tpart = S + (size_t)P.max_m * ld;
    upart = tpart + (size_t)nbmax * nbmax * 32;
    tile = scal + 8 + warp * (kTile * kTilePad);
  }
  __shared__ int s_task;

  for (;;) {
    if constexpr (GR) {
      // one task per group, no counter
      s_task = rounds_done++ == 0 ? (int)blockIdx.x / csize : P.ntasks;
    } else if constexpr (CL) {
      // rank 0 takes the cluster's next task and hands it to every CTA
      cg::cluster_group cluster = cg::this_cluster();
      if (crank == 0 && tid == 0) {
        const int t0 = atomicAdd(P.counter, 1);
        for (int r = 0; r < csize; ++r) *cluster.map_shared_rank(&s_task, r) = t0;
      }
      cluster.sync();
    } else {
      if (tid == 0) s_task = atomicAdd(P.counter, 1);
      __syncthreads();
    }
    const int t = s_task;
    if constexpr (CL) cg::this_cluster().sync();
    else __syncthreads();
    if (t >= P.ntasks) break;
    (void)rounds_done;
    const TridiagTask task = P.tasks[t];
    const int skip = task.skip;
    const int m = task.n - (skip >= 0 ? 1 : 0);
    if (m < 1 || m > P.max_m) {
      if (tid == 0) atomicOr(P.status, (unsigned)ST_BAD_TASK);
      continue;
    }
    double* __restrict__ dout = task.d;
    double* __restrict__ eout = task.e;

    // Edge tiles multiply zeros by vector entries past m; those entries must be
    // finite, so the tails [m, VM) of the three vectors are cleared per task (shared
    // memory keeps whatever an earlier task or launch left there).
    for (int i = m + tid; i < Ly.VM; i += NT) {
      vP[i] = 0.0;
      wP[i] = 0.0;
      vC[i] = 0.0;
    }

    // a1: the minor view -- copy the lower triangle of A without row/col `skip`.
    if (task.rot < 0) {
      for (int r = gwarp; r < m; r += GW) {
        const int i = (skip >= 0 && r >= skip) ? r + 1 : r;
        const double* Arow = task.A + (size_t)i * task.lda;
        for (int c = lane; c <= r; c += 32) {
          const int j = (skip >= 0 && c >= skip) ? c + 1 : c;
          S[(size_t)r * ld + c] = Arow[j];
        }
      }
    } else {
      // the rotated minor (see TridiagTask): w = (e_rot - e_skip)/sqrt2 kept at the
      // position of rot, every other row and column as in the plain minor
      const int rot = task.rot;
      const int rp = rot > skip ? rot - 1 : rot;
      const double* A = task.A;
      const int64_t lda = task.lda;
      auto a_of = [A, lda](int i, int j) {
        return i >= j ? A[(size_t)i * lda + j] : A[(size_t)j * lda + i];
      };
      for (int r = gwarp; r < m; r += GW) {
        const int i = r >= skip ? r + 1 : r;
        for (int c = lane; c <= r; c += 32) {
          const int j = c >= skip ? c + 1 : c;
          double x;
          if (r == rp && c == rp)
            x = 0.5 * (a_of(rot, rot) + a_of(skip, skip)) - a_of(rot, skip);
          else if (r == rp)
            x = (a_of(rot, j) - a_of(skip, j)) * 0.70710678118654752440;
          else if (c == rp)
            x = (a_of(i, rot) - a_of(i, skip)) * 0.70710678118654752440;
          else
            x = A[(size_t)i * lda + j];
          S[(size_t)r * ld + c] = x;
        }
      }
    }
    if constexpr (GR) {
      if (!group_sync(gs, P.status)) return;
    } else {
      block_or_cluster_sync<CL>();
    }

    for (int k = 0; k + 2 < m; ++k) {
      const int base = k + 1;
      const bool upd = (k > 0);
      // ---- Phase A: apply update k-1 to column k; x = column below the diagonal.
      const double vPk = upd ? vP[k] : 0.0, wPk = upd ? wP[k] : 0.0;
      // split variants (short steps): the column's loads are issued four at a time, so a
      // long column costs a few memory latencies, not one per element
      constexpr int QA = (CL || GR) ? 4 : 1;
      for (int i0 = k + tid; i0 < m; i0 += QA * NT) {
        double col[QA];
#pragma unroll
        for (int q = 0; q < QA; ++q) {
          const int i = i0 + q * NT;
          col[q] = i < m ? S[(size_t)i * ld + k] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < QA; ++q) {
          const int i = i0 + q * NT;
          if (i >= m) break;
          double a = col[q];
          if (upd) a = fma(-vP[i], wPk, fma(-wP[i], vPk, a));
          if (i == k) {
            if (crank == 0) dout[k] = a;
          } else if (i == k + 1) {
            scal[0] = a;       // alpha
            vC[i] = 1.0;
          } else {
            vC[i] = a;
          }
        }
      }
      __syncthreads();
      // ---- Phase B: sigma = |x|^2 and the reflector scalars (warp 0), broadcast
      // through shared memory.
      if (warp == 0) {
        const double sig = warp_dot(vC, vC, k + 2, m, lane);
        const double alpha = scal[0];
        double tau = 0.0, scale = 0.0, beta = alpha;
        if (sig != 0.0) {
          const double nrm = sqrt(fma(alpha, alpha, sig));
          beta = (alpha >= 0.0) ? -nrm : nrm;
          tau = (beta - alpha) / beta;
          scale = 1.0 / (alpha - beta);
        }
        if (lane == 0) {
          scal[1] = tau;
          scal[2] = scale;
          if (crank == 0) eout[k] = beta;
        }
      }
      __syncthreads();
      const double tau = scal[1];
      // ---- Phase C: v = x / (alpha - beta), v[k+1] = 1 (already set).
      {
        const double scale = scal[2];
        for (int i = k + 2 + tid; i < m; i += NT) vC[i] *= scale;
      }
      __syncthreads();
      // ---- Phase D: fused pass over the trailing lower triangle [base, m)^2.
      const int s = m - base;
      const int nb = (s + 31) >> 5;
      if (SMEM) {
        for (int I = 0; I < nb; ++I) {
          if (snake_owner(I, W) != warp) continue;
          const int R0 = base + kTile * I;
          double u[4] = {0.0, 0.0, 0.0, 0.0};
          const bool ragged = R0 + kTile > m;
          for (int J = 0; J <= I; ++J) {
            const int C0 = base + kTile * J;
            double* tslot = tpart + ((size_t)I * nbmax + J) * 32 + lane;
            if (J < I && !ragged) {
              if (upd) tile_step<SMEM, false, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
              else     tile_step<SMEM, false, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
            } else {
              if (upd) tile_step<SMEM, true, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
              else     tile_step<SMEM, true, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
            }
          }
          upart[I * 32 + lane] = (u[0] + u[1]) + (u[2] + u[3]);
        }
      } else {
        // contiguous, balanced range of tiles per warp; each tile leaves its column
        // partial in tpart and its row partial in upart (both indexed by tile)
        const int t0 = tile_start(gwarp, nb, GW), t1 = tile_start(gwarp + 1, nb, GW);
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= t0) ++I;
        int J = t0 - I * (I + 1) / 2;
        for (int t = t0; t < t1; ++t) {
          const int R0 = base + kTile * I, C0 = base + kTile * J;
          double* tslot = tpart + ((size_t)I * nbmax + J) * 32 + lane;
          double u[4] = {0.0, 0.0, 0.0, 0.0};
          if (J < I && R0 + kTile <= m) {
            if (upd) tile_step<SMEM, false, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
            else     tile_step<SMEM, false, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
          } else if (J == I) {
            if (upd) diag_tile<true>(S, ld, m, R0, lane, vP, wP, vC, tile, tslot, u);
            else     diag_tile<false>(S, ld, m, R0, lane, vP, wP, vC, tile, tslot, u);
          } else {
            if (upd) tile_step<SMEM, true, true>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
            else     tile_step<SMEM, true, false>(S, ld, m, R0, C0, lane, vP, wP, vC, tile, tslot, u);
          }
          upart[((size_t)I * nbmax + J) * 32 + lane] = u[0];
          if (++J > I) { ++I; J = 0; }
        }
      }
      if constexpr (GR) {
        if (!group_sync(gs, P.status)) return;
      } else {
        block_or_cluster_sync<CL>();
      }
      // ---- Phase E: p = tau * (row partials + column partials); gamma = tau/2 p.v.
      // Element i (block-row I, lane l) sums the row partials of the tiles of block-row I,
      // then the column partials of block-column I, each in tile order: the same order in
      // every variant.  The result goes to w (cluster: to the w of every CTA of the
      // cluster; group: to the group's vector in global memory).
      auto put_p = [&](int i, double p) {
        if constexpr (CL) {
          cg::cluster_group cluster = cg::this_cluster();
          for (int r2 = 0; r2 < csize; ++r2) cluster.map_shared_rank(wC, r2)[i] = p * tau;
        } else if constexpr (GR) {
          gw[i] = p * tau;
        } else {
          wC[i] = p * tau;
        }
      };
      // Split variants whose CTAs hold few block-rows each (short steps): all threads first
      // stage the nb + 1 partials of each element of the CTA's block-rows I = crank,
      // crank + csize, ... in shared memory (the tile scratch, idle now), kEStage loads in
      // flight a thread, and one warp per block-row then adds them from there.  With more
      // block-rows than the scratch holds at once, the plain loop below is faster (the
      // staged sums would run on few warps in several rounds).
      const int e_per = (nb + 1) * 32;
      const int e_rb = (W * kTile * kTilePad) / e_per;
      const int e_rows = (nb + csize - 1) / csize;
      if ((CL || GR) && !SMEM && e_rb >= 1 && e_rows <= e_rb && e_rows <= W) {
        double* stg = scal + 8;
        const int RB = e_rb < W ? e_rb : W;
        for (int I0 = crank; I0 < nb; I0 += RB * csize) {
          const int left = (nb - 1 - I0) / csize + 1;   // block-rows I0, I0 + csize, ... < nb
          const int nrow = left < RB ? left : RB;
          const int total = nrow * e_per;
          for (int x0 = tid; x0 < total; x0 += kEStage * NT) {
            double v[kEStage];
#pragma unroll
            for (int u = 0; u < kEStage; ++u) {
              const int x = x0 + u * NT;
              const int bq = x / e_per, r = x - bq * e_per, q = r >> 5, l = r & 31;
              const int I = I0 + bq * csize;
              v[u] = x >= total ? 0.0
                     : q <= I   ? upart[((size_t)I * nbmax + q) * 32 + l]
                                : tpart[((size_t)(q - 1) * nbmax + I) * 32 + l];
            }
#pragma unroll
            for (int u = 0; u < kEStage; ++u)
              if (x0 + u * NT < total) stg[x0 + u * NT] = v[u];
          }
          __syncthreads();
          if (warp < nrow) {
            const int i = base + 32 * (I0 + warp * csize) + lane;
            const double* sp = stg + warp * e_per + lane;
            double p = sp[0];
            for (int q = 1; q <= nb; ++q) p += sp[q * 32];
            if (i < m) put_p(i, p);
          }
          __syncthreads();
        }
      } else {
        for (int i = base + crank * NT + tid; i < m; i += GW * 32) {
          const int r = i - base, I = r >> 5, l = r & 31;
          double p;
          if (SMEM) {
            p = upart[I * 32 + l];
          } else {
            const double* up = upart + (size_t)I * nbmax * 32 + l;
            p = up[0];
            for (int J = 1; J <= I; ++J) p += up[(size_t)J * 32];
          }
          for (int I2 = I; I2 < nb; ++I2) p += tpart[((size_t)I2 * nbmax + I) * 32 + l];
          put_p(i, p);
        }
      }
      if constexpr (CL) {
        cg::this_cluster().sync();
      } else if constexpr (GR) {
        // every CTA takes the whole p tau from the group's vector (read at L2: other SMs
        // wrote it)
        if (!group_sync(gs, P.status)) return;
        for (int i = base + tid; i < m; i += NT) wC[i] = __ldcg(gw + i);
        __syncthreads();
      } else {
        __syncthreads();
      }
      if (warp == 0) {
        const double dot = warp_dot(wC, vC, base, m, lane);
        if (lane == 0) scal[3] = 0.5 * tau * dot;
      }
      __syncthreads();
      // ---- Phase F: w = p - gamma v.
      {
        const double gamma = scal[3];
        for (int i = base + tid; i < m; i += NT) wC[i] = fma(-gamma, vC[i], wC[i]);
      }
      __syncthreads();
      double* tv = vP; vP = vC; vC = tv;
    }
    // Last 2x2 block (or 1x1): apply the final update and read off d, e.
    if (tid == 0 && crank == 0) {
      if (m == 1) {
        dout[0] = S[0];
      } else {
        const int a0 = m - 2, a1 = m - 1;
        double s00 = S[(size_t)a0 * ld + a0], s10 = S[(size_t)a1 * ld + a0];
        double s11 = S[(size_t)a1 * ld + a1];
        if (m >= 3) {
          s00 = fma(-2.0 * vP[a0], wP[a0], s00);
          s10 = fma(-vP[a1], wP[a0], fma(-wP[a1], vP[a0], s10));
          s11 = fma(-2.0 * vP[a1], wP[a1], s11);
        }
        dout[a0] = s00;
        dout[a1] = s11;
        eout[a0] = s10;
      }
    }
    __syncthreads();
    // restore the canonical vector order for the next task (pointer swaps above)
    vP = sm; vC = sm + 2 * (size_t)Ly.VM;
  }
}

}  // namespace

size_t tridiag_global_slot_doubles(int max_m) {
  const Layout L = make_layout(false, max_m);
  return (size_t)max_m * L.ld + 2 * (size_t)L.nbmax * L.nbmax * 32 + 32;
}

size_t tridiag_smem_bytes(bool smem_path, int max_m, int warps) {
  const Layout L = make_layout(smem_path, max_m);
  size_t d = 3 * (size_t)L.VM + 8;
  if (smem_path)
    d += (size_t)max_m * L.ld + (size_t)L.nbmax * L.nbmax * 32 + (size_t)L.nbmax * 32;
  else
    d += (size_t)warps * kTile * kTilePad;
  return d * sizeof(double);
}

// One "limit raised" flag set per instantiation (see raise_smem_limit_once).
template <bool SMEM, int W>
std::atomic<uint64_t>& smem_limit_set() {
  static std::atomic<uint64_t> done{0};
  return done;
}

template <bool SMEM, int W, bool HI = false>
static cudaError_t launch_one(int grid, const TridiagLaunch& L, cudaStream_t s) {
  const size_t smem = tridiag_smem_bytes(SMEM, L.max_m, W);
  cudaError_t e = raise_smem_limit_once((const void*)k_tridiag<SMEM, W, false, HI>,
                                        smem_limit_set<SMEM, W + (HI ? 200 : 0)>());
  if (e != cudaSuccess) return e;
  k_tridiag<SMEM, W, false, HI><<<grid, W * 32, smem, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_tridiag(bool smem_path, int warps, int grid, const TridiagLaunch& L,
                           cudaStream_t s, bool hi) {
  if (hi && !smem_path) {
    switch (warps) {
      case 4: return launch_one<false, 4, true>(grid, L, s);
      case 8: return launch_one<false, 8, true>(grid, L, s);
    }
    return cudaErrorInvalidValue;
  }
  if (smem_path) {
    switch (warps) {
      case 1: return launch_one<true, 1>(grid, L, s);
      case 2: return launch_one<true, 2>(grid, L, s);
      case 4: return launch_one<true, 4>(grid, L, s);
      case 8: return launch_one<true, 8>(grid, L, s);
    }
  } else {
    switch (warps) {
      case 1: return launch_one<false, 1>(grid, L, s);
      case 2: return launch_one<false, 2>(grid, L, s);
      case 4: return launch_one<false, 4>(grid, L, s);
      case 8: return launch_one<false, 8>(grid, L, s);
      case 12: return launch_one<false, 12>(grid, L, s);
      case 16: return launch_one<false, 16>(grid, L, s);
    }
  }
  return cudaErrorInvalidValue;
}

// ---- cluster variant: one cluster of C CTAs per matrix (global-slot path)

template <int W>
std::atomic<uint64_t>& cluster_attr_set() {
  static std::atomic<uint64_t> done{0};
  return done;
}

// Shared-memory limit and permission for clusters above the portable size of 8, once
// per device (see raise_smem_limit_once for why attributes are set only once).
template <int W>
static cudaError_t prepare_cluster_kernel() {
  const void* kern = (const void*)k_tridiag<false, W, true>;
  cudaError_t e = raise_smem_limit_once(kern, smem_limit_set<false, W + 100>());
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? 1ull << dev : 0;
  if (cluster_attr_set<W>().load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) cluster_attr_set<W>().fetch_or(bit, std::memory_order_release);
  return e;
}

template <int W>
static cudaLaunchConfig_t cluster_config(int nclusters, int csize, size_t smem, cudaStream_t s,
                                         cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * csize), 1, 1);
  cfg.blockDim = dim3(W * 32, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int W>
static cudaError_t launch_cluster_one(int nclusters, int csize, const TridiagLaunch& L,
                                      cudaStream_t s) {
  cudaError_t e = prepare_cluster_kernel<W>();
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg =
      cluster_config<W>(nclusters, csize, tridiag_smem_bytes(false, L.max_m, W), s, attr);
  e = cudaLaunchKernelEx(&cfg, k_tridiag<false, W, true>, L);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_tridiag_cluster(int warps, int nclusters, int csize, const TridiagLaunch& L,
                                   cudaStream_t s) {
  switch (warps) {
    case 8: return launch_cluster_one<8>(nclusters, csize, L, s);
    case 12: return launch_cluster_one<12>(nclusters, csize, L, s);
    case 16: return launch_cluster_one<16>(nclusters, csize, L, s);
  }
  return cudaErrorInvalidValue;
}

// ---- group variant: `group` CTAs per matrix, resident together (cooperative launch)

template <int W>
std::atomic<uint64_t>& group_limit_set() {
  static std::atomic<uint64_t> done{0};
  return done;
}

template <int W>
static cudaError_t launch_group_one(int nctas, const TridiagLaunch& L, cudaStream_t s) {
  const void* kern = (const void*)k_tridiag<false, W, false, false, true>;
  cudaError_t e = raise_smem_limit_once(kern, group_limit_set<W>());
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas, 1, 1);
  cfg.blockDim = dim3(W * 32, 1, 1);
  cfg.dynamicSmemBytes = tridiag_smem_bytes(false, L.max_m, W);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once, or no launch
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_tridiag<false, W, false, false, true>, L);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Launch ngroups groups of `group` CTAs (L.group must equal group; L.ntasks <= ngroups).
cudaError_t launch_tridiag_group(int warps, int ngroups, int group, const TridiagLaunch& L,
                                 cudaStream_t s) {
  if (L.group != group || !L.gsync || !L.gw || group < 1) return cudaErrorInvalidValue;
  switch (warps) {
    case 12: return launch_group_one<12>(ngroups * group, L, s);
    case 16: return launch_group_one<16>(ngroups * group, L, s);
  }
  return cudaErrorInvalidValue;
}

// Self-test of the bounded barrier: one group of L.group >= 2 CTAs of which only
// L.group - 1 are launched, so the group's first barrier never fills and every launched
// CTA gives up after the wait limit with ST_TIMEOUT (L.ntasks = 1).
cudaError_t launch_tridiag_group_short(const TridiagLaunch& L, cudaStream_t s) {
  if (L.group < 2 || !L.gsync || !L.gw || L.ntasks != 1) return cudaErrorInvalidValue;
  return launch_group_one<16>(L.group - 1, L, s);
}

// CTAs of the group variant that fit on one SM for matrices up to max_m (0 on error).
int tridiag_group_blocks_per_sm(int warps, int max_m) {
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  const size_t smem = tridiag_smem_bytes(false, max_m, warps);
  if (warps == 12) {
    e = raise_smem_limit_once((const void*)k_tridiag<false, 12, false, false, true>,
                              group_limit_set<12>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag<false, 12, false, false, true>,
                                                        384, smem);
  } else if (warps == 16) {
    e = raise_smem_limit_once((const void*)k_tridiag<false, 16, false, false, true>,
                              group_limit_set<16>());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag<false, 16, false, false, true>,
                                                        512, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// Clusters of csize CTAs of the `warps`-warp cluster variant that fit on the device at
// once for matrices up to max_m (0 if none, or on an error).
int tridiag_max_active_clusters(int warps, int csize, int max_m) {
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  cudaLaunchAttribute attr[1];
#define EEID_CLQ(W_)                                                                            \
  if (warps == W_) {                                                                             \
    e = prepare_cluster_kernel<W_>();                                                            \
    if (e == cudaSuccess) {                                                                      \
      cudaLaunchConfig_t cfg =                                                                   \
          cluster_config<W_>(1, csize, tridiag_smem_bytes(false, max_m, W_), nullptr, attr);    \
      e = cudaOccupancyMaxActiveClusters(&n, k_tridiag<false, W_, true>, &cfg);                  \
    }                                                                                            \
  }
  EEID_CLQ(8) EEID_CLQ(12) EEID_CLQ(16)
#undef EEID_CLQ
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Occupancy query used by the planner to size persistent grids.
cudaError_t preload_tridiag() {
  cudaError_t e = cudaSuccess;
#define EEID_PRE(S_, W_) \
  if (e == cudaSuccess) e = raise_smem_limit_once((const void*)k_tridiag<S_, W_>, smem_limit_set<S_, W_>());
  EEID_PRE(true, 1) EEID_PRE(true, 2) EEID_PRE(true, 4) EEID_PRE(true, 8)
  EEID_PRE(false, 1) EEID_PRE(false, 2) EEID_PRE(false, 4) EEID_PRE(false, 8) EEID_PRE(false, 12)
  EEID_PRE(false, 16)
#undef EEID_PRE
  if (e == cudaSuccess)
    e = raise_smem_limit_once((const void*)k_tridiag<false, 4, false, true>, smem_limit_set<false, 204>());
  if (e == cudaSuccess)
    e = raise_smem_limit_once((const void*)k_tridiag<false, 8, false, true>, smem_limit_set<false, 208>());
  if (e == cudaSuccess) e = prepare_cluster_kernel<8>();
  if (e == cudaSuccess) e = prepare_cluster_kernel<12>();
  if (e == cudaSuccess) e = prepare_cluster_kernel<16>();
  if (e == cudaSuccess)
    e = raise_smem_limit_once((const void*)k_tridiag<false, 12, false, false, true>,
                              group_limit_set<12>());
  if (e == cudaSuccess)
    e = raise_smem_limit_once((const void*)k_tridiag<false, 16, false, false, true>,
                              group_limit_set<16>());
  return e;
}

int tridiag_blocks_per_sm(bool smem_path, int warps, int max_m, bool hi) {
  const size_t smem = tridiag_smem_bytes(smem_path, max_m, warps);
  int nb = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (hi && !smem_path) {
    if (warps == 4) {
      e = raise_smem_limit_once((const void*)k_tridiag<false, 4, false, true>, smem_limit_set<false, 204>());
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag<false, 4, false, true>, 128, smem);
    } else if (warps == 8) {
      e = raise_smem_limit_once((const void*)k_tridiag<false, 8, false, true>, smem_limit_set<false, 208>());
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag<false, 8, false, true>, 256, smem);
    }
    return e == cudaSuccess ? nb : 0;
  }
#define EEID_OCC(S_, W_)                                                                   \
  if (smem_path == S_ && warps == W_) {                                                    \
    e = raise_smem_limit_once((const void*)k_tridiag<S_, W_>, smem_limit_set<S_, W_>());    \
    if (e == cudaSuccess)                                                                  \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tridiag<S_, W_>, W_ * 32, smem); \
  }
  EEID_OCC(true, 1) EEID_OCC(true, 2) EEID_OCC(true, 4) EEID_OCC(true, 8)
  EEID_OCC(false, 1) EEID_OCC(false, 2) EEID_OCC(false, 4) EEID_OCC(false, 8) EEID_OCC(false, 12)
  EEID_OCC(false, 16)
#undef EEID_OCC
  return e == cudaSuccess ? nb : 0;
}

}  // namespace eeid
