// Host-side planning rules of the CUDA path: how a group of Householder reductions is
// split into launches, how the serving loop bands requests by cost, and the serving
// loop's pinned staging allocator.  Plain C++ with no CUDA dependency, so the host
// tests compile and check these rules on a CPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <iterator>
#include <map>
#include <vector>

namespace eeid {

// Time of one round of the 8-warp global variant at two CTAs per SM (twice the
// matrices) over one round of the 16-warp variant at one CTA per SM, measured on
// GB300 at m = 1023 (the second CTA's reduction and reflector phases overlap the
// first's tile pass, so the FP64 pipe stays busier).
constexpr double kRound8x2Per16 = 1.89;

// Launch plan of one group of near-equal reductions (one cost-sorted task list).
struct RoundPlan {
  bool hybrid = false;  // whole rounds run on the 8-warp variant, two CTAs per SM
  int bulk_grid = 0;    // persistent grid of the first launch
  int tail_at = 0;      // first task of the tail launch (0: no tail launch)
  int tail_grid = 0;    // grid of the tail launch (it runs the group's default variant)
};

// nt: tasks in the group; grid: its default persistent grid; sms: SMs on the device;
// wide: the default variant is a global-slot one of 12 or more warps; blocks8: CTAs per
// SM of the 8-warp global variant at this size (0 when it may not be used: unsupported
// size or a user tuning rule); uniform: all task sizes within 1 of each other;
// last_a: position of the last reduction of an A in the cost-sorted list (every A must
// run in the first launch, since the minors' bisection brackets come from its
// eigenvalues).
//
// Hybrid rounds: with one wide CTA per SM by default and two 8-warp CTAs fitting,
// whole pair-rounds are faster (kRound8x2Per16 < 2); a remainder of at most one round
// becomes the tail.  Otherwise a partial last round (leaving at least 1/16 of the grid
// idle) becomes the tail.  The tail launch runs on a second stream while the caller's
// stream bisects the first launch's matrices on the SMs the tail leaves free.
inline RoundPlan plan_rounds(int nt, int grid, int sms, bool wide, int blocks8, bool uniform,
                             int last_a) {
  RoundPlan p;
  p.bulk_grid = grid;
  if (!uniform || nt <= 0 || grid <= 0) return p;
  if (wide && blocks8 >= 2 && grid == sms) {
    const int g8 = sms * blocks8;
    const int bulk = nt / g8 * g8, r = nt - bulk;
    const double t_hybrid = (double)(bulk / g8) * kRound8x2Per16 + (r > 0 ? 1.0 : 0.0);
    const double t_plain = (double)((nt + grid - 1) / grid);
    if (bulk > 0 && r <= grid && t_hybrid < t_plain && last_a < bulk) {
      p.hybrid = true;
      p.bulk_grid = g8;
      if (r > 0) {
        p.tail_at = bulk;
        p.tail_grid = r;
      }
      return p;
    }
  }
  const int r = nt % grid;
  if (nt > grid && r > 0 && grid - r >= std::max(1, grid / 16) && last_a < nt - r) {
    p.tail_at = nt - r;
    p.tail_grid = r;
  }
  return p;
}

// Cluster plan of one group of reductions: when the group has at most half as many
// matrices as the device has SMs (a few components, or the eigenvalues of one large A,
// the paper's Table 1 tasks), one thread-block cluster of C CTAs reduces each matrix
// instead of one CTA, so the whole group runs in one round on up to C times the SMs.
// C is the largest power of two with nt * C <= sms, at most the cluster limit (16);
// 0 = no cluster plan (too many matrices, or matrices below min_m, whose per-step
// serial phases would dominate a split pass).  The caller then halves C while the
// device cannot hold nt such clusters at once.
constexpr int kClusterMaxCtas = 16;
constexpr int kClusterMinM = 384;
inline int cluster_size_for(int nt, int sms, int max_m, int min_m = kClusterMinM) {
  if (nt < 1 || max_m < min_m || 2 * nt > sms) return 0;
  int c = 1;
  while (2 * c <= kClusterMaxCtas && nt * 2 * c <= sms) c *= 2;
  return c >= 2 ? c : 0;
}

// The narrow global builds of K-a (1 or 2 warps a matrix, 16 or 8 CTAs per SM) win only
// on waves that fill the SMs with them: a group keeps such a build only when it holds at
// least half the SMs' worth of its CTAs (nt * 2 >= sms * blocks_per_sm), and otherwise
// runs 4 warps a matrix (every global build gives the same bits).
inline bool narrow_build_fills(int64_t nt, int sms, int blocks_per_sm) {
  return nt * 2 >= (int64_t)sms * blocks_per_sm;
}

// Group plan (the group variant): when even clusters of 16 would leave most SMs idle (a
// call with a handful of large reductions, e.g. one component of a large A: A and one
// minor), G = sms / nt CTAs reduce each matrix, resident together through a cooperative
// launch, meeting at global-memory barriers.  0 = no group plan (G would not exceed the
// cluster limit, or the matrices are below min_m, where two global barriers a step cost
// more than the split saves).
constexpr int kGroupMinM = 1536;
inline int group_size_for(int nt, int sms, int max_m, int min_m = kGroupMinM) {
  if (nt < 1 || max_m < min_m) return 0;
  const int g = sms / nt;
  return g > kClusterMaxCtas ? g : 0;
}

// Efficiency of a reduction split over a cluster of c CTAs, relative to one CTA, for an
// m x m matrix.  The phases outside the fused pass (column update, reflector, the sums of
// the partials, w) run redundantly in every CTA of a cluster and do not shrink with c;
// they cost about sigma(m) = 40.8/m of a one-CTA step (measured: clusters of 16 at
// m = 4001 ran at 81% of the per-SM FP64 peak against 94% for one CTA per matrix, so
// 1/(1 + 16 sigma) = 0.86).  e(c) = 1 / (1 + c sigma(m)).
constexpr double kClusterSerialPerM = 40.8;
inline double cluster_efficiency(int c, int m) {
  return 1.0 / (1.0 + (double)c * kClusterSerialPerM / (double)(m > 0 ? m : 1));
}

// Cluster rounds for a large uniform group (nt near-equal reductions of size m, more
// than half the SMs, too many for the one-round cluster plan): whole rounds with
// clusters of c1 CTAs (bulk tasks), then one launch of the remaining nt - bulk tasks with
// clusters of c2, so that a partial last round of one CTA per matrix does not leave SMs
// idle.  active[k] = clusters of 2^(k+1) CTAs the device holds at once (k = 0..3).
// t_single: the time of the one-CTA plan in units of one one-CTA reduction (the caller
// takes it from plan_rounds).  Returns c1 = 0 unless the estimate beats t_single by 5%.
struct ClusterRounds {
  int c1 = 0;      // cluster size of the whole rounds
  int per_round = 0;
  int bulk = 0;    // tasks in the whole rounds
  int c2 = 0;      // cluster size of the last launch (0: none)
  double t = 0;    // estimated time, units of one one-CTA reduction
};
inline ClusterRounds plan_cluster_rounds(int nt, int sms, int m, const int active[4],
                                         double t_single, int min_m = kClusterMinM) {
  ClusterRounds best;
  if (nt < 1 || m < min_m) return best;
  for (int k1 = 0; k1 < 2; ++k1) {           // c1 = 2 or 4
    const int c1 = 2 << k1;
    const int K = active[k1];
    if (K < 1) continue;
    const int rounds = nt / K, rem = nt - rounds * K;
    double t = rounds / (c1 * cluster_efficiency(c1, m));
    int c2 = 0;
    if (rem > 0) {
      for (int k2 = 3; k2 >= 0 && !c2; --k2) {
        const int c = 2 << k2;
        if (rem * c <= sms && active[k2] >= rem) c2 = c;
      }
      t += c2 ? 1.0 / (c2 * cluster_efficiency(c2, m)) : 1.0;
    }
    if (rounds > 0 && (best.c1 == 0 || t < best.t)) {
      best.c1 = c1;
      best.per_round = K;
      best.bulk = rounds * K;
      best.c2 = c2;
      best.t = t;
    }
  }
  if (best.c1 && !(best.t < 0.95 * t_single)) best = ClusterRounds();
  return best;
}

// Bisection blocks for a list of tasks (order: task indices, largest first; m_of(t): the
// size of task t).  A task larger than half a block gets blocks of `threads` eigenvalues
// each ({t, k0, 1}); runs of consecutive task indices of one size m >= 4 (the minors of
// one matrix) share a block, up to min(threads / m, max_pack) of them ({t, 0, run}).
struct BisectBlock {
  int task, k0, ntask;
};
template <class MOf>
inline void plan_bisect_blocks(const std::vector<int>& order, MOf m_of, int threads, int max_pack,
                               std::vector<BisectBlock>& out) {
  for (size_t q = 0; q < order.size();) {
    const int t = order[q], m = m_of(t);
    const int cap = (m >= 4 && 2 * m <= threads) ? std::min(threads / m, max_pack) : 1;
    int run = 1;
    while (run < cap && q + run < order.size() && order[q + run] == t + run && m_of(t + run) == m)
      ++run;
    if (run > 1) {
      out.push_back({t, 0, run});
    } else {
      for (int k0 = 0; k0 < m; k0 += threads) out.push_back({t, k0, 1});
    }
    q += (size_t)run;
  }
}

// Serving: cost band of a request, from n^3 (columns + 1), which is proportional to its
// Householder work (the reductions dominate).  Everything below kTinyCost is band 0,
// then one band per factor of 8.  A batch holds requests of one band only.
constexpr double kTinyCost = 1e9;
inline int cost_band(int64_t n, int64_t ncols) {
  const double c = (double)n * (double)n * (double)n * (double)(ncols + 1);
  if (c < kTinyCost) return 0;
  return 1 + (int)(std::log2(c / kTinyCost) / 3.0);
}

// Serving: a pinned staging pool, one page-locked region carved first-fit in 256-byte
// granules, neighbours coalesced on release.  CUDA serialises work of different
// streams around a page-locked allocation, so request buffers come from here.  Not
// thread-safe: the serving loop guards it with its mutex.
struct PinnedPool {
  char* base = nullptr;
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length

  static size_t granule(size_t n) { return (n + 255) & ~(size_t)255; }
  void init(char* b, size_t sz) {
    base = b;
    size = b ? sz : 0;
    free_.clear();
    if (size) free_[0] = size;
  }
  char* take(size_t n) {
    n = granule(n);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        const size_t off = it->first, rest = it->second - n;
        free_.erase(it);
        if (rest) free_[off + n] = rest;
        return base + off;
      }
    return nullptr;
  }
  void give(char* p, size_t n) {
    n = granule(n);
    size_t off = (size_t)(p - base);
    auto next = free_.lower_bound(off);
    if (next != free_.end() && off + n == next->first) {
      n += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += n;
        return;
      }
    }
    free_[off] = n;
  }
};

}  // namespace eeid
