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
