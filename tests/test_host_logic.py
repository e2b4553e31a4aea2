"""Host-side planning rules of the CUDA path (csrc/host_plan.h), compiled with the host
C++ compiler and checked on the CPU: how a group of near-equal Householder reductions is
split into launches (hybrid rounds, tail overlap), the serving cost bands, and the
serving loop's pinned staging allocator, and the cluster plan of few large reductions."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2002_04989_gb300", "csrc")

DRIVER = r"""
#include "host_plan.h"
#include "tile_split.h"
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>
#include <random>
#include <algorithm>
using namespace eeid;
int main(int argc, char** argv) {
  if (!strcmp(argv[1], "plan")) {
    // nt grid sms wide blocks8 uniform last_a
    int a[7];
    for (int i = 0; i < 7; ++i) a[i] = atoi(argv[2 + i]);
    RoundPlan p = plan_rounds(a[0], a[1], a[2], a[3] != 0, a[4], a[5] != 0, a[6]);
    printf("%d %d %d %d\n", p.hybrid ? 1 : 0, p.bulk_grid, p.tail_at, p.tail_grid);
  } else if (!strcmp(argv[1], "cluster")) {
    printf("%d\n", cluster_size_for(atoi(argv[2]), atoi(argv[3]), atoi(argv[4])));
  } else if (!strcmp(argv[1], "tsplit")) {
    // every (nb, GW): the ranges partition the tiles in order, and no warp takes more
    // than the mean plus one tile
    double worst = 0.0;
    for (int nb = 1; nb <= 130; ++nb)
      for (int GW : {1, 2, 3, 4, 8, 12, 16, 24, 48, 96, 128, 192, 256, 608, 912, 1216, 2432}) {
        const int T = nb * (nb + 1) / 2;
        if (tile_start(0, nb, GW) != 0 || tile_start(GW, nb, GW) != T) { printf("BAD ends %d %d\n", nb, GW); return 1; }
        const double mean = (double)T / GW;
        for (int w = 0; w < GW; ++w) {
          const int a = tile_start(w, nb, GW), b = tile_start(w + 1, nb, GW);
          if (b < a) { printf("BAD order %d %d %d\n", nb, GW, w); return 1; }
          const double c = b - a;
          if (c > mean + 1.0 + 1e-9) { printf("BAD balance %d %d %d %f %f\n", nb, GW, w, c, mean); return 1; }
          worst = std::max(worst, c - mean);
        }
      }
    printf("ok %.3f\n", worst);
  } else if (!strcmp(argv[1], "narrow")) {
    printf("%d\n", narrow_build_fills(atoll(argv[2]), atoi(argv[3]), atoi(argv[4])) ? 1 : 0);
  } else if (!strcmp(argv[1], "group")) {
    printf("%d\n", group_size_for(atoi(argv[2]), atoi(argv[3]), atoi(argv[4])));
  } else if (!strcmp(argv[1], "crounds")) {
    // nt sms m a2 a4 a8 a16 t_single
    int act[4] = {atoi(argv[5]), atoi(argv[6]), atoi(argv[7]), atoi(argv[8])};
    ClusterRounds r = plan_cluster_rounds(atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), act, atof(argv[9]));
    printf("%d %d %d %d %.4f\n", r.c1, r.per_round, r.bulk, r.c2, r.t);
  } else if (!strcmp(argv[1], "bblocks")) {
    // sizes of tasks 0..k-1 follow; order = every task, largest first (stable)
    std::vector<int> m;
    for (int i = 2; i < argc; ++i) m.push_back(atoi(argv[i]));
    std::vector<int> order(m.size());
    for (size_t i = 0; i < m.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return m[a] > m[b]; });
    std::vector<BisectBlock> out;
    plan_bisect_blocks(order, [&](int t) { return m[t]; }, 256, 64, out);
    for (auto& b : out) printf("%d %d %d\n", b.task, b.k0, b.ntask);
  } else if (!strcmp(argv[1], "band")) {
    printf("%d\n", cost_band(atoll(argv[2]), atoll(argv[3])));
  } else if (!strcmp(argv[1], "pool")) {
    const size_t size = (size_t)1 << 24;
    std::vector<char> mem(size);
    PinnedPool pool;
    pool.init(mem.data(), size);
    std::mt19937_64 rng(atoi(argv[2]));
    struct Blk { char* p; size_t n; };
    std::vector<Blk> live;
    long takes = 0, fails = 0;
    for (int step = 0; step < 20000; ++step) {
      if (live.empty() || rng() % 3) {
        size_t n = 1 + rng() % 200000;
        char* p = pool.take(n);
        if (!p) { ++fails; continue; }
        ++takes;
        // inside the region, 256-byte aligned offset, no overlap with a live block
        if (p < mem.data() || p + n > mem.data() + size || (p - mem.data()) % 256) { printf("BAD range\n"); return 1; }
        for (auto& b : live)
          if (p < b.p + PinnedPool::granule(b.n) && b.p < p + PinnedPool::granule(n)) { printf("BAD overlap\n"); return 1; }
        live.push_back({p, n});
      } else {
        size_t i = rng() % live.size();
        pool.give(live[i].p, live[i].n);
        live.erase(live.begin() + i);
      }
      // free list: sorted, disjoint, no two adjacent blocks left uncoalesced
      size_t end = 0; bool first = true;
      for (auto& kv : pool.free_) {
        if (!first && kv.first <= end) { printf("BAD free list %zu %zu\n", kv.first, end); return 1; }
        end = kv.first + kv.second; first = false;
      }
    }
    for (auto& b : live) pool.give(b.p, b.n);
    printf("%ld %ld %zu %zu %zu\n", takes, fails, pool.free_.size(),
           pool.free_.empty() ? (size_t)0 : pool.free_.begin()->first,
           pool.free_.empty() ? (size_t)0 : pool.free_.begin()->second);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("host_plan")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(*args):
        out = subprocess.run([str(exe), *map(str, args)], capture_output=True, text=True, check=True)
        return out.stdout.split()
    return run


def plan(driver, nt, grid=152, sms=152, wide=1, blocks8=2, uniform=1, last_a=0):
    h, bulk, at, tg = map(int, driver("plan", nt, grid, sms, wide, blocks8, uniform, last_a))
    return bool(h), bulk, at, tg


def test_plan_benchmark_sizes(driver):
    # n = 1024, all columns: 1025 reductions -> three 8-warp pair-rounds + a 113-task tail
    assert plan(driver, 1025) == (True, 304, 912, 113)
    # 304 tasks: one pair-round beats two 16-warp rounds, nothing left for a tail
    assert plan(driver, 304) == (True, 304, 0, 0)
    # n = 4096 (the 8-warp variant does not fit twice per SM): 257 tasks, 105-task tail
    assert plan(driver, 257, blocks8=1) == (False, 152, 152, 105)
    # n = 520: remainder of the pair-rounds (217) exceeds one round -> plain tail of 65
    assert plan(driver, 521) == (False, 152, 456, 65)
    # exactly one round: nothing to split
    assert plan(driver, 152) == (False, 152, 0, 0)


def test_plan_refusals(driver):
    # sizes not within 1 of each other: no split at all
    assert plan(driver, 1025, uniform=0) == (False, 152, 0, 0)
    # an A among the last tasks: its eigenvalues must come from the first launch
    assert plan(driver, 1025, last_a=1000) == (False, 152, 0, 0)
    # a last round that leaves fewer than 1/16 of the SMs idle is not worth a second launch
    assert plan(driver, 600, blocks8=0) == (False, 152, 0, 0)
    # a narrow default (4-warp variant at several CTAs per SM) is never replaced
    assert plan(driver, 1025, grid=608, wide=0)[0] is False
    # a budget-shrunk grid (fewer CTAs than SMs) does not use pair-rounds
    assert plan(driver, 1025, grid=100)[0] is False


def test_plan_invariants(driver):
    rng = np.random.default_rng(3)
    for _ in range(300):
        sms = int(rng.integers(8, 200))
        grid = sms
        nt = int(rng.integers(1, 6 * sms))
        blocks8 = int(rng.integers(0, 3))
        last_a = int(rng.integers(0, nt))
        h, bulk, at, tg = plan(driver, nt, grid, sms, 1, blocks8, 1, last_a)
        assert 0 <= at < nt or at == 0
        if at:
            assert last_a < at                       # every A in the first launch
            assert 0 < tg <= grid and tg == nt - at  # the tail is at most one round
            assert grid - tg >= max(1, grid // 16) or h
        if h:
            assert blocks8 >= 2 and bulk == sms * blocks8
            assert at == 0 or at % bulk == 0         # the first launch is whole pair-rounds


def test_cost_bands(driver):
    band = lambda n, c: int(driver("band", n, c)[0])
    assert band(16, 1) == 0 and band(100, 100) == 0            # below 1e9: one band
    assert band(2048, 2048) == 5                               # 2048^3 * 2049 ~ 1.8e13
    assert band(1200, 1200) == 4
    costs = sorted((n ** 3 * (c + 1), n, c) for n in (16, 64, 200, 500, 1000, 2048)
                   for c in (1, 8, 64, n))
    bands = [band(n, c) for _, n, c in costs]
    assert bands == sorted(bands)                              # monotone in the cost
    # n = 1000 gives n^3 = 1e9: bands change where (columns + 1) crosses a power of 8
    assert [band(1000, c) for c in (0, 6, 7, 62, 63)] == [1, 1, 2, 2, 3]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pinned_pool(driver, seed):
    takes, fails, nfree, off, length = map(int, driver("pool", seed))
    assert takes > 5000
    # everything given back coalesces into the one region it started as
    assert (nfree, off, length) == (1, 0, 1 << 24)


def test_cluster_plan(driver):
    c = lambda nt, sms=152, m=4001: int(driver("cluster", nt, sms, m)[0])
    # one component of n = 4002 (A and one minor): two clusters of 16 CTAs
    assert c(2) == 16
    # the eigenvalues of one large A: one cluster of 16
    assert c(1) == 16
    # a few columns: the largest power of two with nt * C <= SMs
    assert c(5) == 16 and c(10) == 8 and c(19) == 8 and c(20) == 4 and c(38) == 4
    assert c(39) == 2 and c(76) == 2
    # more matrices than half the SMs, or small matrices: one CTA per matrix
    assert c(77) == 0 and c(1025) == 0 and c(2, m=383) == 0
    rng = np.random.default_rng(4)
    for _ in range(200):
        nt, sms = int(rng.integers(1, 120)), int(rng.integers(2, 200))
        k = c(nt, sms)
        if k:
            assert k & (k - 1) == 0 and 2 <= k <= 16 and nt * k <= sms
            assert k == 16 or nt * 2 * k > sms       # the largest such power of two
        else:
            assert 2 * nt > sms


def test_tile_split_partitions_and_balances(driver):
    out = driver("tsplit")
    assert out[0] == "ok", out


def test_narrow_builds_only_on_full_waves(driver):
    f = lambda nt, sms=152, bps=16: driver("narrow", nt, sms, bps)[0] == "1"
    # a six-copy batch at n = 300 (1806 reductions) fills the 1-warp build's 2432 slots
    # at least half; a single n = 300 call (301 reductions) does not
    assert f(1806) and not f(301)
    # the 2-warp build (8 CTAs per SM): the boundary is half of 1216 slots
    assert f(608, bps=8) and not f(607, bps=8)
    # batch4096's (192, 256] slice: 316 matrices, about 71k reductions
    assert f(71000, bps=8)


def test_group_plan(driver):
    g = lambda nt, sms=152, m=4001: int(driver("group", nt, sms, m)[0])
    # one component of n = 4002 (A and one minor): two groups of 76 CTAs
    assert g(2) == 76
    # the eigenvalues of one large A: every SM
    assert g(1) == 152
    # as long as a group exceeds the cluster limit of 16
    assert g(3) == 50
    assert g(8) == 19 and g(9) == 0 and g(10) == 0
    # below the size floor (two global barriers a step would cost more than they save)
    assert g(2, m=1535) == 0 and g(2, m=1536) == 76
    rng = np.random.default_rng(6)
    for _ in range(200):
        nt, sms = int(rng.integers(1, 40)), int(rng.integers(2, 200))
        k = g(nt, sms)
        assert k == (sms // nt if sms // nt > 16 else 0)
        if k:
            assert nt * k <= sms


def test_cluster_rounds(driver):
    def cr(nt, sms=152, m=4095, act=(76, 38, 19, 9), t_single=None):
        if t_single is None:
            t_single = float(-(-nt // sms))
        c1, per, bulk, c2, t = driver("crounds", nt, sms, m, *act, t_single)
        return int(c1), int(per), int(bulk), int(c2), float(t)
    # n = 4096 with 256 columns: 257 reductions, two one-CTA rounds (105 in the second);
    # three rounds of 76 pairs, then the last 29 on clusters of 4 (116 SMs)
    c1, per, bulk, c2, t = cr(257)
    assert (c1, per, bulk, c2) == (2, 76, 228, 4) and t < 0.95 * 2
    # a group that fills its rounds exactly gains nothing from clusters
    assert cr(304)[0] == 0
    # smaller matrices: the redundant per-step phases cost more, so 1025 reductions of
    # m = 1023 stay with the one-CTA plan (whose pair-rounds are 6.67 rounds' time)
    assert cr(1025, m=1023, t_single=3 * 1.89 + 1)[0] == 0
    # below the size floor, never
    assert cr(257, m=300)[0] == 0
    rng = np.random.default_rng(5)
    for _ in range(200):
        nt = int(rng.integers(77, 1200))
        m = int(rng.integers(384, 4097))
        act = tuple(int(x) for x in (76, 38, 19, 9))
        c1, per, bulk, c2, t = cr(nt, m=m, act=act)
        if c1:
            assert c1 in (2, 4) and per == act[c1 // 2 - 1] and bulk % per == 0
            assert 0 < bulk <= nt and nt - bulk < per
            assert c2 == 0 or ((nt - bulk) * c2 <= 152 and c2 & (c2 - 1) == 0)
            assert t < 0.95 * -(-nt // 152)


def test_bisect_blocks(driver):
    """Minors of one matrix (consecutive tasks of one size) share bisection blocks; every
    eigenvalue of every task is covered exactly once; no block exceeds 256 lanes."""
    def blocks(sizes):
        out = driver("bblocks", *sizes)
        return [tuple(map(int, out[i:i + 3])) for i in range(0, len(out), 3)]
    # an A of 8 and its 8 minors of 7: A alone (8 lanes), the minors in one block
    assert blocks([8] + [7] * 8) == [(0, 0, 1), (1, 0, 8)]
    # 300 minors of 3 (too small to pack) and a 600 task split in 256-lane blocks
    b = blocks([600] + [3] * 2)
    assert b == [(0, 0, 1), (0, 256, 1), (0, 512, 1), (1, 0, 1), (2, 0, 1)]
    rng = np.random.default_rng(6)
    for _ in range(50):
        sizes = []
        for _ in range(int(rng.integers(1, 6))):     # a few "matrices": A then its minors
            n = int(rng.integers(2, 300))
            sizes += [n] + [n - 1] * int(rng.integers(0, n + 1))
        covered = {}
        for t, k0, nt in blocks(sizes):
            m = sizes[t]
            if nt > 1:
                assert nt * m <= 256 and nt <= 64 and m >= 4 and k0 == 0
                assert all(sizes[t + q] == m for q in range(nt))
                for q in range(nt):
                    for k in range(m):
                        covered[(t + q, k)] = covered.get((t + q, k), 0) + 1
            else:
                for k in range(k0, min(m, k0 + 256)):
                    covered[(t, k)] = covered.get((t, k), 0) + 1
        want = {(t, k) for t, m in enumerate(sizes) for k in range(m)}
        assert set(covered) == want and all(v == 1 for v in covered.values())
