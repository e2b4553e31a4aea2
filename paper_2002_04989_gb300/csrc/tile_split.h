// Split of one step's fused pass over the warps of the global-slot Householder variants
// (one CTA, a cluster or a group).  Plain C++ that also compiles as device code, so the
// host tests check the partition on a CPU.
#pragma once

#ifdef __CUDACC__
#define EEID_HD __host__ __device__ __forceinline__
#else
#define EEID_HD inline
#endif

namespace eeid {

// The nb(nb+1)/2 lower-triangle tiles of one step, in row-major order t = I(I+1)/2 + J,
// split over GW warps by count: warp w takes the tiles [start(w), start(w+1)).  (A split
// weighted toward cheaper diagonal tiles measured slower: a diagonal tile's
// matrix-vector half is one dependent FMA chain, so it costs about a full tile.)  Which
// warp runs a tile does not change the tile's arithmetic, so the split never shows in
// the results.
EEID_HD int tile_start(int w, int nb, int GW) {
  const long long T = (long long)nb * (nb + 1) / 2;
  return (int)((long long)w * T / GW);
}

}  // namespace eeid
