// Internal declarations shared by the eeid CUDA translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace eeid {

// Raise a kernel's dynamic shared memory limit to the device's opt-in maximum, once per
// device (one bit of `done` per device).  The limit is only a ceiling, since every launch
// passes its own size.  Changing it while launches of the kernel are queued makes the call
// wait for them, which would serialise otherwise independent streams (two contexts, or
// the serving loop's two batches).  So it is set once and never touched again.
inline cudaError_t raise_smem_limit_once(const void* kernel, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // devices 0..63 are remembered; a higher index is simply set again each time
  const uint64_t bit = dev < 64 ? 1ull << dev : 0;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Device status bits (OR-ed by kernels into a workspace word, read by eeid_sync).
enum : unsigned {
  ST_DEGENERATE = 1u,      // exactly equal eigenvalues of A: Eq. 1 is 0/0
  ST_SMALL_GAP = 2u,       // min relative gap < 1e-4
  ST_BRACKET_FALLBACK = 4u,// an interlacing bracket failed its Sturm check (info)
  ST_BAD_TASK = 8u,        // a kernel met a task it cannot run (size limit)
  ST_TIMEOUT = 16u,        // a bounded wait of a cooperative reduction ran out (no result)
};

// ---------------------------------------------------------------- K-a tridiag
// One matrix to reduce to symmetric tridiagonal form: the parent A (n x n,
// row-major, lower triangle read) with row/column `skip` removed (skip < 0: A
// itself).  Outputs d[m] and e[m-1], m = n - (skip >= 0).
//
// rot >= 0 (with skip >= 0, rot != skip) selects the rotated minor used for signs:
// coordinates rot and skip are first rotated by 45 degrees, u = (e_rot + e_skip)/sqrt2
// and w = (e_rot - e_skip)/sqrt2, and u is removed.  The minor keeps w in the place of
// rot: its row there is (a_rot,k - a_skip,k)/sqrt2 and its diagonal entry
// (a_rot,rot + a_skip,skip)/2 - a_rot,skip.  Eq. 1 on it gives (v_i,rot + v_i,skip)^2 / 2.
struct TridiagTask {
  const double* A;
  int64_t lda;
  int n;
  int skip;
  double* d;
  double* e;
  int rot = -1;
  int pad_ = 0;
};

// Largest m the shared-memory-resident path accepts, per CTA warp count.
constexpr int kTridiagSmemMaxM = 160;
// Largest m any tridiagonalisation kernel accepts (vector staging in shared memory).
constexpr int kTridiagMaxM = 4096;

struct TridiagLaunch {
  const TridiagTask* tasks;  // device array, cost-sorted (largest first)
  int ntasks;
  int* counter;              // device work counter, zeroed before launch
  double* work;              // global path: per-CTA working matrices
  int64_t work_stride;       // doubles per CTA slot (matrix + partials)
  int max_m;                 // largest m among tasks (sizes the per-CTA layout)
  unsigned* status;
  // Group variant only: `group` CTAs reduce task (blockIdx.x / group) together.  gsync:
  // per group kGroupSyncWords words (arrival counter, abort flag), zero at launch; gw: per
  // group a vector of VM doubles through which the CTAs exchange w.
  int group = 0;
  unsigned* gsync = nullptr;
  double* gw = nullptr;
};
constexpr int kGroupSyncWords = 8;

size_t tridiag_global_slot_doubles(int max_m);
size_t tridiag_smem_bytes(bool smem_path, int max_m, int warps);
// hi: the high-occupancy build of the global-slot variant (warps 4 or 8 only).
cudaError_t launch_tridiag(bool smem_path, int warps, int grid, const TridiagLaunch& L,
                           cudaStream_t s, bool hi = false);

// ---------------------------------------------------------------- K-b bisect
// Eigenvalues of one symmetric tridiagonal (d[m], e[m-1]).  With parent != nullptr
// the m eigenvalues are minor eigenvalues interlaced by the parent's m+1 ascending
// eigenvalues (bracket [parent[k], parent[k+1]]); otherwise Gershgorin brackets.
struct BisectTask {
  const double* d;
  const double* e;
  int m;
  const double* parent;
  double* eig;
};
// A block's share of a task: eigenvalues [k0, k0 + blockDim.x).  With ntask > 1 the block
// instead takes all eigenvalues of the ntask consecutive tasks task .. task + ntask - 1,
// all of one size m with ntask * m <= kBisectThreads (lane t: task t / m, eigenvalue t % m):
// small minors of one matrix share a block.
struct BisectItem {
  int task;
  int k0;
  int ntask = 1;
};
constexpr int kBisectThreads = 256;
constexpr int kBisectMaxPack = 64;   // packed tasks per block (so m >= 4 when packing)
// threads: block size (a multiple of 32, at most kBisectThreads; the items were planned for
// it).  Launches with few eigenvalues use small blocks so that they reach more SMs.
cudaError_t launch_bisect(const BisectTask* tasks, const BisectItem* items, int nitems,
                          int max_m, unsigned* status, cudaStream_t s,
                          int threads = kBisectThreads);

// ---------------------------------------------------------------- K-c identity
// D_i = prod_{k != i} |lam_i - lam_k| for the requested eigen-indices i = rows[r] of
// one problem, kept as a mantissa dm[i] in [0.5, 1) (0 if degenerate) and a binary
// exponent de[i] (arrays indexed by i, n long).
struct DenomTask {
  const double* lam;
  int n;
  double* dm;
  int* de;
  const int* rows;
  int nrows;
};
// A block's share of a task: rows [r0, r0 + kDenomThreads).
struct DenomItem {
  int task;
  int r0;
};
constexpr int kDenomThreads = 256;
cudaError_t launch_denominators(const DenomTask* tasks, const DenomItem* items, int nitems,
                                int max_n, unsigned* status, cudaStream_t s);

// One identity block: column c of one problem (minor eigenvalues mu[n-1]) for the
// rows [r0, r0 + blockDim.x) of that problem's row list.
struct IdentityProblem {
  const double* lam;     // n
  const double* dm;      // n
  const int* de;         // n
  const double* mu;      // ncols x (n-1)
  const int* rows;       // nrows eigen-indices (device)
  int n, nrows, ncols;
  double* out;           // nrows x ncols
};
struct IdentityItem {
  int prob;
  int col;
  int r0;
};
constexpr int kIdentityThreads = 128;
cudaError_t launch_identity(const IdentityProblem* probs, const IdentityItem* items, int nitems,
                            int max_n, cudaStream_t s);

// Load every kernel of a translation unit (and raise its shared memory limit) now.
// With lazy module loading a kernel is otherwise loaded at its first launch, and a
// load issued while other kernels run waits for them: the first batch of a serving
// process would serialise behind whatever it overlaps.
cudaError_t preload_tridiag();
cudaError_t preload_bisect();
cudaError_t preload_identity();

// Deterministic symmetric matrix (uniform [-0.5, 0.5) entries) for the autotuner.
cudaError_t launch_fill_symmetric(double* A, int n, int64_t lda, unsigned long long seed,
                                  cudaStream_t s);

}  // namespace eeid
