// eeid_eigvals_noalloc: eigenvalues of A with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code embedded in an application whose own
// memory pool owns the whole device, or code on a latency-critical path where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.  They
// cannot create an eeid_ctx either (its workspace is allocated).  This entry point
// runs the same Householder kernel (K-a, global-slot variant) and the same
// bisection kernel (K-b) as eeid_eigvals, with all scratch -- the working matrix,
// the tile partial sums, d/e and the task descriptors -- in one file-scope
// __device__ array of fixed size.  The caller passes only A and the output.
#include "eeid.h"
#include "internal.cuh"

#include <mutex>
#include <string>

namespace eeid {
size_t tridiag_global_slot_doubles(int max_m);
void set_last_error(const char* msg);
}

using namespace eeid;

namespace {

// Largest n accepted.  The working matrix and its tile partial sums take
// n*round4(n) + nb^2*32 + nb*16*32 + 32 doubles (nb = ceil(n/32)); at n = 512 that is
// 278,560 doubles.
constexpr int kNoAllocMaxN = 512;
constexpr int kNoAllocWarps = 4;
constexpr size_t kNb = (kNoAllocMaxN + 31) / 32;
constexpr size_t kSlotDoubles = (size_t)kNoAllocMaxN * kNoAllocMaxN + 2 * kNb * kNb * 32 + 32;
constexpr size_t kDEDoubles = 2 * (size_t)kNoAllocMaxN;         // d[n], e[n-1]
constexpr size_t kMetaDoubles = 64;                              // 512 bytes of descriptors
constexpr size_t kScratchDoubles = kSlotDoubles + kDEDoubles + kMetaDoubles;

// Byte offsets inside the descriptor area.
constexpr size_t kOffTask = 0;       // TridiagTask
constexpr size_t kOffCounter = 64;   // int work counter (must start at 0)
constexpr size_t kOffBisect = 128;   // BisectTask
constexpr size_t kOffItems = 192;    // BisectItem[ceil(n/kBisectThreads)] (<= 4 items)
constexpr size_t kOffStatus = 256;   // unsigned status word
static_assert(sizeof(TridiagTask) <= 64, "descriptor layout");
static_assert(sizeof(BisectTask) <= 64, "descriptor layout");
static_assert(kOffItems + 4 * sizeof(BisectItem) <= kOffStatus, "descriptor layout");
static_assert(ST_DEGENERATE == EEID_DEV_DEGENERATE && ST_SMALL_GAP == EEID_DEV_SMALL_GAP &&
                  ST_BRACKET_FALLBACK == EEID_DEV_BRACKET_FALLBACK && ST_BAD_TASK == EEID_DEV_BAD_TASK &&
                  ST_TIMEOUT == EEID_DEV_TIMEOUT,
              "device status bits of the header");

// The scratch: 2.2 MB held by every GPU that loads the library, for the life of
// the process.  Every call uses it; calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Writes the descriptors for one call and clears what must start at zero: the work
// counter and the status word of this call (the caller's word, or the scratch's own).
__global__ void k_noalloc_setup(TridiagTask t, BisectTask b, int nitems, unsigned* status) {
  char* meta = (char*)(g_noalloc_scratch + kSlotDoubles + kDEDoubles);
  if (threadIdx.x == 0) {
    *(TridiagTask*)(meta + kOffTask) = t;
    *(int*)(meta + kOffCounter) = 0;
    *(BisectTask*)(meta + kOffBisect) = b;
    *status = 0u;
  }
  if ((int)threadIdx.x < nitems) {
    BisectItem it;
    it.task = 0;
    it.k0 = (int)threadIdx.x * kBisectThreads;
    ((BisectItem*)(meta + kOffItems))[threadIdx.x] = it;
  }
}

// Errors are reported through eeid_last_error(), like every other entry point.
eeid_status na_fail(eeid_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

// Device address of the scratch array, looked up once per device (with that
// device current) under a lock.  The same first call loads the two kernels and raises
// their shared-memory limits, so that later calls change no kernel attribute.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_ptr[kMaxDevices] = {};

eeid_status scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return na_fail(EEID_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    if (tridiag_global_slot_doubles(kNoAllocMaxN) > kSlotDoubles)
      return na_fail(EEID_ERR_INVALID, "internal: scratch layout smaller than the kernel needs");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(EEID_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                                        cudaGetErrorString(e));
    e = preload_tridiag();
    if (e == cudaSuccess) e = preload_bisect();
    if (e != cudaSuccess)
      return na_fail(EEID_ERR_CUDA, std::string("kernel set-up failed: ") + cudaGetErrorString(e));
    g_ptr[dev] = (double*)p;
  }
  *out = g_ptr[dev];
  return EEID_OK;
}

}  // namespace

extern "C" {

eeid_status eeid_eigvals_noalloc(const double* dA, int64_t lda, int64_t n, double* d_lambda,
                                 unsigned* d_status_opt, void* stream) {
  if (n < 0) return na_fail(EEID_ERR_INVALID, "n < 0");
  if (n == 0) return EEID_OK;
  if (n > kNoAllocMaxN)
    return na_fail(EEID_ERR_INVALID, "eeid_eigvals_noalloc: n = " + std::to_string(n) +
                                         " exceeds the fixed scratch limit of " +
                                         std::to_string(kNoAllocMaxN));
  if (!dA || lda < n || !d_lambda) return na_fail(EEID_ERR_INVALID, "bad matrix or output pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(EEID_ERR_CUDA, cudaGetErrorString(e));
  double* base = nullptr;
  eeid_status st = scratch_for_device(dev, &base);
  if (st != EEID_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* d = base + kSlotDoubles;
  double* ev = d + kNoAllocMaxN;
  char* meta = (char*)(base + kSlotDoubles + kDEDoubles);
  unsigned* status = d_status_opt ? d_status_opt : (unsigned*)(meta + kOffStatus);

  TridiagTask t;
  t.A = dA;
  t.lda = lda;
  t.n = (int)n;
  t.skip = -1;
  t.rot = -1;
  t.d = d;
  t.e = ev;
  BisectTask b;
  b.d = d;
  b.e = ev;
  b.m = (int)n;
  b.parent = nullptr;
  b.eig = d_lambda;
  const int nitems = (int)((n + kBisectThreads - 1) / kBisectThreads);
  k_noalloc_setup<<<1, 32, 0, s>>>(t, b, nitems, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(EEID_ERR_CUDA, cudaGetErrorString(e));

  TridiagLaunch L;
  L.tasks = (const TridiagTask*)(meta + kOffTask);
  L.ntasks = 1;
  L.counter = (int*)(meta + kOffCounter);
  L.work = base;
  L.work_stride = (int64_t)kSlotDoubles;
  L.max_m = (int)n;
  L.status = status;
  e = launch_tridiag(false, kNoAllocWarps, 1, L, s);
  if (e != cudaSuccess) return na_fail(EEID_ERR_CUDA, cudaGetErrorString(e));
  e = launch_bisect((const BisectTask*)(meta + kOffBisect), (const BisectItem*)(meta + kOffItems),
                    nitems, (int)n, status, s);
  if (e != cudaSuccess) return na_fail(EEID_ERR_CUDA, cudaGetErrorString(e));
  return EEID_OK;
}

}  // extern "C"
