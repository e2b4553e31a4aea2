// Deterministic symmetric test matrices generated on the device (used by the
// autotuner to time kernel variants; the values do not affect the work done).
#include "internal.cuh"

namespace eeid {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014)
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

__global__ void k_fill_symmetric(double* A, int n, int64_t lda, unsigned long long seed) {
  const int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const int r = i > j ? i : j, c = i > j ? j : i;
    const unsigned long long h = mix64(seed ^ ((unsigned long long)r << 32 | (unsigned)c));
    A[(int64_t)i * lda + j] = (double)(h >> 11) * 0x1p-53 - 0.5;  // uniform in [-0.5, 0.5)
  }
}

}  // namespace

cudaError_t launch_fill_symmetric(double* A, int n, int64_t lda, unsigned long long seed,
                                  cudaStream_t s) {
  k_fill_symmetric<<<512, 256, 0, s>>>(A, n, lda, seed);
  return cudaGetLastError();
}

}  // namespace eeid
