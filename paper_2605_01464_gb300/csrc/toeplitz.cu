// toeplitz.cu -- the data matrix of quaternion signal filtering (Sec. 5.2):
// X(i, j) = x(t0 + i - j), i, j = 0..p, from four planes of N samples, so
// that s(t) ~ sum_m x(t - m) h_m reads X h = s.  One coalesced write per
// entry; the samples come from cache (every sample appears on a diagonal).
#include "common.cuh"

namespace qp {
namespace {

__global__ void k_toeplitz(const double* __restrict__ x, long xps, int p, int t0, double* __restrict__ X) {
  const long n = p + 1, ps = n * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < ps; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    const long k = (long)t0 + i - j;
#pragma unroll
    for (int q = 0; q < 4; q++) X[q * ps + t] = x[q * xps + k];
  }
}

}  // namespace

cudaError_t launch_toeplitz(const double* x, long xps, int p, int t0, double* X, cudaStream_t st) {
  const long total = (long)(p + 1) * (p + 1);
  long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  k_toeplitz<<<(int)blocks, 256, 0, st>>>(x, xps, p, t0, X);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
