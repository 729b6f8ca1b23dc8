// cur.cu -- the elementwise kernels of CUR image completion (Sec. 5.1):
//   fill    C = Omega . M + (1 - Omega) . X   (data consistency, eq. (update))
//   gather  C_J = C(:, J), R_I = C(I, :), W = C(I, J)  (the CUR factors)
//   filter  X <- G_sigma * X, the 2-D Gaussian spatial regulariser
// on four contiguous row-major planes of m x n.  The pseudoinverses and the
// products of the reconstruction run through the solver and the GEMM kernels
// (solver.cu).  All three kernels are bandwidth-bound grid-stride loops.
#include "common.cuh"

namespace qp {
namespace {

int grid_of(long total) {
  long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// C(q, i, j) = mask(i, j) ? M(q, i, j) : (X ? X(q, i, j) : 0).  C may alias X.
__global__ void k_cur_fill(CurFill f) {
  const long total = (long)f.m * f.n, ps = total;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t / f.n), j = (int)(t % f.n);
    const bool obs = f.mask[(long)i * f.ldk + j] != 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      double v = f.X ? f.X[q * ps + t] : 0.0;
      if (obs) v = f.M[q][(long)i * f.ldm + j];
      f.C[q * ps + t] = v;
    }
  }
}

// C_J (m x r), R_I (r x n) and, when W is given, W (r x r) from C (m x n).
__global__ void k_cur_gather(const double* __restrict__ C, int m, int n, int r, const int* __restrict__ I,
                             const int* __restrict__ J, double* __restrict__ CJ, double* __restrict__ RI,
                             double* __restrict__ W) {
  const long ps = (long)m * n, nc = (long)m * r, nr = (long)r * n, nw = W ? (long)r * r : 0;
  const long total = nc + nr + nw;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    long src;
    double* dst;
    long dps, u;
    if (t < nc) {
      const int i = (int)(t / r), k = (int)(t % r);
      src = (long)i * n + J[k];
      dst = CJ;
      dps = nc;
      u = t;
    } else if (t < nc + nr) {
      u = t - nc;
      const int k = (int)(u / n), j = (int)(u % n);
      src = (long)I[k] * n + j;
      dst = RI;
      dps = nr;
    } else {
      u = t - nc - nr;
      const int k = (int)(u / r), l = (int)(u % r);
      src = (long)I[k] * n + J[l];
      dst = W;
      dps = nw;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) dst[q * dps + u] = C[q * ps + src];
  }
}

// out(q, i, j) = sum_a sum_b g_a g_b in(q, clamp(i + a - R), clamp(j + b - R)),
// offsets a (rows) outer, b (columns) inner; replicated borders.
__global__ void k_cur_gauss(const double* __restrict__ in, double* __restrict__ out, int m, int n, GaussTaps g) {
  const long ps = (long)m * n, total = 4 * ps;
  const int R = g.radius;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int q = (int)(t / ps);
    const long e = t - q * ps;
    const int i = (int)(e / n), j = (int)(e % n);
    const double* p = in + q * ps;
    double acc = 0.0;
    for (int a = 0; a <= 2 * R; a++) {
      const int ii = min(max(i + a - R, 0), m - 1);
      for (int b = 0; b <= 2 * R; b++) {
        const int jj = min(max(j + b - R, 0), n - 1);
        acc += (g.w[a] * g.w[b]) * p[(long)ii * n + jj];
      }
    }
    out[t] = acc;
  }
}

}  // namespace

cudaError_t launch_cur_fill(const CurFill& f, cudaStream_t st) {
  k_cur_fill<<<grid_of((long)f.m * f.n), 256, 0, st>>>(f);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_cur_gather(const double* C, int m, int n, int r, const int* I, const int* J, double* CJ,
                              double* RI, double* W, cudaStream_t st) {
  const long total = (long)m * r + (long)r * n + (W ? (long)r * r : 0);
  k_cur_gather<<<grid_of(total), 256, 0, st>>>(C, m, n, r, I, J, CJ, RI, W);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_cur_gauss(const double* in, double* out, int m, int n, const GaussTaps& g, cudaStream_t st) {
  k_cur_gauss<<<grid_of(4L * m * n), 256, 0, st>>>(in, out, m, n, g);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
