// qgemm_f64.cu -- FP64 quaternion GEMM on the CUDA cores.
//
// C = A B with the Hamilton product per scalar (Sec. 2):
//   (a0 + a1 i + a2 j + a3 k)(b0 + b1 i + b2 j + b3 k) =
//     (a0b0 - a1b1 - a2b2 - a3b3) + (a0b1 + a1b0 + a2b3 - a3b2) i
//   + (a0b2 - a1b3 + a2b0 + a3b1) j + (a0b3 + a1b2 - a2b1 + a3b0) k.
// GB300 has a small FP64 pipe (about 1 TFLOP/s for the whole chip), so this
// kernel is bound by FP64 issue at any reasonable tiling: a 32x32-quaternion
// block tile staged in shared memory, 2x2 quaternion outputs per thread.
#include "common.cuh"

namespace qp {
namespace {

constexpr int BM = 32, BN = 32, BK = 16;

__global__ void __launch_bounds__(256) k_qgemm_f64(int M, int K, int N, Planes<const double> A,
                                                   Planes<const double> B, Planes<double> C) {
  __shared__ double sa[4][BK][BM + 1];  // sa[c][k][i]
  __shared__ double sb[4][BK][BN + 1];  // sb[c][k][j]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  double acc[2][2][4];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int c = 0; c < 4; c++) acc[a][b][c] = 0.0;

  for (int k0 = 0; k0 < K; k0 += BK) {
    // A tile: BM x BK per plane = 512 elements per plane; 256 threads x 2.
    for (int t = threadIdx.x; t < BM * BK; t += 256) {
      const int ii = t / BK, kk = t % BK;
      const int gi = i0 + ii, gk = k0 + kk;
      const bool ok = gi < M && gk < K;
#pragma unroll
      for (int c = 0; c < 4; c++) sa[c][kk][ii] = ok ? A.p[c * A.ps + (long)gi * A.ld + gk] : 0.0;
    }
    for (int t = threadIdx.x; t < BK * BN; t += 256) {
      const int kk = t / BN, jj = t % BN;
      const int gk = k0 + kk, gj = j0 + jj;
      const bool ok = gk < K && gj < N;
#pragma unroll
      for (int c = 0; c < 4; c++) sb[c][kk][jj] = ok ? B.p[c * B.ps + (long)gk * B.ld + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; kk++) {
      double a[2][4], b[2][4];
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) a[r][c] = sa[c][kk][ty + 16 * r];
#pragma unroll
      for (int s = 0; s < 2; s++)
#pragma unroll
        for (int c = 0; c < 4; c++) b[s][c] = sb[c][kk][tx + 16 * s];
#pragma unroll
      for (int r = 0; r < 2; r++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
          double* o = acc[r][s];
          const double* p = a[r];
          const double* q = b[s];
          o[0] = fma(p[0], q[0], fma(-p[1], q[1], fma(-p[2], q[2], fma(-p[3], q[3], o[0]))));
          o[1] = fma(p[0], q[1], fma(p[1], q[0], fma(p[2], q[3], fma(-p[3], q[2], o[1]))));
          o[2] = fma(p[0], q[2], fma(-p[1], q[3], fma(p[2], q[0], fma(p[3], q[1], o[2]))));
          o[3] = fma(p[0], q[3], fma(p[1], q[2], fma(-p[2], q[1], fma(p[3], q[0], o[3]))));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 2; r++)
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * s;
      if (gi < M && gj < N)
#pragma unroll
        for (int c = 0; c < 4; c++) C.p[c * C.ps + (long)gi * C.ld + gj] = acc[r][s][c];
    }
}

}  // namespace

cudaError_t launch_qgemm_f64(int M, int K, int N, const Planes<const double>& A, const Planes<const double>& B,
                             const Planes<double>& C, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  k_qgemm_f64<<<grid, 256, 0, st>>>(M, K, N, A, B, C);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
