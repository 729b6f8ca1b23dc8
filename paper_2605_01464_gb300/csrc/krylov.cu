// krylov.cu -- vector kernels of the global quaternion Krylov solvers
// (Gl-QGMRES / Gl-QFOM, Sec. 3.5).  A block is an n x m quaternion matrix
// stored as L = 4 n m contiguous doubles (four planes); the global inner
// product <V, W> = Re tr(V^H W) is the plain dot product of those arrays.
// The basis V_0, V_1, ... is one array of blocks with stride L.  Reductions
// are deterministic (fixed block shapes, tree sums in shared memory).
#include "common.cuh"

namespace qp {
namespace {

constexpr int KT = 256;

__device__ double block_reduce(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// h[i] = <V_i, W>, i < c: block i reduces over the L elements.
__global__ void __launch_bounds__(KT) k_block_dot(const double* __restrict__ V, int c, const double* __restrict__ W,
                                                   long L, double* __restrict__ h) {
  __shared__ double sh[KT / 32];
  const double* v = V + (long)blockIdx.x * L;
  double s = 0.0;
  for (long e = threadIdx.x; e < L; e += KT) s += v[e] * W[e];
  s = block_reduce(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// W += sign * sum_{i<c} h[i] V_i.  A block takes 32 consecutive elements
// (one per lane, coalesced across the basis), its warps split the basis
// index i, and the warps' partial sums are added in a fixed order.  Block 0
// also adds h into the Hessenberg column when hcol is given.
constexpr int kCombWarps = 16;
__global__ void __launch_bounds__(32 * kCombWarps) k_block_combine(double* __restrict__ W, const double* __restrict__ V,
                                                                   const double* __restrict__ h, int c, long L,
                                                                   double sign, double* __restrict__ hcol) {
  __shared__ double part[kCombWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long e = (long)blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < L)
    for (int i = w; i < c; i += kCombWarps) s += h[i] * V[(long)i * L + e];
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && e < L) {
    double t = 0.0;
    for (int q = 0; q < kCombWarps; q++) t += part[q][lane];
    W[e] += sign * t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && hcol)
    for (int i = 0; i < c; i++) hcol[i] += h[i];
}

// nrm = ||W||; out = W / nrm (out may alias W; left unscaled when nrm = 0).
// One block: the blocks of these solvers are small (L = 4 n m).
__global__ void __launch_bounds__(1024) k_norm_scale(const double* W, long L, double* __restrict__ nrm, double* out) {
  __shared__ double sh[32];
  __shared__ double tot;
  double s = 0.0;
  for (long e = threadIdx.x; e < L; e += blockDim.x) s += W[e] * W[e];
  s = block_reduce(s, sh);
  if (threadIdx.x == 0) {
    tot = sqrt(s);
    *nrm = tot;
  }
  __syncthreads();
  const double t = tot;
  if (out && t > 0.0)
    for (long e = threadIdx.x; e < L; e += blockDim.x) out[e] = W[e] / t;
}

// out = a - b
__global__ void k_sub(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b, long L) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < L; e += (long)gridDim.x * blockDim.x)
    out[e] = a[e] - b[e];
}

// C = A B for a skinny right-hand side (m <= kSkinnyMax columns): block i
// computes row i of C; its threads stride over k, accumulate the Hamilton
// products for every column, and reduce across the block.  The general GEMM
// kernels tile 64 x 64 outputs and leave almost every SM idle at m <= 16.
constexpr int kSkinnyMax = 16;
__global__ void __launch_bounds__(128) k_qgemm_skinny(Planes<const double> A, Planes<const double> B, int K, int m,
                                                      Planes<double> C) {
  __shared__ double sh[4 * kSkinnyMax][4];
  const int i = blockIdx.x;
  double acc[4 * kSkinnyMax];
#pragma unroll
  for (int t = 0; t < 4 * kSkinnyMax; t++) acc[t] = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const long ai = (long)i * A.ld + k;
    const double as = A.p[ai], ax = A.p[A.ps + ai], ay = A.p[2 * A.ps + ai], az = A.p[3 * A.ps + ai];
#pragma unroll
    for (int l = 0; l < kSkinnyMax; l++) {
      if (l < m) {
        const long bi = (long)k * B.ld + l;
        const double bs = B.p[bi], bx = B.p[B.ps + bi], by = B.p[2 * B.ps + bi], bz = B.p[3 * B.ps + bi];
        acc[4 * l + 0] += as * bs - ax * bx - ay * by - az * bz;
        acc[4 * l + 1] += as * bx + ax * bs + ay * bz - az * by;
        acc[4 * l + 2] += as * by - ax * bz + ay * bs + az * bx;
        acc[4 * l + 3] += as * bz + ax * by - ay * bx + az * bs;
      }
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < 4 * kSkinnyMax; t++) {
    if (t < 4 * m) {
      double v = acc[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sh[t][w] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 * m) {
    const int t = threadIdx.x, l = t >> 2, q = t & 3;
    C.p[q * C.ps + (long)i * C.ld + l] = sh[t][0] + sh[t][1] + sh[t][2] + sh[t][3];
  }
}

// Givens step j of the GMRES / FOM least-squares update, on the device so
// that the host need not read every Hessenberg column: applies the rotations
// of steps 0..j-1 to column j (in place; h_{j+1,j} = col[j+1] is kept), forms
// rotation j, updates g, and writes the residual estimate |g_{j+1}| (GMRES)
// or |g_{j+1}| / |c_j| (FOM).  Sequential by nature: one thread.
__global__ void k_givens(double* __restrict__ col, double* __restrict__ cs, double* __restrict__ sn,
                         double* __restrict__ g, int j, int fom, double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  // the running entry stays in a register: every load is of an entry not yet
  // written, so the loads pipeline and only the rotation chain is serial
  double a = col[0];
  for (int i = 0; i < j; i++) {
    const double b = col[i + 1], c = cs[i], s = sn[i];
    col[i] = c * a + s * b;
    a = -s * a + c * b;
  }
  const double b = col[j + 1];
  const double rho = hypot(a, b);
  const double c = rho > 0.0 ? a / rho : 1.0, s = rho > 0.0 ? b / rho : 0.0;
  cs[j] = c;
  sn[j] = s;
  const double gp = g[j];
  g[j + 1] = -s * gp;
  g[j] = c * gp;
  col[j] = rho;
  res[j] = fom ? (c != 0.0 ? fabs(g[j + 1]) / fabs(c) : INFINITY) : fabs(g[j + 1]);
}

int grid_of(long L) {
  long b = (L + KT - 1) / KT;
  return (int)(b < 1 ? 1 : b > 4096 ? 4096 : b);
}

}  // namespace

bool skinny_ok(int m) { return m >= 1 && m <= kSkinnyMax; }

cudaError_t launch_qgemm_skinny(int M, int K, int m, const Planes<const double>& A, const Planes<const double>& B,
                                const Planes<double>& C, cudaStream_t st) {
  k_qgemm_skinny<<<M, 128, 0, st>>>(A, B, K, m, C);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_givens(double* col, double* cs, double* sn, double* g, int j, int fom, double* res,
                          cudaStream_t st) {
  k_givens<<<1, 32, 0, st>>>(col, cs, sn, g, j, fom, res);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_block_dot(const double* V, int c, const double* W, long L, double* h, cudaStream_t st) {
  k_block_dot<<<c, KT, 0, st>>>(V, c, W, L, h);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_block_sub(double* W, const double* V, const double* h, int c, long L, double* hcol,
                             cudaStream_t st) {
  k_block_combine<<<(int)((L + 31) / 32), 32 * kCombWarps, 0, st>>>(W, V, h, c, L, -1.0, hcol);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_norm_scale(const double* W, long L, double* nrm, double* out, cudaStream_t st) {
  k_norm_scale<<<1, 1024, 0, st>>>(W, L, nrm, out);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_basis_add(double* X, const double* V, const double* y, int k, long L, cudaStream_t st) {
  k_block_combine<<<(int)((L + 31) / 32), 32 * kCombWarps, 0, st>>>(X, V, y, k, L, 1.0, nullptr);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_sub(double* out, const double* a, const double* b, long L, cudaStream_t st) {
  k_sub<<<grid_of(L), KT, 0, st>>>(out, a, b, L);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
