// alpha.cu -- learned initial scaling alpha for X_0 = alpha A^H (Thm. 1).
//
// Features (32 floats, cheap sketches of A computed on the GPU):
//   0 log m, 1 log n, 2 log(||A||_F^2 / theta_1), 3 log ||A||_F,
//   4 log ||A||_1, 5 log ||A||_inf, 6 log theta_1, 7 log(theta_1 / (||A||_1 ||A||_inf)),
//   8..23  theta_i / theta_1, i = 1..16 (Ritz values of A^H A, descending),
//   24..31 log(theta_i / theta_1), i = 2..9 (floored at 1e-30),
// where theta_i come from a 16-step Lanczos run on A^H A (quaternion
// Hermitian, so the Lanczos tridiagonal is real) from a fixed start vector;
// theta_1 estimates sigma_1^2 from below.
//
// Network: x -> tanh(W1 xhat + b1) -> tanh(W2 h1 + b2) -> w3 . h2 + b3 = y,
// xhat = (x - mu) / sd, 32 -> 64 -> 64 -> 1, FP32.  It predicts
// y = log(alpha * theta_1), so alpha = exp(y) / theta_1; the optimum of
// Thm. 1's spectral radius max |1 - alpha sigma_i^2| is
// alpha* = 2 / (sigma_1^2 + sigma_r^2) (sigma_r the smallest nonzero).
// Training: mean squared error, Adam, minibatches; every kernel is this
// file's own (forward, per-sample backward, per-weight gradient sums in a
// fixed order, Adam update).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qp {

constexpr int NF = 32, H = 64;
// weight block layout (floats)
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * NF, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, OFF_MU = OFF_B3 + 1, OFF_SD = OFF_MU + NF,
              NWEIGHTS = OFF_SD + NF;
constexpr int NTRAIN = OFF_MU;  // trainable parameters (mu, sd are fixed per training set)

namespace {

// ------------------------------------------------------------ Lanczos
// y = A x  (A m x n FP32 planes, x n quaternions) -- one warp per row.
__global__ void k_gemv(Planes<const float> A, int m, int n, const float* x, float* y) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= m) return;
  float s[4] = {0, 0, 0, 0};
  for (int j = lane; j < n; j += 32) {
    float a[4], b[4];
    for (int c = 0; c < 4; c++) {
      a[c] = A.p[c * A.ps + (long)row * A.ld + j];
      b[c] = x[4 * j + c];
    }
    s[0] += a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    s[1] += a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    s[2] += a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    s[3] += a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
  }
  for (int c = 0; c < 4; c++)
    for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
  if (lane == 0)
    for (int c = 0; c < 4; c++) y[4 * row + c] = s[c];
}

// z = A^H y  (z_j = sum_i conj(A_ij) y_i): blocks of 32 columns x one row
// chunk (a warp reads 32 consecutive entries of a row) write partial sums per
// (chunk, column); the finishing kernel adds the chunks in order.
constexpr int GV_COLS = 32, GV_ROWS = 8, GV_MAX_CHUNKS = 64;

__global__ void k_gemv_h_part(Planes<const float> A, int m, int n, const float* y, int chunk_rows, float* part) {
  __shared__ float sh[GV_ROWS][4][GV_COLS];
  const int j = blockIdx.x * GV_COLS + threadIdx.x;
  const int r0 = blockIdx.y * chunk_rows, r1 = min(m, r0 + chunk_rows);
  float s[4] = {0, 0, 0, 0};
  if (j < n)
    for (int i = r0 + threadIdx.y; i < r1; i += GV_ROWS) {
      float a[4], b[4];
      for (int c = 0; c < 4; c++) {
        a[c] = A.p[c * A.ps + (long)i * A.ld + j];
        b[c] = y[4 * i + c];
      }
      a[1] = -a[1];
      a[2] = -a[2];
      a[3] = -a[3];
      s[0] += a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
      s[1] += a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
      s[2] += a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
      s[3] += a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    }
  for (int c = 0; c < 4; c++) sh[threadIdx.y][c][threadIdx.x] = s[c];
  __syncthreads();
  if (threadIdx.y == 0 && j < n)
    for (int c = 0; c < 4; c++) {
      float t = s[c];
      for (int r = 1; r < GV_ROWS; r++) t += sh[r][c][threadIdx.x];
      part[((long)blockIdx.y * n + j) * 4 + c] = t;
    }
}

__global__ void k_gemv_h_finish(const float* part, int chunks, int n, float* z) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // t = 4 j + c
  if (t >= 4 * n) return;
  float s = 0.f;
  for (int ch = 0; ch < chunks; ch++) s += part[(long)ch * 4 * n + t];
  z[t] = s;
}

// out[0] = sum a_k b_k over 4n floats (real part of the quaternion inner product).
__global__ void k_dot(const float* a, const float* b, int len, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int t = threadIdx.x; t < len; t += blockDim.x) s += (double)a[t] * b[t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    out[0] = r;
  }
}

// Lanczos scalars stay on the device: alpha_j = dal[0], beta_j^2 = dbe2[0]
// (none for j = 0).  w = w - alpha_j q - beta_j qprev.
__global__ void k_lanczos_axpy(float* w, const float* q, const float* qprev, const double* dal,
                               const double* dbe2, int len) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  const float a = (float)dal[0];
  const float b = dbe2 ? (float)sqrt(fmax(dbe2[0], 0.0)) : 0.f;
  w[t] = w[t] - a * q[t] - b * qprev[t];
}
// qprev = q, q = w / beta (beta^2 = dbe2[0]); a vanishing beta leaves q = 0,
// and the host truncates the run there.
__global__ void k_lanczos_next(const float* w, float* q, float* qprev, const double* dbe2, int len) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= len) return;
  const double b2 = dbe2[0];
  const float inv = b2 > 1e-60 ? (float)(1.0 / sqrt(b2)) : 0.f;
  qprev[t] = q[t];
  q[t] = w[t] * inv;
}
// One power-iteration step: y = M v with v = yprev / ||yprev|| (v = yprev on
// the first step, d2prev null; 0 when the norm vanishes), and d2[0] = ||y||^2.
// One warp per row; each block writes the sum of its rows' squares to
// part[blockIdx.x], and the last block to finish (counted in *count, which it
// resets) adds the block sums in a fixed order, so the result does not
// depend on the blocks' timing.
constexpr int PW_ROWS = 8;
__global__ void __launch_bounds__(32 * PW_ROWS) k_power_step(Planes<const float> M, int s, const float* yprev,
                                                             const double* d2prev, float* y, double* part,
                                                             unsigned int* count, double* d2) {
  __shared__ double wsum[PW_ROWS];
  __shared__ int last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * PW_ROWS + warp;
  float inv = 1.f;
  if (d2prev) {
    const double b2 = d2prev[0];
    inv = b2 > 1e-60 ? (float)(1.0 / sqrt(b2)) : 0.f;
  }
  double rs = 0.0;
  if (row < s) {
    float acc[4] = {0, 0, 0, 0};
    const float* mr = M.p + (long)row * M.ld;
#pragma unroll 4
    for (int j = lane; j < s; j += 32) {
      float a[4], b[4];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        a[c] = mr[c * M.ps + j];
        b[c] = yprev[4 * j + c] * inv;
      }
      acc[0] += a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
      acc[1] += a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
      acc[2] += a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
      acc[3] += a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    }
#pragma unroll
    for (int c = 0; c < 4; c++)
      for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0)
      for (int c = 0; c < 4; c++) {
        y[4 * row + c] = acc[c];
        rs += (double)acc[c] * acc[c];
      }
  }
  if (lane == 0) wsum[warp] = rs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < PW_ROWS; w++) t += wsum[w];
    part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {  // the whole block: strided sums, then a fixed shuffle and warp order
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(part + b);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) wsum[warp] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double r = 0.0;
      for (int w = 0; w < PW_ROWS; w++) r += wsum[w];
      d2[0] = r;
      *count = 0;
    }
  }
}

// ------------------------------------------------------------ MLP kernels
// Forward for B samples (thread per sample); stores activations for backward.
__global__ void k_mlp_fwd(const float* W, const float* X, int B, float* xh, float* h1, float* h2, float* y) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float xs[NF];
  for (int j = 0; j < NF; j++) {
    xs[j] = (X[b * NF + j] - W[OFF_MU + j]) / W[OFF_SD + j];
    xh[b * NF + j] = xs[j];
  }
  float a1[H];
  for (int i = 0; i < H; i++) {
    float s = W[OFF_B1 + i];
    for (int j = 0; j < NF; j++) s += W[OFF_W1 + i * NF + j] * xs[j];
    a1[i] = tanhf(s);
    h1[b * H + i] = a1[i];
  }
  float out = W[OFF_B3];
  for (int i = 0; i < H; i++) {
    float s = W[OFF_B2 + i];
    for (int j = 0; j < H; j++) s += W[OFF_W2 + i * H + j] * a1[j];
    const float a2 = tanhf(s);
    h2[b * H + i] = a2;
    out += W[OFF_W3 + i] * a2;
  }
  y[b] = out;
}

// Per-sample backward of the mean squared error: dy, dz2, dz1.
__global__ void k_mlp_bwd_samples(const float* W, const float* h1, const float* h2, const float* y,
                                  const float* target, int B, float* dy, float* dz2, float* dz1) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float g = 2.f * (y[b] - target[b]) / (float)B;
  dy[b] = g;
  float d2[H];
  for (int i = 0; i < H; i++) {
    const float a2 = h2[b * H + i];
    d2[i] = g * W[OFF_W3 + i] * (1.f - a2 * a2);
    dz2[b * H + i] = d2[i];
  }
  for (int j = 0; j < H; j++) {
    float s = 0.f;
    for (int i = 0; i < H; i++) s += W[OFF_W2 + i * H + j] * d2[i];
    const float a1 = h1[b * H + j];
    dz1[b * H + j] = s * (1.f - a1 * a1);
  }
}

// Gradient of every trainable parameter: one thread per parameter, summing
// over the samples in order (deterministic).
__global__ void k_mlp_grad(const float* xh, const float* h1, const float* h2, const float* dy, const float* dz2,
                           const float* dz1, int B, float* G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NTRAIN) return;
  float s = 0.f;
  if (p < OFF_B1) {
    const int i = p / NF, j = p % NF;
    for (int b = 0; b < B; b++) s += dz1[b * H + i] * xh[b * NF + j];
  } else if (p < OFF_W2) {
    const int i = p - OFF_B1;
    for (int b = 0; b < B; b++) s += dz1[b * H + i];
  } else if (p < OFF_B2) {
    const int q = p - OFF_W2, i = q / H, j = q % H;
    for (int b = 0; b < B; b++) s += dz2[b * H + i] * h1[b * H + j];
  } else if (p < OFF_W3) {
    const int i = p - OFF_B2;
    for (int b = 0; b < B; b++) s += dz2[b * H + i];
  } else if (p < OFF_B3) {
    const int j = p - OFF_W3;
    for (int b = 0; b < B; b++) s += dy[b] * h2[b * H + j];
  } else {
    for (int b = 0; b < B; b++) s += dy[b];
  }
  G[p] = s;
}

__global__ void k_adam(float* W, const float* G, float* M1, float* M2, int t, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NTRAIN) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float g = G[p];
  M1[p] = b1 * M1[p] + (1.f - b1) * g;
  M2[p] = b2 * M2[p] + (1.f - b2) * g * g;
  const float mh = M1[p] / (1.f - powf(b1, (float)t));
  const float vh = M2[p] / (1.f - powf(b2, (float)t));
  W[p] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_sqerr(const float* y, const float* t, int B, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += (double)(y[b] - t[b]) * (y[b] - t[b]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    out[0] = r / B;
  }
}

unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unit(unsigned long long& st) {
  st = mix64(st);
  return (double)(st >> 11) * (1.0 / 9007199254740992.0);
}

// Eigenvalues of a real symmetric k x k matrix (cyclic Jacobi).
std::vector<double> sym_eig(std::vector<double> a, int k) {
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0.0;
    for (int p = 0; p < k; p++)
      for (int q = p + 1; q < k; q++) off += a[p * k + q] * a[p * k + q];
    if (off < 1e-30) break;
    for (int p = 0; p < k; p++)
      for (int q = p + 1; q < k; q++) {
        const double apq = a[p * k + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (a[q * k + q] - a[p * k + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int r = 0; r < k; r++) {
          const double arp = a[r * k + p], arq = a[r * k + q];
          a[r * k + p] = cs * arp - sn * arq;
          a[r * k + q] = sn * arp + cs * arq;
        }
        for (int r = 0; r < k; r++) {
          const double apr = a[p * k + r], aqr = a[q * k + r];
          a[p * k + r] = cs * apr - sn * aqr;
          a[q * k + r] = sn * apr + cs * aqr;
        }
      }
  }
  std::vector<double> ev(k);
  for (int i = 0; i < k; i++) ev[i] = a[i * k + i];
  std::sort(ev.begin(), ev.end(), [](double x, double y) { return x > y; });
  return ev;
}

}  // namespace

int alpha_nweights() { return NWEIGHTS; }
int alpha_ntrain() { return NTRAIN; }

// Features of A (FP32 planes on the device; fro2, n1, ninf precomputed).  The
// scratch buffers hold alpha_feature_scratch_floats(m, n) floats and 2 * 16
// doubles; `pin` is pinned host memory for 2 * 16 doubles.  One host
// synchronisation per call.
int alpha_feature_scratch_floats(int m, int n) { return 4 * (3 * n + m) + 4 * GV_MAX_CHUNKS * n + 64; }

cudaError_t alpha_features(const Planes<const float>& A, int m, int n, double fro2, double norm1, double norminf,
                           float* scratch, double* dscratch, double* pin, cudaStream_t st, float* feat,
                           double* theta1_out) {
  const int K = 16;
  float* q = scratch;
  float* qprev = q + 4 * n;
  float* w = qprev + 4 * n;
  float* y = w + 4 * n;
  float* part = y + 4 * m;
  double* dal = dscratch;
  double* dbe2 = dscratch + K;
  std::vector<float> hq(4 * (size_t)n);
  double nrm = 0.0;
  for (int i = 0; i < 4 * n; i++) {
    hq[i] = (float)(1.0 / (1.0 + 0.37 * (i % 7) + 0.11 * i));
    nrm += (double)hq[i] * hq[i];
  }
  for (int i = 0; i < 4 * n; i++) hq[i] = (float)(hq[i] / std::sqrt(nrm));
  cudaError_t e;
  if ((e = cudaMemcpyAsync(q, hq.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(qprev, 0, sizeof(float) * 4 * n, st)) != cudaSuccess) return e;
  const int len = 4 * n, tb = 256, gb = (len + tb - 1) / tb;
  const int steps = std::min(K, n);
  const int colblocks = (n + GV_COLS - 1) / GV_COLS;
  int ch = (608 + colblocks - 1) / colblocks;
  ch = std::max(1, std::min({ch, (m + 63) / 64, GV_MAX_CHUNKS}));
  const int chunk_rows = (m + ch - 1) / ch;
  for (int j = 0; j < steps; j++) {
    k_gemv<<<(m * 32 + 255) / 256, 256, 0, st>>>(A, m, n, q, y);
    k_gemv_h_part<<<dim3(colblocks, ch), dim3(GV_COLS, GV_ROWS), 0, st>>>(A, m, n, y, chunk_rows, part);
    k_gemv_h_finish<<<gb, tb, 0, st>>>(part, ch, n, w);
    k_dot<<<1, 256, 0, st>>>(q, w, len, dal + j);
    k_lanczos_axpy<<<gb, tb, 0, st>>>(w, q, qprev, dal + j, j > 0 ? dbe2 + j - 1 : nullptr, len);
    k_dot<<<1, 256, 0, st>>>(w, w, len, dbe2 + j);
    if (j + 1 < steps) k_lanczos_next<<<gb, tb, 0, st>>>(w, q, qprev, dbe2 + j, len);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(pin, dscratch, sizeof(double) * 2 * K, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  std::vector<double> al, be;
  for (int j = 0; j < steps; j++) {
    al.push_back(pin[j]);
    if (j + 1 < steps) {
      const double beta = std::sqrt(std::max(pin[K + j], 0.0));
      if (!(beta > 1e-30 * std::max(1.0, std::fabs(pin[j])))) break;  // invariant subspace found
      be.push_back(beta);
    }
  }
  const int k = (int)al.size();
  std::vector<double> T((size_t)k * k, 0.0);
  for (int i = 0; i < k; i++) {
    T[i * k + i] = al[i];
    if (i + 1 < k) T[i * k + i + 1] = T[(i + 1) * k + i] = be[i];
  }
  std::vector<double> th = sym_eig(T, k);
  const double t1 = std::max(th[0], 1e-300);
  *theta1_out = t1;
  auto lg = [](double x) { return (float)std::log(std::max(x, 1e-300)); };
  feat[0] = lg(m);
  feat[1] = lg(n);
  feat[2] = lg(fro2 / t1);
  feat[3] = 0.5f * lg(fro2);
  feat[4] = lg(norm1);
  feat[5] = lg(norminf);
  feat[6] = lg(t1);
  feat[7] = lg(t1 / (norm1 * norminf));
  for (int i = 0; i < 16; i++) feat[8 + i] = i < k ? (float)std::max(th[i] / t1, 0.0) : 0.f;
  for (int i = 0; i < 8; i++) feat[24 + i] = i + 1 < k ? lg(std::max(th[i + 1] / t1, 1e-30)) : lg(1e-30);
  return cudaSuccess;
}

int power_radius_doubles(int s, int steps) { return steps + (s + PW_ROWS - 1) / PW_ROWS + 1; }

// Spectral radius of a square quaternion matrix M (FP32 planes, s x s) by
// power iteration v <- M v / ||M v|| from the features' start vector: the
// geometric mean of the last four norms ||M v_k|| (a complex-conjugate
// dominant pair makes single norms oscillate).  Scratch: 8 s floats and
// power_radius_doubles(s, steps) doubles; one launch per step, one host
// synchronisation.
cudaError_t power_radius(const Planes<const float>& M, int s, int steps, float* scratch, double* dscratch,
                         double* pin, cudaStream_t st, double* rho) {
  float* v = scratch;
  float* y = v + 4 * s;
  const int blocks = (s + PW_ROWS - 1) / PW_ROWS;
  double* part = dscratch + steps;
  unsigned int* count = reinterpret_cast<unsigned int*>(part + blocks);
  std::vector<float> hv(4 * (size_t)s);
  double nrm = 0.0;
  for (int i = 0; i < 4 * s; i++) {
    hv[i] = (float)(1.0 / (1.0 + 0.37 * (i % 7) + 0.11 * i));
    nrm += (double)hv[i] * hv[i];
  }
  for (int i = 0; i < 4 * s; i++) hv[i] = (float)(hv[i] / std::sqrt(nrm));
  cudaError_t e;
  if ((e = cudaMemcpyAsync(v, hv.data(), sizeof(float) * 4 * s, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
  float* buf2[2] = {v, y};
  for (int k = 0; k < steps; k++)
    k_power_step<<<blocks, 32 * PW_ROWS, 0, st>>>(M, s, buf2[k & 1], k ? dscratch + k - 1 : nullptr,
                                                    buf2[(k + 1) & 1], part, count, dscratch + k);
  g_kernel_launches += steps;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(pin, dscratch, sizeof(double) * steps, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  const int last = std::min(4, steps);
  double lg = 0.0;
  for (int k = steps - last; k < steps; k++) lg += 0.5 * std::log(std::max(pin[k], 1e-300));
  *rho = std::exp(lg / last);
  return cudaSuccess;
}

// Initial weights (uniform Xavier from `seed`), mu = 0, sd = 1.
void alpha_init_weights(float* W, unsigned long long seed) {
  unsigned long long st = seed ^ 0xA5A5A5A5DEADBEEFull;
  auto fill = [&](int off, int cnt, int fan_in, int fan_out) {
    const double r = std::sqrt(6.0 / (fan_in + fan_out));
    for (int t = 0; t < cnt; t++) W[off + t] = (float)((2.0 * unit(st) - 1.0) * r);
  };
  fill(OFF_W1, H * NF, NF, H);
  fill(OFF_W2, H * H, H, H);
  fill(OFF_W3, H, H, 1);
  for (int i = 0; i < H; i++) W[OFF_B1 + i] = W[OFF_B2 + i] = 0.f;
  W[OFF_B3] = 0.f;
  for (int j = 0; j < NF; j++) {
    W[OFF_MU + j] = 0.f;
    W[OFF_SD + j] = 1.f;
  }
}

// Scratch for B samples: xh (B*NF), h1, h2 (B*H), y, dy (B), dz1, dz2 (B*H) floats.
size_t alpha_scratch_floats(int B) { return (size_t)B * (NF + 4 * H + 2); }

cudaError_t alpha_forward(const float* dW, const float* dX, int B, float* scratch, float* dy_out, cudaStream_t st) {
  float* xh = scratch;
  float* h1 = xh + (size_t)B * NF;
  float* h2 = h1 + (size_t)B * H;
  k_mlp_fwd<<<(B + 127) / 128, 128, 0, st>>>(dW, dX, B, xh, h1, h2, dy_out);
  return cudaGetLastError();
}

// Gradient of the mean squared error over B samples into dG (NTRAIN floats); loss into dloss.
cudaError_t alpha_gradient(const float* dW, const float* dX, const float* dT, int B, float* scratch, float* dG,
                           double* dloss, cudaStream_t st) {
  float* xh = scratch;
  float* h1 = xh + (size_t)B * NF;
  float* h2 = h1 + (size_t)B * H;
  float* dz1 = h2 + (size_t)B * H;
  float* dz2 = dz1 + (size_t)B * H;
  float* y = dz2 + (size_t)B * H;
  float* dy = y + B;
  k_mlp_fwd<<<(B + 127) / 128, 128, 0, st>>>(dW, dX, B, xh, h1, h2, y);
  k_sqerr<<<1, 256, 0, st>>>(y, dT, B, dloss);
  k_mlp_bwd_samples<<<(B + 127) / 128, 128, 0, st>>>(dW, h1, h2, y, dT, B, dy, dz2, dz1);
  k_mlp_grad<<<(NTRAIN + 255) / 256, 256, 0, st>>>(xh, h1, h2, dy, dz2, dz1, B, dG);
  return cudaGetLastError();
}

cudaError_t alpha_adam(float* dW, const float* dG, float* dM1, float* dM2, int t, float lr, cudaStream_t st) {
  k_adam<<<(NTRAIN + 255) / 256, 256, 0, st>>>(dW, dG, dM1, dM2, t, lr);
  return cudaGetLastError();
}

}  // namespace qp
