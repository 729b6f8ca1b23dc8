// batched_impl.cuh -- qpinv_solve_batched: thousands of small quaternion
// pseudoinverses (m, n <= 256) in ONE persistent kernel launch.
//
// Compiled six times: batched.cu includes it for the host side (no kernel
// instantiated), and batched_tile<t>.cu (t = 0..4) each define
// QP_BATCHED_TILE and instantiate the kernel for one CTA tile shape, so the
// five heavy instantiations compile in parallel.
//
// Every CTA takes matrices from an atomic work counter (largest cost first)
// and solves each one end to end -- alpha, X_0 = alpha A^H, the method's
// iteration with its stop rule, E1..E4 -- with CTA-level quaternion GEMMs on
// a workspace slot of its own in global memory (the working set of one
// 256 x 256 problem, ~40 MB per slot, streams through L2).
//
// Arithmetic: double-FP32 ("df": a value is an unevaluated sum hi + lo of two
// floats, ~2^-46 relative accuracy).  Small blocks such as CUR intersection
// matrices are typically rank deficient, and rounding noise that lands in
// null(A) is multiplied by the method's order every iteration -- about
// kappa_eff^2 over a solve -- so FP32 alone cannot serve them; GB300's FP64
// pipe is too small to, while df products run on the FP32 pipe: each real
// multiply-add is an exact product split (FMA) plus a compensated add.
//
// The iteration schedules are the small-correction forms of the single-matrix
// solver (X_{j+1} = X + X t with t built from R, R^2, R^4), residual on the
// smaller side.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/qpinv.h"
#include "common.cuh"

namespace qp {
namespace {

constexpr int MAXD = 256;
constexpr int NBUF = 22;  // workspace matrices per slot
constexpr int TPB = 256;      // threads of the CUDA-core engine's CTA
constexpr int TPB_MAX = 352;  // largest CTA of any engine (the per-matrix code uses blockDim.x)
// CTA GEMM: a 16 x 16 thread grid, each thread RM x RN outputs 16 apart, so
// the CTA tile is 16 RM x 16 RN quaternion entries; BK = K step.  The tile
// shape is a template parameter of the kernel, chosen per batch by the
// autotuner in qpinv_solve_batched (or fixed by the caller).
constexpr int BK = 8;
constexpr int TMAX = 64;  // largest tile side

}  // namespace

// ------------------------------------------------------------ df arithmetic
struct dfv {
  float hi, lo;
};

namespace {
__device__ __forceinline__ dfv df_quick(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfv df_add(dfv a, dfv b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = (a.hi - (s - v)) + (b.hi - v);
  return df_quick(s, e + a.lo + b.lo);
}
__device__ __forceinline__ dfv df_neg(dfv a) { return {-a.hi, -a.lo}; }
// c + a * b (product split exactly with FMA, then a compensated add)
__device__ __forceinline__ dfv df_fma(dfv a, dfv b, dfv c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = c.hi + p;
  const float v = s - c.hi;
  const float t = (c.hi - (s - v)) + (p - v);
  return df_quick(s, t + e + c.lo);
}
__device__ __forceinline__ dfv df_mul(dfv a, dfv b) { return df_fma(a, b, dfv{0.f, 0.f}); }
// Lazy accumulation for dot products (compensated summation in the manner of
// Ogita, Rump and Oishi's Dot2, with df inputs): acc.hi is the running sum,
// acc.lo collects the rounding and low-order terms of a few products
// unnormalised; df_norm turns it back into a df value.
__device__ __forceinline__ void df_dot_add(dfv& acc, dfv a, dfv b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = acc.hi + p;
  const float v = s - acc.hi;
  acc.lo += ((acc.hi - (s - v)) + (p - v)) + e;
  acc.hi = s;
}
// Renormalisation by a full two-sum: exact whichever part is larger (after
// cancellation in the running sum the low part can exceed the high part).
__device__ __forceinline__ dfv df_norm(dfv a) {
  const float s = a.hi + a.lo;
  const float v = s - a.hi;
  return dfv{s, (a.hi - (s - v)) + (a.lo - v)};
}
__device__ __forceinline__ dfv df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to(dfv a) { return (double)a.hi + (double)a.lo; }

// A workspace matrix: 4 planes rows x cols of df values, compact.
struct DM {
  dfv* p;
  int rows, cols;
  __device__ long ps() const { return (long)rows * cols; }
  __device__ dfv& at(int c, int i, int j) const { return p[c * ps() + (long)i * cols + j]; }
};

struct Coef {
  dfv v;
};

// Output of a fused CTA GEMM pass: out = ca * (P Q) + sum_t ct * aux_t + diag * I,
// and up to two more outputs formed from it: xo_k = out + sum_t cx_k,t * aux_t
// (the polynomial blocks that would otherwise take their own elementwise
// passes).  A zero coefficient skips its term.
struct Epi {
  dfv ca = {1.f, 0.f};
  const DM* aux[3] = {nullptr, nullptr, nullptr};
  dfv ct[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  dfv diag = {0.f, 0.f};
  const DM* ref = nullptr;  // if set: accumulate ||out - ref||^2 and ||out||^2
  int nx = 0;
  const DM* xo[2] = {nullptr, nullptr};
  dfv cx[2][3] = {{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}};
};
__device__ __forceinline__ bool df_nonzero(dfv x) { return x.hi != 0.f || x.lo != 0.f; }

// The pass's epilogue for one entry (i, j) of component c (tensor-core
// engine): v = ca acc + sum ct aux + diag, stored to C, and the extra
// outputs; av are the aux
// values at (c, i, j) (loaded before any store: an output may alias an aux
// plane at this entry only).  Returns v.
__device__ __forceinline__ dfv epi_entry(const Epi& e, dfv acc, const dfv* av, int c, int i, int j, const DM& C) {
  dfv v = df_mul(e.ca, acc);
#pragma unroll
  for (int t = 0; t < 3; t++)
    if (e.aux[t] && df_nonzero(e.ct[t])) v = df_fma(e.ct[t], av[t], v);
  if (c == 0 && i == j) v = df_add(v, e.diag);
  for (int k = 0; k < e.nx; k++) {
    dfv w = v;
#pragma unroll
    for (int t = 0; t < 3; t++)
      if (e.aux[t] && df_nonzero(e.cx[k][t])) w = df_fma(e.cx[k][t], av[t], w);
    e.xo[k]->at(c, i, j) = w;
  }
  C.at(c, i, j) = v;
  return v;
}

}  // namespace

// Types shared by the host side and the per-tile translation units.
struct BatchItem {
  const double* A[4];
  double* X[4];
  long lda, ldx;
  int m, n;
};

struct BatchResult {
  int status, iters, side, gemms;
  double alpha, delta, delta_rel;
  double E[4], E_rel[4];
};

struct BatchParams {
  const BatchItem* items;
  const int* order;
  int count;
  int* counter;
  BatchResult* results;
  dfv* ws;
  long slot_elems;
  int method, mparam, stop_rule, max_iter, alpha_mode;  // mparam: QRAPID's N or QHPIM's order k
  double tol, alpha_user;
  double k[12];  // QHPI19 coefficients a1 a2 a3 b1 b2 c1 c2 d1 d2 d3 e1 e2
  // tensor-core engine (batched_tc.cu): per-slot slice scratch and its TMA maps
  const CUtensorMap* tc_maps;  // 2 per slot: A-form slices, B-form slices
  char* tc_ws;
  long tc_slot_bytes;
  int tc_slices;  // exact 7-bit slices per operand
  int* err;       // device error word (bounded-wait expiry)
};

// Per-tile entry points, defined in batched_tile<t>.cu.
cudaError_t batched_launch_t0(int slots, const BatchParams& P, cudaStream_t st);
cudaError_t batched_launch_t1(int slots, const BatchParams& P, cudaStream_t st);
cudaError_t batched_launch_t2(int slots, const BatchParams& P, cudaStream_t st);
cudaError_t batched_launch_t3(int slots, const BatchParams& P, cudaStream_t st);
cudaError_t batched_launch_t4(int slots, const BatchParams& P, cudaStream_t st);
cudaError_t batched_launch_tc(int slots, const BatchParams& P, cudaStream_t st);
int batched_occupancy_t0();
int batched_occupancy_t1();
int batched_occupancy_t2();
int batched_occupancy_t3();
int batched_occupancy_t4();
size_t batched_tc_slot_bytes();
cudaError_t batched_tc_maps(char* tc_ws, int slots, CUtensorMap* host_maps, void* dev_maps, cudaStream_t st);

namespace {

struct Shared {
  double red[TPB_MAX / 32][2];
  double bc[4];
};
// operand tiles of the CUDA-core CTA GEMM
struct SimtTiles {
  dfv a[4][BK][TMAX];
  dfv b[4][BK][TMAX];
};

__device__ double block_sum(double v, Shared& sh, int slot) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5][slot] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh.red[w][slot];
  __syncthreads();
  return r;  // valid in every thread
}

// C (P.rows x Q.cols) = epilogue(P Q), quaternion; every thread of the CTA calls it.
// Returns (in every thread) the two norms of Epi::ref, if requested.
template <int RM, int RN>
__device__ __noinline__ void cta_gemm(const DM& P, const DM& Q, const DM& C, const Epi& e, Shared& sh, SimtTiles& tl,
                         double* norms) {
  constexpr int BM = 16 * RM, BN = 16 * RN;
  const int M = P.rows, K = P.cols, N = Q.cols;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float nd = 0.f, nx = 0.f;
  for (int i0 = 0; i0 < M; i0 += BM) {
    for (int j0 = 0; j0 < N; j0 += BN) {
      dfv acc[RM][RN][4];
#pragma unroll
      for (int a = 0; a < RM; a++)
#pragma unroll
        for (int b = 0; b < RN; b++)
#pragma unroll
          for (int c = 0; c < 4; c++) acc[a][b][c] = dfv{0.f, 0.f};
      for (int k0 = 0; k0 < K; k0 += BK) {
        for (int t = threadIdx.x; t < BM * BK; t += TPB) {
          const int ii = t / BK, kk = t % BK, gi = i0 + ii, gk = k0 + kk;
          const bool ok = gi < M && gk < K;
#pragma unroll
          for (int c = 0; c < 4; c++) tl.a[c][kk][ii] = ok ? P.at(c, gi, gk) : dfv{0.f, 0.f};
        }
        for (int t = threadIdx.x; t < BK * BN; t += TPB) {
          const int kk = t / BN, jj = t % BN, gk = k0 + kk, gj = j0 + jj;
          const bool ok = gk < K && gj < N;
#pragma unroll
          for (int c = 0; c < 4; c++) tl.b[c][kk][jj] = ok ? Q.at(c, gk, gj) : dfv{0.f, 0.f};
        }
        __syncthreads();
        const int kmax = min(BK, K - k0);
        for (int kk = 0; kk < kmax; kk++) {
          dfv a[RM][4], b[RN][4];
#pragma unroll
          for (int r = 0; r < RM; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) a[r][c] = tl.a[c][kk][ty + 16 * r];
#pragma unroll
          for (int q = 0; q < RN; q++)
#pragma unroll
            for (int c = 0; c < 4; c++) b[q][c] = tl.b[c][kk][tx + 16 * q];
#pragma unroll
          for (int r = 0; r < RM; r++)
#pragma unroll
            for (int q = 0; q < RN; q++) {
              dfv* o = acc[r][q];
              const dfv* x = a[r];
              const dfv* y = b[q];
              // Hamilton product x y (Sec. 2), accumulated per component
              df_dot_add(o[0], x[0], y[0]);
              df_dot_add(o[0], df_neg(x[1]), y[1]);
              df_dot_add(o[0], df_neg(x[2]), y[2]);
              df_dot_add(o[0], df_neg(x[3]), y[3]);
              df_dot_add(o[1], x[0], y[1]);
              df_dot_add(o[1], x[1], y[0]);
              df_dot_add(o[1], x[2], y[3]);
              df_dot_add(o[1], df_neg(x[3]), y[2]);
              df_dot_add(o[2], x[0], y[2]);
              df_dot_add(o[2], df_neg(x[1]), y[3]);
              df_dot_add(o[2], x[2], y[0]);
              df_dot_add(o[2], x[3], y[1]);
              df_dot_add(o[3], x[0], y[3]);
              df_dot_add(o[3], x[1], y[2]);
              df_dot_add(o[3], df_neg(x[2]), y[1]);
              df_dot_add(o[3], x[3], y[0]);
              // renormalise after every quaternion term (four real terms): the
              // unnormalised low part must stay near u |hi|, or its own
              // rounding grows with the square of the dot-product length (a
              // fast two-sum; its rare inexact case under cancellation costs
              // O(u^2) of the partial sums, the df level)
#pragma unroll
              for (int c = 0; c < 4; c++) o[c] = df_quick(o[c].hi, o[c].lo);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < RM; r++)
#pragma unroll
        for (int q = 0; q < RN; q++) {
          const int gi = i0 + ty + 16 * r, gj = j0 + tx + 16 * q;
          if (gi < M && gj < N) {
            for (int c = 0; c < 4; c++) {
              dfv v = df_mul(e.ca, df_norm(acc[r][q][c]));
              for (int t = 0; t < 3; t++)
                if (e.aux[t] && df_nonzero(e.ct[t])) v = df_fma(e.ct[t], e.aux[t]->at(c, gi, gj), v);
              if (c == 0 && gi == gj) v = df_add(v, e.diag);
              if (e.ref) {
                const dfv d = df_add(v, df_neg(e.ref->at(c, gi, gj)));
                nd += d.hi * d.hi;
                nx += v.hi * v.hi;
              }
              C.at(c, gi, gj) = v;
            }
          }
        }
    }
  }
  if (e.nx) {
    // the extra outputs from the finished main output (one pass: their
    // code stays out of the register-tile epilogue above)
    __syncthreads();
    for (long t = threadIdx.x; t < (long)M * N; t += blockDim.x) {
      const int i = (int)(t / N), j = (int)(t % N);
      for (int c = 0; c < 4; c++) {
        const dfv v = C.at(c, i, j);
        for (int k = 0; k < e.nx; k++) {
          dfv w = v;
          for (int u = 0; u < 3; u++)
            if (e.aux[u] && df_nonzero(e.cx[k][u])) w = df_fma(e.cx[k][u], e.aux[u]->at(c, i, j), w);
          e.xo[k]->at(c, i, j) = w;
        }
      }
    }
  }
  if (e.ref) {
    norms[0] = block_sum((double)nd, sh, 0);
    norms[1] = block_sum((double)nx, sh, 1);
  } else {
    __syncthreads();
  }
}

// out = ca * X + sum ct * aux + diag I  (elementwise; no product).
__device__ void cta_axpy(const DM& X, const DM& out, dfv ca, const DM* aux, dfv ct, dfv diag) {
  const long total = (long)X.rows * X.cols;
  for (long t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = (int)(t / X.cols), j = (int)(t % X.cols);
    for (int c = 0; c < 4; c++) {
      dfv v = df_mul(ca, X.at(c, i, j));
      if (aux) v = df_fma(ct, aux->at(c, i, j), v);
      if (c == 0 && i == j) v = df_add(v, diag);
      out.at(c, i, j) = v;
    }
  }
  __syncthreads();
}

// ||M^H - M||_F^2 for square M.
__device__ double cta_antiherm2(const DM& M, Shared& sh) {
  float s = 0.f;
  const long total = (long)M.rows * M.cols;
  for (long t = threadIdx.x; t < total; t += blockDim.x) {
    const int i = (int)(t / M.cols), j = (int)(t % M.cols);
    for (int c = 0; c < 4; c++) {
      const dfv mji = M.at(c, j, i), mij = M.at(c, i, j);
      const dfv d = df_add(c == 0 ? mji : df_neg(mji), df_neg(mij));
      s += d.hi * d.hi;
    }
  }
  return block_sum((double)s, sh, 0);
}

__device__ double cta_fro2(const DM& M, Shared& sh) {
  float s = 0.f;
  const long total = 4L * M.rows * M.cols;
  for (long t = threadIdx.x; t < total; t += blockDim.x) s += M.p[t].hi * M.p[t].hi;
  return block_sum((double)s, sh, 0);
}

__device__ __forceinline__ dfv dc(double x) { return df_from(x); }

// ---------------------------------------------------------------- one solve
struct Ctx {
  const BatchParams* P;
  Shared* sh;
  dfv* base;
  int m, n, s;
  bool left;
  int gemms;
  __device__ DM buf(int idx, int rows, int cols) const {
    DM d;
    d.p = base + (long)idx * 4 * MAXD * MAXD;
    d.rows = rows;
    d.cols = cols;
    return d;
  }
};

enum { B_A = 0, B_X0, B_X1, B_R, B_R2, B_R4, B_S, B_FA, B_FB, B_U, B_V, B_W, B_G, B_T, B_Z0, B_Z1, B_Z2, B_E, B_P1,
       B_P2, B_P3, B_P4 };

// The CUDA-core CTA GEMM as a policy of Solve (the tensor-core engine in
// batched_tc.cu provides another with the same call).
template <int RM, int RN>
struct SimtGemm {
  Shared* sh;
  SimtTiles* tl;
  __device__ void operator()(const DM& P, const DM& Q, const DM& C, const Epi& e, double* norms) {
    cta_gemm<RM, RN>(P, Q, C, e, *sh, *tl, norms);
  }
};

template <class G>
struct Solve {
  Ctx& c;
  G& g;
  DM A, X[2];
  int cur = 0;
  double nd = 0, nx = 0;
  __device__ Solve(Ctx& cc, G& gg) : c(cc), g(gg) {}

  __device__ void gemm(const DM& P, const DM& Q, const DM& C, const Epi& e) {
    c.gemms++;
    double nrm[2] = {0, 0};
    g(P, Q, C, e, nrm);
    if (e.ref) {
      nd = nrm[0];
      nx = nrm[1];
    }
  }
  // residual product of Y: right A Y (m x m), left Y A (n x n); R = I - that
  __device__ void residual(const DM& Y, const DM& R) {
    Epi e;
    e.ca = dc(-1.0);
    e.diag = dc(1.0);
    if (c.left) gemm(Y, A, R, e);
    else gemm(A, Y, R, e);
  }
  // out = base + (Y T | T Y), with the stop norms against X[cur] when final
  __device__ void apply(const DM& Y, const DM& T, const DM& base, const DM& out, bool final_update) {
    Epi e;
    e.aux[0] = &base;
    e.ct[0] = dc(1.0);
    if (final_update) e.ref = &X[cur];
    if (c.left) gemm(T, Y, out, e);
    else gemm(Y, T, out, e);
  }

  __device__ void step_ns() {
    const DM R = c.buf(B_R, c.s, c.s);
    residual(X[cur], R);
    apply(X[cur], R, X[cur], X[cur ^ 1], true);
  }

  __device__ void step_qsai() {
    const double b1 = 0.5 * (1.0 + sqrt(5.0)), b2 = 0.5 * (1.0 - sqrt(5.0));
    const int s = c.s;
    const DM R = c.buf(B_R, s, s), R2 = c.buf(B_R2, s, s), R4 = c.buf(B_R4, s, s);
    const DM Fa = c.buf(B_FA, s, s), Fb = c.buf(B_FB, s, s), q = c.buf(B_U, s, s), t = c.buf(B_T, s, s);
    residual(X[cur], R);
    gemm(R, R, R2, Epi());
    {
      Epi e;  // R4 = R2 R2, with Fa = R4 + b1 R2 and Fb = R4 + b2 R2
      e.aux[0] = &R2;
      e.nx = 2;
      e.xo[0] = &Fa;
      e.cx[0][0] = dc(b1);
      e.xo[1] = &Fb;
      e.cx[1][0] = dc(b2);
      gemm(R2, R2, R4, e);
    }
    {
      Epi e;  // q = Fa Fb + (b1 + b2) R2 + 2 R4
      e.aux[0] = &R2;
      e.ct[0] = dc(b1 + b2);
      e.aux[1] = &R4;
      e.ct[1] = dc(2.0);
      gemm(Fa, Fb, q, e);
    }
    {
      Epi e;  // t = R q + R + q
      e.aux[0] = &R;
      e.ct[0] = dc(1.0);
      e.aux[1] = &q;
      e.ct[1] = dc(1.0);
      gemm(R, q, t, e);
    }
    apply(X[cur], t, X[cur], X[cur ^ 1], true);
  }

  __device__ void step_qhpi19() {
    const double* k = c.P->k;
    const double c1 = k[5], c2 = k[6], d1 = k[7], d2 = k[8], d3 = k[9], e1 = k[10], e2 = k[11];
    const int s = c.s;
    const DM R = c.buf(B_R, s, s), R2 = c.buf(B_R2, s, s), R4 = c.buf(B_R4, s, s), S = c.buf(B_S, s, s);
    const DM Fa = c.buf(B_FA, s, s), Fb = c.buf(B_FB, s, s), u = c.buf(B_U, s, s), v = c.buf(B_V, s, s);
    const DM w = c.buf(B_W, s, s), g = c.buf(B_G, s, s), t = c.buf(B_T, s, s);
    residual(X[cur], R);
    {
      Epi e;  // R2 = R R, with S = R2 + R
      e.aux[0] = &R;
      e.nx = 1;
      e.xo[0] = &S;
      e.cx[0][0] = dc(1.0);
      gemm(R, R, R2, e);
    }
    {
      Epi e;  // R4 = R2 R2, with Fa = R4 + d1 R2 and Fb = R4 + d2 R2
      e.aux[0] = &R2;
      e.nx = 2;
      e.xo[0] = &Fa;
      e.cx[0][0] = dc(d1);
      e.xo[1] = &Fb;
      e.cx[1][0] = dc(d2);
      gemm(R2, R2, R4, e);
    }
    {
      // u = Fa Fb + (d1 + d2) R2 + 2 R4, with v = u + d3 R2 and
      // w = u + e1 R2 + e2 R4
      Epi e;
      e.aux[0] = &R2;
      e.ct[0] = dc(d1 + d2);
      e.aux[1] = &R4;
      e.ct[1] = dc(2.0);
      e.nx = 2;
      e.xo[0] = &v;
      e.cx[0][0] = dc(d3);
      e.xo[1] = &w;
      e.cx[1][0] = dc(e1);
      e.cx[1][1] = dc(e2);
      gemm(Fa, Fb, u, e);
    }
    {
      Epi e;  // g = v w + 2 u + (d3 + e1 + c1) R2 + (e2 + c2) R4
      e.aux[0] = &u;
      e.ct[0] = dc(2.0);
      e.aux[1] = &R2;
      e.ct[1] = dc(d3 + e1 + c1);
      e.aux[2] = &R4;
      e.ct[2] = dc(e2 + c2);
      gemm(v, w, g, e);
    }
    {
      Epi e;  // t = S g + S
      e.aux[0] = &S;
      e.ct[0] = dc(1.0);
      gemm(S, g, t, e);
    }
    apply(X[cur], t, X[cur], X[cur ^ 1], true);
  }

  // W + Y (I - A W) (right) / W + (I - W A) Y (left) into Z
  __device__ void rapid_correct(const DM& W, const DM& Y, const DM& Z, bool final_update) {
    const DM E = c.buf(B_E, c.s, c.s);
    residual(W, E);
    apply(Y, E, W, Z, final_update);
  }

  __device__ void step_qrapid() {
    const int s = c.s;
    const DM R = c.buf(B_R, s, s), R2 = c.buf(B_R2, s, s), t = c.buf(B_T, s, s);
    residual(X[cur], R);
    gemm(R, R, R2, Epi());
    {
      Epi e;  // t = R3/4 + R + R2
      e.ca = dc(0.25);
      e.aux[0] = &R;
      e.ct[0] = dc(1.0);
      e.aux[1] = &R2;
      e.ct[1] = dc(1.0);
      gemm(R, R2, t, e);
    }
    DM Z[3] = {c.buf(B_Z0, c.n, c.m), c.buf(B_Z1, c.n, c.m), c.buf(B_Z2, c.n, c.m)};
    apply(X[cur], t, X[cur], Z[0], false);       // U
    rapid_correct(Z[0], X[cur], Z[1], false);    // V
    int y = 0, w = 1;
    for (int it = 1; it <= c.P->mparam; it++) {
      const int z = 3 - y - w;
      rapid_correct(Z[w], Z[y], Z[z], false);
      y = w;
      w = z;
    }
    rapid_correct(Z[w], X[cur], X[cur ^ 1], true);
  }

  // Unfactorized hyperpower iteration of order k (Definition 1): X + X t
  // with t = R + R^2 + ... + R^(k-1) by Horner's rule h <- R + R h from h = R.
  __device__ void step_qhpim() {
    const int s = c.s, k = c.P->mparam;
    const DM R = c.buf(B_R, s, s);
    const DM H[2] = {c.buf(B_U, s, s), c.buf(B_V, s, s)};
    residual(X[cur], R);
    const DM* h = &R;
    for (int i = 2; i < k; i++) {
      Epi e;  // h <- R h + R
      e.aux[0] = &R;
      e.ct[0] = dc(1.0);
      gemm(R, *h, H[i & 1], e);
      h = &H[i & 1];
    }
    apply(X[cur], *h, X[cur], X[cur ^ 1], true);
  }
};

// One matrix end to end (every thread of the CTA): alpha, X_0, the
// iteration with its stop rule, E1..E4, X written to the caller.
template <class G>
__device__ void solve_item(const BatchParams& P, Ctx& c, G& g, int b) {
    Shared& sh = *c.sh;
    const BatchItem it = P.items[b];
    c.m = it.m;
    c.n = it.n;
    c.left = it.m > it.n;
    c.s = c.left ? it.n : it.m;
    c.gemms = 0;
    Solve<G> S(c, g);
    S.A = c.buf(B_A, it.m, it.n);
    S.X[0] = c.buf(B_X0, it.n, it.m);
    S.X[1] = c.buf(B_X1, it.n, it.m);
    // load A; row / column sums of moduli; ||A||_F^2
    float fro = 0.f;
    int bad = 0;
    for (long t = threadIdx.x; t < (long)it.m * it.n; t += blockDim.x) {
      const int i = (int)(t / it.n), j = (int)(t % it.n);
      for (int q = 0; q < 4; q++) {
        const double a = it.A[q][(long)i * it.lda + j];
        bad += isfinite(a) ? 0 : 1;
        S.A.at(q, i, j) = df_from(a);
        fro += (float)(a * a);
      }
    }
    __syncthreads();
    const double a_f2 = block_sum((double)fro, sh, 0);
    const double nbad = block_sum((double)bad, sh, 1);
    float rmax = 0.f, cmax = 0.f;
    for (int i = threadIdx.x; i < it.m; i += blockDim.x) {
      float r = 0.f;
      for (int j = 0; j < it.n; j++) {
        float q2 = 0.f;
        for (int q = 0; q < 4; q++) q2 += S.A.at(q, i, j).hi * S.A.at(q, i, j).hi;
        r += sqrtf(q2);
      }
      rmax = fmaxf(rmax, r);
    }
    for (int j = threadIdx.x; j < it.n; j += blockDim.x) {
      float r = 0.f;
      for (int i = 0; i < it.m; i++) {
        float q2 = 0.f;
        for (int q = 0; q < 4; q++) q2 += S.A.at(q, i, j).hi * S.A.at(q, i, j).hi;
        r += sqrtf(q2);
      }
      cmax = fmaxf(cmax, r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
      sh.red[threadIdx.x >> 5][0] = rmax;
      sh.red[threadIdx.x >> 5][1] = cmax;
    }
    __syncthreads();
    double nrm_inf = 0, nrm_1 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      nrm_inf = fmax(nrm_inf, sh.red[w][0]);
      nrm_1 = fmax(nrm_1, sh.red[w][1]);
    }
    __syncthreads();
    BatchResult res;
    memset(&res, 0, sizeof(res));
    res.side = c.left ? QPINV_SIDE_LEFT : QPINV_SIDE_RIGHT;
    double alpha = 0.0;
    if (a_f2 > 0.0) {
      if (P.alpha_mode == QPINV_ALPHA_USER) alpha = P.alpha_user;
      else if (P.alpha_mode == QPINV_ALPHA_FRO) alpha = 1.0 / a_f2;
      else alpha = 1.0 / (nrm_1 * nrm_inf);
    }
    res.alpha = alpha;
    if (nbad > 0.0) {
      res.status = -1;  // non-finite input: reported by the host
    } else {
      // X_0 = alpha A^H
      const dfv al = df_from(alpha);
      for (long t = threadIdx.x; t < (long)it.m * it.n; t += blockDim.x) {
        const int i = (int)(t / it.n), j = (int)(t % it.n);
        for (int q = 0; q < 4; q++) {
          const dfv a = S.A.at(q, i, j);
          S.X[0].at(q, j, i) = df_mul(al, q == 0 ? a : df_neg(a));
        }
      }
      __syncthreads();
      S.cur = 0;
      double prev = INFINITY;
      res.status = QPINV_NOT_CONVERGED;
      for (int j = 0; j < P.max_iter; j++) {
        switch (P.method) {
          case QPINV_NS: S.step_ns(); break;
          case QPINV_QSAI: S.step_qsai(); break;
          case QPINV_QRAPID: S.step_qrapid(); break;
          case QPINV_QHPIM: S.step_qhpim(); break;
          default: S.step_qhpi19(); break;
        }
        const double d = sqrt(S.nd), xn = sqrt(S.nx);
        if (!isfinite(d) || !isfinite(xn)) {
          res.status = QPINV_DIVERGED;
          break;
        }
        const double drel = xn > 0 ? d / xn : d;
        res.delta = d;
        res.delta_rel = drel;
        bool accept = true, stop = false;
        if (P.stop_rule == QPINV_STOP_PAPER_ABS) {
          if (d < P.tol) stop = true, res.status = QPINV_CONVERGED;
        } else if (drel <= P.tol) {
          stop = true;
          res.status = QPINV_CONVERGED;
        } else if (prev < 1e-3 && drel >= prev) {
          stop = true;
          accept = false;
          res.status = QPINV_PLATEAU;
        }
        if (accept) {
          S.cur ^= 1;
          res.iters = j + 1;
        }
        if (stop) break;
        prev = drel;
      }
      // Penrose residuals (Sec. 4): E1 = ||(AX - I) A||, E2 = ||(XA - I) X||,
      // E3, E4 = anti-Hermitian parts of AX - I and XA - I.
      const DM& Xf = S.X[S.cur];
      const DM Rr = c.buf(B_P1, it.m, it.m), Rl = c.buf(B_P2, it.n, it.n);
      const DM E1 = c.buf(B_P3, it.m, it.n), E2 = c.buf(B_P4, it.n, it.m);
      Epi e;
      e.diag = dc(-1.0);
      S.gemm(S.A, Xf, Rr, e);
      S.gemm(Xf, S.A, Rl, e);
      S.gemm(Rr, S.A, E1, Epi());
      S.gemm(Rl, Xf, E2, Epi());
      res.E[0] = sqrt(cta_fro2(E1, sh));
      res.E[1] = sqrt(cta_fro2(E2, sh));
      res.E[2] = sqrt(cta_antiherm2(Rr, sh));
      res.E[3] = sqrt(cta_antiherm2(Rl, sh));
      // norms of A, X, AX = Rr + I, XA = Rl + I
      cta_axpy(Rr, Rr, dc(1.0), nullptr, dc(0.0), dc(1.0));
      cta_axpy(Rl, Rl, dc(1.0), nullptr, dc(0.0), dc(1.0));
      const double nr[4] = {sqrt(a_f2), sqrt(cta_fro2(Xf, sh)), sqrt(cta_fro2(Rr, sh)), sqrt(cta_fro2(Rl, sh))};
      for (int q = 0; q < 4; q++) res.E_rel[q] = nr[q] > 0 ? res.E[q] / nr[q] : res.E[q];
      // write X
      for (long t = threadIdx.x; t < (long)it.n * it.m; t += blockDim.x) {
        const int i = (int)(t / it.m), j = (int)(t % it.m);
        for (int q = 0; q < 4; q++) it.X[q][(long)i * it.ldx + j] = df_to(Xf.at(q, i, j));
      }
    }
    res.gemms = c.gemms;
    if (threadIdx.x == 0) P.results[b] = res;
    __syncthreads();
}

template <int RM, int RN, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_batched(BatchParams P) {
  __shared__ Shared sh;
  __shared__ SimtTiles tl;
  __shared__ int next;
  Ctx c;
  c.P = &P;
  c.sh = &sh;
  c.base = P.ws + (long)blockIdx.x * P.slot_elems;
  SimtGemm<RM, RN> g{&sh, &tl};
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(P.counter, 1);
    __syncthreads();
    const int slot = next;
    __syncthreads();
    if (slot >= P.count) break;
    solve_item(P, c, g, P.order[slot]);
  }
}

#ifndef QP_BATCHED_TILE
cudaError_t launch_batched(int tile, int slots, const BatchParams& P, cudaStream_t st) {
  switch (tile) {
    case 0: return batched_launch_t0(slots, P, st);
    case 1: return batched_launch_t1(slots, P, st);
    case 2: return batched_launch_t2(slots, P, st);
    case 3: return batched_launch_t3(slots, P, st);
    case 4: return batched_launch_t4(slots, P, st);
    case 5: return batched_launch_tc(slots, P, st);
    default: return cudaErrorInvalidValue;
  }
}
#endif

unsigned long long mix(unsigned long long h, unsigned long long v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

}  // namespace

#if defined(QP_BATCHED_TILE) && !defined(QP_BATCHED_TC_UNIT)
// One kernel instantiation: QP_TILE_RM x QP_TILE_RN outputs per thread,
// QP_TILE_MINB resident CTAs per SM requested from the compiler.
cudaError_t QP_TILE_LAUNCH(int slots, const BatchParams& P, cudaStream_t st) {
  k_batched<QP_TILE_RM, QP_TILE_RN, QP_TILE_MINB><<<slots, TPB, 0, st>>>(P);
  return cudaGetLastError();
}
int QP_TILE_OCCUPANCY() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched<QP_TILE_RM, QP_TILE_RN, QP_TILE_MINB>, TPB, 0) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}
#elif !defined(QP_BATCHED_TILE)
const char* batched_tile_name(int tile) {
  static const char* names[BATCH_TILES] = {"16x16", "32x32", "64x32", "32x64", "64x64", "tc"};
  return tile >= 0 && tile < BATCH_TILES ? names[tile] : "?";
}

int batched_slots_per_sm(int tile) {
  switch (tile) {
    case 0: return batched_occupancy_t0();
    case 1: return batched_occupancy_t1();
    case 2: return batched_occupancy_t2();
    case 3: return batched_occupancy_t3();
    case 4: return batched_occupancy_t4();
    case 5: return 1;  // tensor-core engine: one CTA (all of TMEM) per SM
    default: return 1;
  }
}

// One batched call: host descriptors (largest cost first) into pinned
// staging, then upload + counter reset + persistent kernel + result download
// on `st` -- or, with `graph`, on the graph's own stream as one replayed CUDA
// graph (captured again whenever the launch shape changes).
cudaError_t run_batched(int batch, const int* m, const int* n, const double* const* A, const long* lda,
                        double* const* X, const long* ldx, int method, double tol, int max_iter, int mparam,
                        int stop_rule, int alpha_mode, double alpha_user, const double* hpi19_k, const BatchRun& r,
                        BatchGraph* graph, std::vector<BatchResultHost>& out, cudaStream_t st) {
  BatchItem* items = static_cast<BatchItem*>(r.host_items);
  int* order = static_cast<int*>(r.host_order);
  std::vector<double> cost(batch);
  for (int b = 0; b < batch; b++) {
    BatchItem& it = items[b];
    for (int q = 0; q < 4; q++) {
      it.A[q] = A[4 * b + q];
      it.X[q] = X[4 * b + q];
    }
    it.lda = lda[b];
    it.ldx = ldx[b];
    it.m = m[b];
    it.n = n[b];
    const double sm = std::min(m[b], n[b]), l = std::max(m[b], n[b]);
    cost[b] = sm * sm * l;
    order[b] = b;
  }
  std::stable_sort(order, order + batch, [&](int x, int y) { return cost[x] > cost[y]; });
  BatchParams P;
  P.items = (const BatchItem*)r.dev_items;
  P.order = (const int*)r.dev_order;
  P.count = batch;
  P.counter = r.dev_counter;
  P.results = (BatchResult*)r.dev_results;
  P.ws = (dfv*)r.ws;
  P.slot_elems = (long)NBUF * 4 * MAXD * MAXD;
  P.method = method;
  P.mparam = mparam;
  P.stop_rule = stop_rule;
  P.max_iter = max_iter;
  P.alpha_mode = alpha_mode;
  P.tol = tol;
  P.alpha_user = alpha_user;
  for (int t = 0; t < 12; t++) P.k[t] = hpi19_k[t];
  P.tc_maps = (const CUtensorMap*)r.tc_maps;
  P.tc_ws = (char*)r.tc_ws;
  P.tc_slot_bytes = (long)batched_tc_slot_bytes();
  P.tc_slices = 7;
  P.err = r.err;
  if (r.tile == BATCH_TILE_TC) {
    if (!r.tc_ws || !r.tc_maps || !r.host_maps || !r.err) return cudaErrorInvalidValue;
    cudaError_t e = batched_tc_maps((char*)r.tc_ws, r.slots, (CUtensorMap*)r.host_maps, r.tc_maps, st);
    if (e != cudaSuccess) return e;
  }
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(r.dev_items, r.host_items, sizeof(BatchItem) * batch, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(r.dev_order, r.host_order, sizeof(int) * batch, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(r.dev_counter, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = launch_batched(r.tile, r.slots, P, s)) != cudaSuccess) return e;
    ++g_kernel_launches;
    return cudaMemcpyAsync(r.host_results, r.dev_results, sizeof(BatchResult) * batch, cudaMemcpyDeviceToHost, s);
  };
  cudaError_t e;
  if (!graph) {
    if ((e = enqueue(st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  } else {
    // the launch shape: everything the captured nodes bake in
    unsigned long long key = 1469598103934665603ull;
    const unsigned long long parts[] = {(unsigned long long)batch, (unsigned long long)r.tile,
                                        (unsigned long long)r.slots, (unsigned long long)(uintptr_t)r.ws,
                                        (unsigned long long)(uintptr_t)r.dev_items,
                                        (unsigned long long)(uintptr_t)r.host_items,
                                        (unsigned long long)(uintptr_t)r.host_results,
                                        (unsigned long long)method, (unsigned long long)max_iter,
                                        (unsigned long long)mparam, (unsigned long long)stop_rule,
                                        (unsigned long long)alpha_mode};
    for (unsigned long long v : parts) key = mix(key, v);
    unsigned long long tb, ab;
    memcpy(&tb, &tol, 8);
    memcpy(&ab, &alpha_user, 8);
    key = mix(mix(key, tb), ab);
    if (!graph->exec || graph->key != key) {
      if (graph->exec) {
        cudaGraphExecDestroy(graph->exec);
        graph->exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      if ((e = cudaStreamBeginCapture(graph->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
      const long long launches_before = g_kernel_launches;
      const cudaError_t eq = enqueue(graph->stream);
      g_kernel_launches = launches_before;  // counted when the graph runs
      e = cudaStreamEndCapture(graph->stream, &g);
      if (eq != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return eq;
      }
      if (e != cudaSuccess) return e;
      e = cudaGraphInstantiate(&graph->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        graph->exec = nullptr;
        return e;
      }
      graph->key = key;
      graph->replays = 0;
    }
    // order the replay after the caller's stream
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    cudaEventRecord(ev, st);
    cudaStreamWaitEvent(graph->stream, ev, 0);
    e = cudaGraphLaunch(graph->exec, graph->stream);
    if (e == cudaSuccess) {
      ++g_kernel_launches;
      graph->replays++;
      e = cudaStreamSynchronize(graph->stream);
    }
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return e;
  }
  const BatchResult* res = static_cast<const BatchResult*>(r.host_results);
  out.resize(batch);
  for (int b = 0; b < batch; b++) {
    BatchResultHost& h = out[b];
    h.status = res[b].status;
    h.iters = res[b].iters;
    h.side = res[b].side;
    h.gemms = res[b].gemms;
    h.alpha = res[b].alpha;
    h.delta = res[b].delta;
    h.delta_rel = res[b].delta_rel;
    for (int q = 0; q < 4; q++) {
      h.E[q] = res[b].E[q];
      h.E_rel[q] = res[b].E_rel[q];
    }
  }
  return cudaSuccess;
}

size_t batched_slot_bytes() { return sizeof(float) * 2 * (size_t)NBUF * 4 * MAXD * MAXD; }
size_t batched_item_bytes() { return sizeof(BatchItem); }
size_t batched_result_bytes() { return sizeof(BatchResult); }
int batched_max_dim() { return MAXD; }
#endif  // QP_BATCHED_TILE

}  // namespace qp
