// solver.cu -- C ABI of libqpinv: context, device workspace, the per-method
// iteration schedules, the precision schedule and the stop rules.
//
// Every iteration is a fixed list of quaternion GEMMs, each followed by one
// fused combine pass (elementwise.cu).  The schedules are Algorithms 1-3 and
// Newton-Schulz rewritten with small quantities, which is exact algebra and
// keeps low-precision products from rounding away the corrections:
//   QHPI19 (Alg. 3): R = I - AX, R2, R4; (I + d1R2 + R4)(I + d2R2 + R4) = I + u
//     with u = a + b + ab (a = d1R2 + R4, b = d2R2 + R4); V = I + v,
//     W = I + w; Gamma = VW + c1R2 + c2R4 = I + gamma;
//     X_{j+1} = X (I + (R + R2) Gamma) = X + X t,  t = S + S gamma, S = R + R2.
//     Seven products: AX, RR, R2R2, ab, vw, S gamma, X t.
//   QSAI (Alg. 2): Q = (I + b1R2 + R4)(I + b2R2 + R4) = I + q,
//     X (I + R) Q = X + X t with t = R + q + R q.  Six products.
//   Newton-Schulz: X (2I - AX) = X + X R.  Two products.
//   QRAPID (Alg. 1): U = X (13I - P(15I - P(7I - P)))/4 = X + X (R + R2 + R3/4)
//     (P = I - R); V = U + X(I - AU); Z_l = W + Y(I - AW); X_{j+1} = Z + X(I - AZ).
//     8 + 2N products.
//   QHPIM(k) (Definition 1, unfactorized): X (I + R + ... + R^(k-1)) = X + X t,
//     t by Horner's rule h <- R + R h from h = R.  k products.
// Side: the paper's right form (R = I_m - A X, m x m) or the left form
// (R = I_n - X A, X_{j+1} = p(R) X), identical in exact arithmetic since
// X (AX)^k = (XA)^k X; AUTO picks the smaller residual.
//
// Precision.  Products of polynomials in R ("R-products") carry errors that
// are relative to R-sized quantities; products with A or X ("X-products":
// the residual A X and the update X t) carry errors that the next residual
// multiplies by about ||A|| ||X||.  Hence:
//   tensor-core phase: FP32 masters; R-products on BF16 splits (split_level
//     terms); X-products on BF16 splits while kappa_est = ||A|| ||X_j||_F is
//     small, then as exact-slice products with 4 slices (about FP32 level);
//   polish phase (MIXED): FP64 masters; X-products FP64-accurate (8 exact
//     slices, 56 bits); R-products stay on BF16 splits.
// Penrose residuals use FP64-accurate products (exact slices, or the
// CUDA-core FP64 kernel in the FP64 form).
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/qpinv.h"
#include "common.cuh"

using namespace qp;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum { EV_TC = 0, EV_F64 = 1, EV_EW = 2, EV_EMU = 3 };
enum { PM_TC = 0, PM_F64 = 1, PM_EMU = 2 };

struct EvRec {
  cudaEvent_t a, b;
  int kind;
};

// Row pitch of BF16 operand planes (split forms, exact slices): 64 elements,
// 128 bytes, so that every 64-byte TMA box row lies in whole 32-byte L2
// sectors (an odd K such as 2001 otherwise makes each row straddle one: 1.5x
// the sectors, measured 2x slower exact-slice products at n = 2001).
long rup64(long x) { return (x + 63) / 64 * 64; }

}  // namespace

struct qpinv_ctx {
  int device = 0;
  qpinv_options opt;
  std::string err = "no error";
  std::map<std::string, DevBuf> bufs;
  qpinv_stats stats;
  std::vector<EvRec> pending;
  std::vector<cudaEvent_t> pool;
  int* d_err = nullptr;
  double* h_pin = nullptr;  // pinned host scalars
  cudaStream_t st = nullptr;
  bool trace = false;
  std::vector<float> alpha_w;  // learned-alpha network (empty: untrained)
  // batched solves: pinned staging, the replayed CUDA graph, tuned tiles
  void* bh_buf[3] = {nullptr, nullptr, nullptr};  // items, order, results (pinned)
  size_t bh_cap[3] = {0, 0, 0};
  qp::BatchGraph bgraph;
  std::map<unsigned long long, int> tile_of;  // batch signature -> tuned tile
  void* bmaps_host = nullptr;                 // pinned TMA maps of the batched tensor-core engine
};

namespace {

// ------------------------------------------------------------- utilities

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct QpError {
  int code;
  std::string msg;
};

void ck(qpinv_ctx* c, cudaError_t e, const char* what) {
  (void)c;
  if (e != cudaSuccess) throw QpError{QPINV_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

void* buf(qpinv_ctx* c, const std::string& name, size_t bytes) {
  DevBuf& b = c->bufs[name];
  if (b.bytes < bytes) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw QpError{QPINV_E_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes for " + name + " failed"};
    }
    b.bytes = bytes;
  }
  return b.p;
}

// A quaternion matrix of the workspace: FP64 and/or FP32 master planes and
// BF16 operand forms (round-to-nearest splits) for the tensor cores.
struct QMat {
  int rows = 0, cols = 0;
  Planes<double> d;
  Planes<float> f;
  Split16 s16;
};

enum { MST_F = 1, MST_D = 2 };

QMat mat(qpinv_ctx* c, const std::string& name, int rows, int cols, int masters, bool aform, bool bform,
         int levels = 3) {
  QMat M;
  M.rows = rows;
  M.cols = cols;
  const long ps = (long)rows * cols;
  if (masters & MST_D) {
    M.d.ld = cols;
    M.d.ps = ps;
    M.d.p = (double*)buf(c, name + ".d", sizeof(double) * 4 * (size_t)ps + 64);
  }
  if (masters & MST_F) {
    // 16-byte rows, so that the tensor-core epilogues' FP32 accesses stay
    // vectorised for any column count
    M.f.ld = (cols + 3) / 4 * 4;
    M.f.ps = (long)rows * M.f.ld;
    M.f.p = (float*)buf(c, name + ".f", sizeof(float) * 4 * (size_t)M.f.ps + 64);
  }
  M.s16.levels = levels;
  if (aform) {
    M.s16.lda = rup64(cols);
    M.s16.psa = (long)rows * M.s16.lda;
    M.s16.a = (bf16*)buf(c, name + ".a16", sizeof(bf16) * 4 * levels * (size_t)M.s16.psa + 64);
  }
  if (bform) {
    M.s16.ldb = rup64(rows);
    M.s16.psb = (long)cols * M.s16.ldb;
    M.s16.b = (bf16*)buf(c, name + ".b16", sizeof(bf16) * 4 * levels * (size_t)M.s16.psb + 64);
  }
  return M;
}

Planes<const double> dview(const QMat& M) {
  Planes<const double> p;
  p.p = M.d.p;
  p.ld = M.d.ld;
  p.ps = M.d.ps;
  return p;
}
Planes<const float> fview(const QMat& M) {
  Planes<const float> p;
  p.p = M.f.p;
  p.ld = M.f.ld;
  p.ps = M.f.ps;
  return p;
}

cudaEvent_t ev_get(qpinv_ctx* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  ck(c, cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

// Runs `launch` with optional event timing and counts it.
template <typename F>
void timed(qpinv_ctx* c, int kind, double flops, double issued, double bytes, F&& launch) {
  EvRec r{nullptr, nullptr, kind};
  if (c->opt.profile) {
    r.a = ev_get(c);
    r.b = ev_get(c);
    ck(c, cudaEventRecord(r.a, c->st), "cudaEventRecord");
  }
  const long long before = g_kernel_launches;
  ck(c, launch(), "kernel launch");
  c->stats.kernel_launches += g_kernel_launches - before;
  if (kind == EV_TC) {
    c->stats.tc_gemm_launches++;
    c->stats.tc_gemm_flops += flops;
    c->stats.tc_gemm_flops_issued += issued;
  } else if (kind == EV_F64) {
    c->stats.f64_gemm_launches++;
    c->stats.f64_gemm_flops += flops;
  } else if (kind == EV_EMU) {
    c->stats.emu_gemm_launches++;
    c->stats.emu_gemm_flops += flops;
    c->stats.emu_gemm_flops_issued += issued;
  } else {
    c->stats.ew_launches++;
    c->stats.ew_bytes += bytes;
  }
  if (c->opt.profile) {
    ck(c, cudaEventRecord(r.b, c->st), "cudaEventRecord");
    c->pending.push_back(r);
  }
}

void flush_events(qpinv_ctx* c) {
  for (EvRec& r : c->pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (r.kind == EV_TC) c->stats.tc_gemm_ms += ms;
    else if (r.kind == EV_F64) c->stats.f64_gemm_ms += ms;
    else if (r.kind == EV_EMU) c->stats.emu_gemm_ms += ms;
    else c->stats.ew_ms += ms;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->pending.clear();
}

// Host read of `n` doubles from device (synchronises the stream).
void read_back(qpinv_ctx* c, const double* d, int n, double* h) {
  ck(c, cudaMemcpyAsync(c->h_pin, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st), "read back");
  ck(c, cudaStreamSynchronize(c->st), "stream sync");
  memcpy(h, c->h_pin, sizeof(double) * n);
}

void check_kernel_error(qpinv_ctx* c) {
  int h = 0;
  ck(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "read error word");
  ck(c, cudaStreamSynchronize(c->st), "stream sync");
  if (h != 0) {
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st);
    throw QpError{QPINV_E_TIMEOUT, "tensor-core GEMM bounded wait expired (code " + std::to_string(h) + ")"};
  }
}

// -------------------------------------------------------- solver state

struct Solver {
  qpinv_ctx* c = nullptr;
  int m = 0, n = 0;
  bool left = false;
  int s = 0;              // residual side (s x s)
  bool dbl = false;       // master type of the current phase: double (true) or float
  int L = 3;              // BF16 split terms written for tensor-core operands (0: every product in FP64)
  int Lr = 2;             // BF16 split terms of tensor-core R-products
  int Lx = 3;             // BF16 split terms of tensor-core X-products
  int Lcur = 3;           // split terms of the product being issued
  int xmode = PM_TC;      // mode of the X-products this iteration
  int rmode = -1;         // mode of the R-products (-1: PM_F64 if L == 0, else PM_TC)
  int xS = 8;             // exact slices of X-products in PM_EMU mode
  int xSu = 3;            // ... of the update product X t while the masters are FP32
  int xSp = 0;            // ... of the update product in a polish step (0: xS)
  bool pre_res = false;   // pre_R is the residual of X[cur], computed ahead of the step
  QMat pre_R;
  // The buffer "R" holds I - (residual product of X[res_cur]) with FP64
  // masters and FP64-accurate products (-1: it does not): the Penrose pass
  // then reuses it instead of forming that side's product again.
  int res_cur = -1;
  QMat res_R;
  // Exponents and exact slices of A (an operand of every residual product,
  // constant during the solve), kept in their own buffers across products:
  // the form (0: A-form rows, 1: B-form columns), slice count and master
  // precision they were made for (form -1: none yet).
  int acache_form = -1, acache_S = 0;
  bool acache_dbl = false;
  long long gemms = 0;
  QMat A, X[2];
  int cur = 0;
  double* partials = nullptr;
  int partial_cap = 0;

  // ---------------- products ----------------
  struct Acc {
    const void* p;
    int kind;
    long ld, ps;
    const int* erow;
    const int* ecol;
    int shift;
    const long long* p2 = nullptr;  // ACC_I64: second accumulator of the same layout, summed
  };

  // acc(rows x cols) = P (rows x K) * Q (K x cols) in one of three modes:
  //   PM_TC  - tcgen05 on BF16 splits (L terms), FP32 accumulation;
  //   PM_F64 - CUDA-core FP64 on the FP64 masters;
  //   PM_EMU - exact-slice product on the tensor cores from the masters of the
  //            current phase (xS slices; FP64-accurate for 8).
  Acc prod(const QMat& P, const QMat& Q, int mode) {
    const int M = P.rows, K = P.cols, N = Q.cols;
    gemms++;
    const double flops = 32.0 * M * (double)K * N;
    if (mode == PM_EMU) return prod_emu(P, Q, xS, flops);
    if (mode == PM_F64) {
      Planes<double> C;
      C.ld = N;
      C.ps = (long)M * N;
      C.p = (double*)buf(c, "acc64", sizeof(double) * 4 * (size_t)C.ps + 64);
      Planes<const double> a = dview(P), b = dview(Q);
      timed(c, EV_F64, flops, flops, 0, [&] { return launch_qgemm_f64(M, K, N, a, b, C, c->st); });
      return Acc{C.p, ACC_F64, C.ld, C.ps, nullptr, nullptr, 0};
    }
    Planes<float> C;
    C.ld = (N + 31) / 32 * 32;  // 128-byte FP32 rows
    C.ps = (long)M * C.ld;
    C.p = (float*)buf(c, "acc32", sizeof(float) * 4 * (size_t)C.ps + 64);
    TcGemmArgs g = tc_args(P, Q);
    g.C = C;
    timed(c, EV_TC, flops, flops * g.npairs, 0, [&] { return launch_qgemm_tc(g, c->st); });
    return Acc{C.p, ACC_F32, C.ld, C.ps, nullptr, nullptr, 0};
  }

  // Tensor-core GEMM arguments of P Q on BF16 splits of Lcur terms
  // (1 pair, 3 pairs with i + j <= 1, 6 pairs with i + j <= 2).
  TcGemmArgs tc_args(const QMat& P, const QMat& Q) const {
    TcGemmArgs g;
    g.M = P.rows;
    g.N = Q.cols;
    g.K = P.cols;
    g.k0 = 0;
    g.k1 = P.cols;
    g.A = &P.s16;
    g.B = &Q.s16;
    static const int pi3[6] = {2, 1, 0, 1, 0, 0}, pj3[6] = {0, 1, 2, 0, 1, 0};
    static const int pi2[3] = {1, 0, 0}, pj2[3] = {0, 1, 0};
    if (Lcur >= 3) {
      g.npairs = 6;
      for (int t = 0; t < 6; t++) g.pair_i[t] = pi3[t], g.pair_j[t] = pj3[t];
    } else if (Lcur == 2) {
      g.npairs = 3;
      for (int t = 0; t < 3; t++) g.pair_i[t] = pi2[t], g.pair_j[t] = pj2[t];
    } else {
      g.npairs = 1;
    }
    g.err = c->d_err;
    g.broad = c->opt.tc_broad;
    return g;
  }

  static void set_acc(CombineArgs& a, const Acc& acc) {
    a.acc = acc.p;
    a.acc_kind = acc.kind;
    a.ld_acc = acc.ld;
    a.ps_acc = acc.ps;
    a.acc_erow = acc.erow;
    a.acc_ecol = acc.ecol;
    a.acc_shift = acc.shift;
    a.acc2 = acc.p2;
  }

  // Whether the combine pass `a` (no accumulator set yet) can run in the
  // epilogue of the tensor-core product P Q: round-to-nearest splits only, no
  // output that overwrites an operand form the product is still reading, and
  // in the FP64 phase no stop-test partials (those norms stay FP64 sums).
  bool epi_fusable(const CombineArgs& a, const QMat& P, const QMat& Q, bool with_partials) const {
    if (!c->opt.fuse_epilogue || a.acc || a.nout < 1 || a.nout > kMaxOut) return false;
    if (a.f64 != (dbl ? 1 : 0) || (dbl && with_partials)) return false;
    for (int o = 0; o < a.nout; o++) {
      const OutSpec& O = a.out[o];
      if (O.exp_a || O.exp_b) return false;
      if ((O.s16.a || O.s16.b) && O.s16.levels < 1) return false;
      const void* forms[4] = {P.s16.a, P.s16.b, Q.s16.a, Q.s16.b};
      for (const void* f : forms)
        if (f && (O.s16.a == f || O.s16.b == f)) return false;
    }
    return true;
  }

  // The product P Q in `mode` followed by the combine pass `a` (accumulator
  // unset): one tensor-core launch with the pass in its epilogue when
  // possible, else the product and the combine kernel.
  void prod_run(const QMat& P, const QMat& Q, int mode, CombineArgs a, bool with_partials = false,
                int red_slot = 0) {
    if (mode == PM_TC && epi_fusable(a, P, Q, with_partials)) {
      const int M = P.rows, K = P.cols, N = Q.cols;
      gemms++;
      const double flops = 32.0 * M * (double)K * N;
      TcGemmArgs g = tc_args(P, Q);
      EpiArgs& e = g.epi;
      e.nout = a.nout;
      for (int o = 0; o < a.nout; o++) {
        const OutSpec& O = a.out[o];
        EpiOut& d = e.out[o];
        d.mp = O.mp;
        d.mld = O.mld;
        d.mps = O.mps;
        d.a = O.s16.a;
        d.lda = O.s16.lda;
        d.psa = O.s16.psa;
        d.b = O.s16.b;
        d.ldb = O.s16.ldb;
        d.psb = O.s16.psb;
        d.levels = O.s16.levels;
        d.cacc = O.cacc;
        for (int t = 0; t < 4; t++) d.caux[t] = O.caux[t];
        d.diag = O.diag;
      }
      e.f64 = a.f64;
      for (int t = 0; t < 4; t++) {
        e.aux[t] = a.aux[t];
        e.ld_aux[t] = a.ld_aux[t];
        e.ps_aux[t] = a.ps_aux[t];
      }
      const int blocks = tc_partial_blocks(M, N, c->opt.tc_broad);
      if (with_partials) {
        if (blocks > partial_cap) {
          partials = (double*)buf(c, "partials", sizeof(double) * 3 * (size_t)blocks + 64);
          partial_cap = blocks;
        }
        e.partials = partials;
      }
      timed(c, EV_TC, flops, flops * g.npairs, 0, [&] { return launch_qgemm_tc(g, c->st); });
      c->stats.fused_epilogues++;
      if (with_partials) {
        double* red = (double*)buf(c, "red", sizeof(double) * 8);
        timed(c, EV_EW, 0, 0, 24.0 * blocks,
              [&] { return launch_reduce_partials(partials, blocks, 3, red + red_slot, c->st); });
      }
      return;
    }
    Acc acc = prod(P, Q, mode);
    set_acc(a, acc);
    run(a, with_partials, red_slot);
  }

  Acc prod_emu(const QMat& P, const QMat& Q, int S, double flops) {
    const int M = P.rows, K = P.cols, N = Q.cols;
    // A as an operand: its exponents and slices come from (or go to) the cache
    const bool pA = &P == &A, qA = &Q == &A;
    const bool pA_hit = pA && acache_form == 0 && acache_S == S && acache_dbl == dbl;
    const bool qA_hit = qA && acache_form == 1 && acache_S == S && acache_dbl == dbl;
    int* eP = (int*)buf(c, pA ? "emu.cacheA.e" : "emu.eP", sizeof(int) * (size_t)M + 64);
    int* eQ = (int*)buf(c, qA ? "emu.cacheA.e" : "emu.eQ", sizeof(int) * (size_t)N + 64);
    int* eS = (int*)buf(c, "emu.eS", sizeof(int) * (size_t)COL_SCRATCH(N) + 64);
    if (dbl) {
      if (!pA_hit)
        timed(c, EV_EW, 0, 0, 32.0 * M * K, [&] { return launch_maxexp(dview(P), M, K, 0, eP, nullptr, c->st); });
      if (!qA_hit)
        timed(c, EV_EW, 0, 0, 32.0 * K * N, [&] { return launch_maxexp(dview(Q), K, N, 1, eQ, eS, c->st); });
    } else {
      if (!pA_hit)
        timed(c, EV_EW, 0, 0, 16.0 * M * K,
              [&] { return launch_maxexp_f32(fview(P), M, K, 0, eP, nullptr, c->st); });
      if (!qA_hit)
        timed(c, EV_EW, 0, 0, 16.0 * K * N, [&] { return launch_maxexp_f32(fview(Q), K, N, 1, eQ, eS, c->st); });
    }
    Split16 za, zb;
    za.levels = zb.levels = S;
    za.lda = rup64(K);
    za.psa = (long)M * za.lda;
    za.a = (bf16*)buf(c, pA ? "emu.cacheA.z" : "emu.za", sizeof(bf16) * 4 * S * (size_t)za.psa + 64);
    zb.ldb = rup64(K);
    zb.psb = (long)N * zb.ldb;
    zb.b = (bf16*)buf(c, qA ? "emu.cacheA.z" : "emu.zb", sizeof(bf16) * 4 * S * (size_t)zb.psb + 64);
    // the slices: P's rows (A-form), Q's columns (B-form, transposed)
    const double sbytes = 2.0 * S * 4;
    if (dbl) {
      if (!pA_hit)
        timed(c, EV_EW, 0, 0, (32.0 + sbytes) * M * K,
              [&] { return launch_slice_rows(dview(P), M, K, eP, S, za.a, za.lda, za.psa, c->st); });
      if (!qA_hit)
        timed(c, EV_EW, 0, 0, (32.0 + sbytes) * K * N,
              [&] { return launch_slice_cols(dview(Q), K, N, eQ, S, zb.b, zb.ldb, zb.psb, c->st); });
    } else {
      if (!pA_hit)
        timed(c, EV_EW, 0, 0, (16.0 + sbytes) * M * K,
              [&] { return launch_slice_rows(fview(P), M, K, eP, S, za.a, za.lda, za.psa, c->st); });
      if (!qA_hit)
        timed(c, EV_EW, 0, 0, (16.0 + sbytes) * K * N,
              [&] { return launch_slice_cols(fview(Q), K, N, eQ, S, zb.b, zb.ldb, zb.psb, c->st); });
    }
    if (pA || qA) {
      acache_form = pA ? 0 : 1;
      acache_S = S;
      acache_dbl = dbl;
    }
    long long* acc = (long long*)buf(c, "emu.acc", sizeof(long long) * 4 * (size_t)M * N + 64);
    int lg = 0;
    while ((1L << lg) < 4L * K) lg++;
    const int shift = 61 - lg;  // |sum| < 4K in normalized units: no int64 overflow
    // Levels d = s + t are launched two at a time (two TMEM accumulators
    // summed by the epilogue), lowest first.  Levels whose FP32 rounding
    // could matter are summed in K chunks small enough for every partial sum
    // to be exact: balanced digits are at most 2^7 (slice 0) and 2^6, so one
    // level-d product term is at most 2^14 (d = 0) or 2^12 (d + 3) over the
    // pairs (2^13 for (0, d) and (d, 0), 2^12 for the rest); with 4 Kc terms
    // per output this stays <= 2^24 for Kc <= 256 (d = 0) and 2^10 / (d + 3).
    // The two lowest levels are summed over the whole K.
    auto chunk = [&](int d) {
      if (d > S - 3) return K;
      const int lim = d == 0 ? 256 : 1024 / (d + 3);
      return lim >= 64 ? (lim / 64) * 64 : 64;
    };
    if (emu_fused_ok(K, S)) {
      // all levels and chunks in one launch, int32 level sums in TMEM
      EmuGemmArgs g;
      g.M = M;
      g.N = N;
      g.K = K;
      g.A = &za;
      g.B = &zb;
      g.S = S;
      for (int d = 0; d < S; d++) {
        if (d > S - 3) {
          g.kc[d] = K;
        } else {
          const int lim = d == 0 ? 256 : 1024 / (d + 3);
          g.kc[d] = (lim / 32) * 32;
        }
      }
      // half of the levels go to a second accumulator (see qgemm_emu.cu)
      // (each group's first level stores: neither accumulator needs clearing)
      long long* acc2 = (long long*)buf(c, "emu.acc2", sizeof(long long) * 4 * (size_t)M * N + 64);
      g.C64 = acc;
      g.C64b = S >= 2 ? acc2 : nullptr;
      g.ld64 = N;
      g.ps64 = (long)M * N;
      g.shift = shift;
      g.err = c->d_err;
      const bool pair = M > 128 && c->opt.emu_pair == 1;
      timed(c, EV_EMU, flops, flops * S * (S + 1) / 2, 0,
            [&] { return pair ? launch_qgemm_emu_pair(g, c->st) : launch_qgemm_emu(g, c->st); });
      Acc r{acc, ACC_I64, (long)N, (long)M * N, eP, eQ, shift};
      r.p2 = g.C64b;
      return r;
    }
    ck(c, cudaMemsetAsync(acc, 0, sizeof(long long) * 4 * (size_t)M * N, c->st), "memset");
    for (int hi = S - 1; hi >= 0; hi -= 2) {
      const int lo = hi - 1;  // second level of the launch (-1: none)
      TcGemmArgs g;
      g.M = M;
      g.N = N;
      g.K = K;
      g.A = &za;
      g.B = &zb;
      g.npairs = 0;
      for (int t = 0; t <= hi; t++, g.npairs++) {
        g.pair_i[g.npairs] = t;
        g.pair_j[g.npairs] = hi - t;
        g.pair_acc[g.npairs] = 0;
      }
      if (lo >= 0)
        for (int t = 0; t <= lo; t++, g.npairs++) {
          g.pair_i[g.npairs] = t;
          g.pair_j[g.npairs] = lo - t;
          g.pair_acc[g.npairs] = 1;
        }
      g.C64 = acc;
      g.ld64 = N;
      g.ps64 = (long)M * N;
      g.shift = shift;
      g.err = c->d_err;
      const int kc = lo >= 0 ? std::min(chunk(hi), chunk(lo)) : chunk(hi);
      for (int k0 = 0; k0 < K; k0 += kc) {
        g.k0 = k0;
        g.k1 = k0 + kc < K ? k0 + kc : K;
        const double part = flops * (double)(g.k1 - g.k0) / K;
        timed(c, EV_TC, (lo == 0 || hi == 0) ? part : 0.0, part * g.npairs, 0, [&] { return launch_qgemm_tc(g, c->st); });
      }
    }
    return Acc{acc, ACC_I64, (long)N, (long)M * N, eP, eQ, shift};
  }

  // ---------------- combine helpers ----------------
  CombineArgs base_args(int rows, int cols, const Acc* acc) {
    CombineArgs a;
    a.rows = rows;
    a.cols = cols;
    a.f64 = dbl ? 1 : 0;
    if (acc) {
      a.acc = acc->p;
      a.acc_kind = acc->kind;
      a.ld_acc = acc->ld;
      a.ps_acc = acc->ps;
      a.acc_erow = acc->erow;
      a.acc_ecol = acc->ecol;
      a.acc_shift = acc->shift;
      a.acc2 = acc->p2;
    }
    return a;
  }
  void aux(CombineArgs& a, int t, const QMat& M) {
    if (dbl) {
      a.aux[t] = M.d.p;
      a.ld_aux[t] = M.d.ld;
      a.ps_aux[t] = M.d.ps;
    } else {
      a.aux[t] = M.f.p;
      a.ld_aux[t] = M.f.ld;
      a.ps_aux[t] = M.f.ps;
    }
  }
  // Adds an output; forms: 'f' master of the phase type, 'a' A-form, 'b' B-form.
  OutSpec& out(CombineArgs& a, const QMat& M, const char* forms, double cacc, double diag = 0.0) {
    OutSpec& o = a.out[a.nout++];
    o = OutSpec();
    if (strchr(forms, 'f')) {
      if (dbl) {
        o.mp = M.d.p;
        o.mld = M.d.ld;
        o.mps = M.d.ps;
      } else {
        o.mp = M.f.p;
        o.mld = M.f.ld;
        o.mps = M.f.ps;
      }
    }
    if (L > 0) {
      o.s16.levels = L;
      if (strchr(forms, 'a')) {
        o.s16.a = M.s16.a;
        o.s16.lda = M.s16.lda;
        o.s16.psa = M.s16.psa;
      }
      if (strchr(forms, 'b')) {
        o.s16.b = M.s16.b;
        o.s16.ldb = M.s16.ldb;
        o.s16.psb = M.s16.psb;
      }
    }
    o.cacc = cacc;
    o.diag = diag;
    return o;
  }
  // with_partials: block partials of ||out - aux0||^2, ||out||^2 and the
  // non-finite count, reduced into red_slot[0..2] of the "red" buffer.
  void run(CombineArgs& a, bool with_partials = false, int red_slot = 0) {
    const int blocks = combine_blocks(a);
    if (with_partials) {
      if (blocks > partial_cap) {
        partials = (double*)buf(c, "partials", sizeof(double) * 3 * (size_t)blocks + 64);
        partial_cap = blocks;
      }
      a.partials = partials;
    }
    double bytes = 0;
    const double el = (double)a.rows * a.cols * 4, ms = dbl ? 8 : 4;
    if (a.acc) bytes += el * (a.acc_kind == ACC_F32 ? 4 : 8);
    for (int t = 0; t < 4; t++)
      if (a.aux[t]) bytes += el * ms;
    for (int o = 0; o < a.nout; o++) {
      if (a.out[o].mp) bytes += el * ms;
      if (a.out[o].s16.a) bytes += el * 2 * a.out[o].s16.levels;
      if (a.out[o].s16.b) bytes += el * 2 * a.out[o].s16.levels;
    }
    timed(c, EV_EW, 0, 0, bytes, [&] { return launch_combine(a, c->st, nullptr); });
    if (with_partials) {
      double* red = (double*)buf(c, "red", sizeof(double) * 8);
      timed(c, EV_EW, 0, 0, 24.0 * blocks,
            [&] { return launch_reduce_partials(partials, blocks, 3, red + red_slot, c->st); });
    }
  }

  // ---------------- shape helpers ----------------
  // Each product is followed by its combine pass `a` (built with no
  // accumulator): prod_run fuses the two when it can.
  // R-products (polynomials in R) take rmode and Lr split terms.
  void rprod_run(const QMat& P, const QMat& Q, const CombineArgs& a) {
    Lcur = Lr;
    prod_run(P, Q, rmode >= 0 ? rmode : (L == 0 ? PM_F64 : PM_TC), a);
  }
  // X-products take the mode of the phase (xmode).
  // Residual product: right A*Y (m x m), left Y*A (n x n).
  void res_run(const QMat& Y, const CombineArgs& a, bool with_partials, int red_slot) {
    Lcur = Lx;
    if (left) prod_run(Y, A, xmode, a, with_partials, red_slot);
    else prod_run(A, Y, xmode, a, with_partials, red_slot);
  }
  // Apply a side polynomial T (s x s) to Y (n x m): right Y*T, left T*Y.
  void apply_run(const QMat& Y, const QMat& T, const CombineArgs& a, bool with_partials = false) {
    Lcur = Lx;
    const int save = xS;
    if (xmode == PM_EMU && !dbl) xS = xSu;
    else if (xmode == PM_EMU && dbl && xSp > 0) xS = xSp;
    if (left) prod_run(T, Y, xmode, a, with_partials);
    else prod_run(Y, T, xmode, a, with_partials);
    xS = save;
  }
  const char* tform() const { return left ? "fa" : "fb"; }
  QMat sq(const char* name, bool a, bool b) { return mat(c, name, s, s, MST_F | MST_D, a, b); }
  QMat big(const char* name) { return mat(c, name, n, m, MST_F | MST_D, true, true); }

  // R = I - (residual product of Y).
  // norm: also reduce ||R||_F^2 into red[4] (the iteration's own residual).
  QMat residual(const QMat& Y, const char* name, const char* forms, bool norm = false) {
    if (pre_res && strcmp(name, "R") == 0) {  // computed ahead of the step for X[cur]
      pre_res = false;
      return pre_R;
    }
    QMat R = sq(name, strchr(forms, 'a') != nullptr, strchr(forms, 'b') != nullptr);
    CombineArgs a = base_args(s, s, nullptr);
    out(a, R, forms, -1.0, 1.0);
    res_run(Y, a, norm, 4);
    if (strcmp(name, "R") == 0) {
      const bool exact = dbl && (xmode == PM_F64 || (xmode == PM_EMU && xS >= 8));
      res_cur = exact && &Y == &X[cur] ? cur : -1;
      if (res_cur >= 0) res_R = R;
    }
    return R;
  }

  // X_{j+1} = base + (Y T | T Y) (master + both forms) with the stop-test
  // partials against X[cur].
  void apply_update(const QMat& Y, const QMat& T, const QMat& base) {
    QMat& Xn = X[cur ^ 1];
    CombineArgs a = base_args(n, m, nullptr);
    aux(a, 0, X[cur]);
    aux(a, 1, base);
    OutSpec& o = out(a, Xn, "fab", 1.0);
    o.caux[1] = 1.0;  // + base (aux 0 = X_j is only the reference of the norm)
    apply_run(Y, T, a, true);
  }

  // ---------------- one iteration of each method ----------------
  void step_ns() {
    QMat R = residual(X[cur], "R", tform(), true);
    apply_update(X[cur], R, X[cur]);
  }

  void step_qsai(double b1, double b2) {
    QMat R = residual(X[cur], "R", "fab", true);
    QMat R2 = sq("R2", true, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      out(a, R2, "fab", 1.0);
      rprod_run(R, R, a);
    }
    QMat R4 = sq("R4", false, false), Fa = sq("Fa", true, false), Fb = sq("Fb", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R2);
      out(a, R4, "f", 1.0);
      out(a, Fa, "fa", 1.0).caux[0] = b1;
      out(a, Fb, "fb", 1.0).caux[0] = b2;
      rprod_run(R2, R2, a);
    }
    QMat q = sq("q", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R2);
      aux(a, 1, R4);
      OutSpec& o = out(a, q, "fb", 1.0);
      o.caux[0] = b1 + b2;
      o.caux[1] = 2.0;
      rprod_run(Fa, Fb, a);
    }
    QMat t = sq("t", left, !left);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R);
      aux(a, 1, q);
      OutSpec& o = out(a, t, tform(), 1.0);
      o.caux[0] = 1.0;
      o.caux[1] = 1.0;
      rprod_run(R, q, a);
    }
    apply_update(X[cur], t, X[cur]);
  }

  void step_qhpi19(const double* k) {
    // k: a1 a2 a3 b1 b2 c1 c2 d1 d2 d3 e1 e2
    const double c1 = k[5], c2 = k[6], d1 = k[7], d2 = k[8], d3 = k[9], e1 = k[10], e2 = k[11];
    QMat R = residual(X[cur], "R", "fab", true);
    QMat R2 = sq("R2", true, true), S = sq("S", true, false);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R);
      out(a, R2, "fab", 1.0);
      out(a, S, "fa", 1.0).caux[0] = 1.0;
      rprod_run(R, R, a);
    }
    QMat R4 = sq("R4", false, false), Fa = sq("Fa", true, false), Fb = sq("Fb", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R2);
      out(a, R4, "f", 1.0);
      out(a, Fa, "fa", 1.0).caux[0] = d1;
      out(a, Fb, "fb", 1.0).caux[0] = d2;
      rprod_run(R2, R2, a);
    }
    QMat u = sq("u", false, false), v = sq("v", true, false), w = sq("w", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R2);
      aux(a, 1, R4);
      OutSpec& ou = out(a, u, "f", 1.0);
      ou.caux[0] = d1 + d2;
      ou.caux[1] = 2.0;
      OutSpec& ov = out(a, v, "fa", 1.0);
      ov.caux[0] = d1 + d2 + d3;
      ov.caux[1] = 2.0;
      OutSpec& ow = out(a, w, "fb", 1.0);
      ow.caux[0] = d1 + d2 + e1;
      ow.caux[1] = 2.0 + e2;
      rprod_run(Fa, Fb, a);
    }
    QMat g = sq("g", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, u);
      aux(a, 1, R2);
      aux(a, 2, R4);
      OutSpec& o = out(a, g, "fb", 1.0);
      o.caux[0] = 2.0;
      o.caux[1] = d3 + e1 + c1;
      o.caux[2] = e2 + c2;
      rprod_run(v, w, a);
    }
    QMat t = sq("t", left, !left);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, S);
      out(a, t, tform(), 1.0).caux[0] = 1.0;
      rprod_run(S, g, a);
    }
    apply_update(X[cur], t, X[cur]);
  }

  // Unfactorized hyperpower iteration of order k (Definition 1):
  // X_{j+1} = X (I + R + ... + R^(k-1)) = X + X t, t = R + R^2 + ... + R^(k-1)
  // by Horner's rule h <- R + R h from h = R: k - 2 R-products, then the
  // update; k products per iteration with the residual.
  void step_qhpim(int k) {
    QMat R = residual(X[cur], "R", k == 2 ? tform() : "fab", true);
    QMat H[2] = {sq("h0", true, true), sq("h1", true, true)};
    const QMat* h = &R;
    for (int i = 2; i < k; i++) {
      QMat& hn = H[i & 1];
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R);
      out(a, hn, i == k - 1 ? tform() : "fb", 1.0).caux[0] = 1.0;
      rprod_run(R, *h, a);
      h = &hn;
    }
    apply_update(X[cur], *h, X[cur]);
  }

  // QRAPID correction  W + Y (I - A W)  (right) / W + (I - W A) Y (left) into Z.
  void rapid_correct(const QMat& W, const QMat& Y, QMat& Z, bool is_final) {
    QMat E = residual(W, "E", tform());
    if (is_final) {
      apply_update(Y, E, W);
      return;
    }
    CombineArgs a = base_args(n, m, nullptr);
    aux(a, 0, W);
    out(a, Z, "fab", 1.0).caux[0] = 1.0;
    apply_run(Y, E, a);
  }

  void step_qrapid(int N) {
    QMat R = residual(X[cur], "R", "fab", true);
    QMat R2 = sq("R2", false, true);
    {
      CombineArgs a = base_args(s, s, nullptr);
      out(a, R2, "fb", 1.0);
      rprod_run(R, R, a);
    }
    QMat tU = sq("t", left, !left);
    {
      CombineArgs a = base_args(s, s, nullptr);
      aux(a, 0, R);
      aux(a, 1, R2);
      OutSpec& o = out(a, tU, tform(), 0.25);
      o.caux[0] = 1.0;
      o.caux[1] = 1.0;
      rprod_run(R, R2, a);
    }
    QMat Zb[3] = {big("Z0"), big("Z1"), big("Z2")};
    {  // U = X + X tU
      CombineArgs a = base_args(n, m, nullptr);
      aux(a, 0, X[cur]);
      out(a, Zb[0], "fab", 1.0).caux[0] = 1.0;
      apply_run(X[cur], tU, a);
    }
    rapid_correct(Zb[0], X[cur], Zb[1], false);  // V = U + X (I - A U)
    int y = 0, w = 1;                             // Y_0 = U, W_0 = V
    for (int it = 1; it <= N; it++) {
      const int z = 3 - y - w;
      rapid_correct(Zb[w], Zb[y], Zb[z], false);
      y = w;
      w = z;
    }
    rapid_correct(Zb[w], X[cur], Zb[w], true);  // X_{j+1} = Z + X (I - A Z)
  }

  // Removes the component of X that rounding puts outside the ranges of the
  // pseudoinverse.  For full-rank rectangular A the iteration corrects only
  // what its residual sees: with a tall A (left form, residual I - XA) the
  // part of X acting on range(A)^perp is invisible, with a wide A (right
  // form) the part of X's range in null(A) is.  X (AX)^H = X X^H A^H (tall)
  // and (XA)^H X = A^H X^H X (wide) equal A^dagger for X = A^dagger and
  // remove such a component E to first order (it becomes O(E^2)).  FP64
  // masters, FP64-accurate products.
  void range_projection() {
    const bool tall = m > n;
    const int k = tall ? n : m;
    QMat XH = mat(c, "XH", m, n, MST_D, false, false), AH = mat(c, "AHp", n, m, MST_D, false, false);
    QMat G = mat(c, "G", k, k, MST_D, false, false);
    ck(c, launch_init_x0(dview(X[cur]), n, m, 1.0, XH.d, c->st), "adjoint X");
    ck(c, launch_init_x0(dview(A), m, n, 1.0, AH.d, c->st), "adjoint A");
    const int L0 = L, xm0 = xmode, xs0 = xS;
    L = 0;
    xS = 8;
    {
      Acc g = tall ? prod(X[cur], XH, PM_EMU) : prod(XH, X[cur], PM_EMU);
      CombineArgs a = base_args(k, k, &g);
      out(a, G, "f", 1.0);
      run(a);
    }
    Acc y = tall ? prod(G, AH, PM_EMU) : prod(AH, G, PM_EMU);
    CombineArgs a = base_args(n, m, &y);
    out(a, X[cur ^ 1], "f", 1.0);
    run(a);
    cur ^= 1;
    L = L0;
    xmode = xm0;
    xS = xs0;
  }

  // Writes the BF16 operand forms of a matrix from the master of the phase.
  void forms(const QMat& M, bool a, bool b) {
    if (L == 0) return;
    CombineArgs args = base_args(M.rows, M.cols, nullptr);
    aux(args, 0, M);
    OutSpec& o = out(args, M, a && b ? "ab" : (a ? "a" : "b"), 0.0);
    o.caux[0] = 1.0;
    run(args);
  }
};

double hpi19_k[12];
void init_constants() {
  const double s93 = std::sqrt(93.0);
  const double r = std::sqrt(27.0 - 2.0 * s93);
  hpi19_k[0] = 5.0 / 496.0 * (31.0 + s93);    // a1
  hpi19_k[1] = (3.0 + s93) / 8.0;             // a2
  hpi19_k[2] = 0.5;                           // a3
  hpi19_k[3] = 5.0 / 496.0 * (31.0 - s93);    // b1
  hpi19_k[4] = (3.0 - s93) / 8.0;             // b2
  hpi19_k[5] = 3.0 / 8.0;                     // c1
  hpi19_k[6] = 321.0 / 1984.0;                // c2
  hpi19_k[7] = 0.25 * (1.0 + r);              // d1
  hpi19_k[8] = 0.25 * (1.0 - r);              // d2
  hpi19_k[9] = (5.0 * s93 - 93.0) / 496.0;    // d3
  hpi19_k[10] = -(93.0 + 5.0 * s93) / 496.0;  // e1
  hpi19_k[11] = -s93 / 4.0;                   // e2
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copies a caller matrix (device or host planes) into a workspace FP64 master.
void load_planes(qpinv_ctx* c, const double* const src[4], long ld, int rows, int cols, const QMat& dst) {
  for (int p = 0; p < 4; p++) {
    const bool dev = is_device_ptr(src[p]);
    ck(c,
       cudaMemcpy2DAsync(dst.d.p + p * dst.d.ps, sizeof(double) * dst.d.ld, src[p], sizeof(double) * ld,
                         sizeof(double) * cols, rows, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st),
       "copy in");
  }
}
void store_planes(qpinv_ctx* c, const QMat& src, double* const dst[4], long ld, int rows, int cols) {
  for (int p = 0; p < 4; p++) {
    const bool dev = is_device_ptr(dst[p]);
    ck(c,
       cudaMemcpy2DAsync(dst[p], sizeof(double) * ld, src.d.p + p * src.d.ps, sizeof(double) * src.d.ld,
                         sizeof(double) * cols, rows, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st),
       "copy out");
  }
}

// ||scale P + diag I - Q||_F^2 (Q optional; diag on plane s).
double fro2(qpinv_ctx* c, const Planes<const double>& P, const Planes<const double>* Q, int rows, int cols,
            double* bad = nullptr, double scale = 1.0, double diag = 0.0) {
  int blocks = 0;
  double* part = (double*)buf(c, "fro_part", sizeof(double) * 2 * 1024 + 64);
  double* red = (double*)buf(c, "fro_red", sizeof(double) * 4);
  timed(c, EV_EW, 0, 0, (double)rows * cols * 32 * (Q ? 2 : 1),
        [&] { return launch_fro2_partials(P, Q, rows, cols, part, c->st, &blocks, scale, diag); });
  timed(c, EV_EW, 0, 0, 16.0 * blocks, [&] { return launch_reduce_partials(part, blocks, 2, red, c->st); });
  double h[2];
  read_back(c, red, 2, h);
  if (bad) *bad = h[1];
  return h[0];
}

double antiherm2(qpinv_ctx* c, const QMat& M) {
  int blocks = ((M.rows + 31) / 32) * ((M.rows + 31) / 32);
  double* part = (double*)buf(c, "ah_part", sizeof(double) * (size_t)blocks + 64);
  double* red = (double*)buf(c, "fro_red", sizeof(double) * 4);
  timed(c, EV_EW, 0, 0, (double)M.rows * M.rows * 64,
        [&] { return launch_antiherm_partials(dview(M), M.rows, part, c->st, &blocks); });
  timed(c, EV_EW, 0, 0, 8.0 * blocks, [&] { return launch_reduce_partials(part, blocks, 1, red, c->st); });
  double h;
  read_back(c, red, 1, &h);
  return h;
}

// Penrose residuals (Sec. 4) for A (m x n) and X (n x m) FP64 masters, with
// FP64-accurate products (mode PM_F64 or PM_EMU with 8 slices) and FP64 norms.
// Rgiven: I - AX (right) or I - XA (left, given_left) of this X, already
// formed with FP64 masters and FP64-accurate products (or null): that side's
// product is not formed again (the norms do not depend on the sign).
void penrose(qpinv_ctx* c, const QMat& A, const QMat& X, int mode, double* E, double* Er, long long* gemms,
             const QMat* Rgiven = nullptr, bool given_left = false) {
  // E1 = ||AXA - A|| = ||(AX - I) A||, E2 = ||XAX - X|| = ||(XA - I) X||,
  // E3 = ||(AX)^H - AX|| = ||Rr^H - Rr|| (Rr = AX - I), E4 likewise with XA.
  // Every product is FP64-accurate: AX - I is not small when A is
  // rectangular or rank deficient (it is -1 on the complement of the range).
  const int m = A.rows, n = A.cols;
  Solver S;
  S.c = c;
  S.dbl = true;
  S.L = 0;
  QMat Rr = mat(c, "pRr", m, m, MST_D, false, false), Rl = mat(c, "pRl", n, n, MST_D, false, false);
  QMat E1m = mat(c, "pE1", m, n, MST_D, false, false), E2m = mat(c, "pE2", n, m, MST_D, false, false);
  auto product = [&](const QMat& P, const QMat& Q, QMat& Out, int slices, double diag) {
    S.xS = slices;
    Solver::Acc acc = S.prod(P, Q, mode);
    CombineArgs a = S.base_args(Out.rows, Out.cols, &acc);
    S.out(a, Out, "f", 1.0, diag);
    S.run(a);
  };
  double sr = 1.0, sl = 1.0;  // Rr = sr (AX - I), Rl = sl (XA - I)
  if (Rgiven && !given_left) {
    Rr = *Rgiven;
    sr = -1.0;
  } else {
    product(A, X, Rr, 8, -1.0);
  }
  if (Rgiven && given_left) {
    Rl = *Rgiven;
    sl = -1.0;
  } else {
    product(X, A, Rl, 8, -1.0);
  }
  Planes<const double> a = dview(A), x = dview(X);
  const double fa = std::sqrt(fro2(c, a, nullptr, m, n)), fx = std::sqrt(fro2(c, x, nullptr, n, m));
  // ||R Q||_F with R = AX - I or XA - I.  When R is small (square
  // full-rank A) the product needs only a few digits relative to ||R|| ||Q||:
  // 6 slices are accepted when the result exceeds 1e3 times a bound on their
  // truncation error, 2^(10 - 7S) K ||R||_F ||Q||_F; otherwise 8 slices.
  auto outer = [&](const QMat& R, const QMat& Q, QMat& Out, double fq) {
    const int rows = R.rows, cols = Q.cols, K = R.cols;
    if (mode == PM_EMU) {
      const double fr = std::sqrt(fro2(c, dview(R), nullptr, R.rows, R.cols));
      if (fr <= 1e-3) {
        product(R, Q, Out, 6, 0.0);
        const double e = std::sqrt(fro2(c, dview(Out), nullptr, rows, cols));
        if (e >= 1e3 * std::ldexp(1.0, 10 - 7 * 6) * K * fr * fq) return e;
      }
    }
    product(R, Q, Out, 8, 0.0);
    return std::sqrt(fro2(c, dview(Out), nullptr, rows, cols));
  };
  E[0] = outer(Rr, A, E1m, fa);
  E[1] = outer(Rl, X, E2m, fx);
  if (gemms) *gemms += S.gemms;
  E[2] = std::sqrt(antiherm2(c, Rr));
  E[3] = std::sqrt(antiherm2(c, Rl));
  // ||AX||_F^2 = ||Rr||^2 + 2 Re tr(Rr) + m: computed directly from
  // AX = sr Rr + I instead (each element formed in registers, as a combine
  // pass would store it), and XA = sl Rl + I likewise
  const double nr[4] = {fa, fx, std::sqrt(fro2(c, dview(Rr), nullptr, m, m, nullptr, sr, 1.0)),
                        std::sqrt(fro2(c, dview(Rl), nullptr, n, n, nullptr, sl, 1.0))};
  for (int t = 0; t < 4; t++) Er[t] = nr[t] > 0 ? E[t] / nr[t] : E[t];
}

int fail(qpinv_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// Learned-alpha features of an m x n matrix whose FP32 master is A.f.
void features_of(qpinv_ctx* c, const QMat& A, double fro2, double n1, double ninf, float* feat, double* theta1) {
  const int m = A.rows, n = A.cols;
  float* sc = (float*)buf(c, "alpha.lanczos", sizeof(float) * (size_t)alpha_feature_scratch_floats(m, n) + 256);
  double* ds = (double*)buf(c, "alpha.dot", sizeof(double) * 32);
  const int steps = n < 16 ? n : 16;
  ck(c, alpha_features(fview(A), m, n, fro2, n1, ninf, sc, ds, c->h_pin, c->st, feat, theta1), "alpha features");
  c->stats.kernel_launches += 7 * steps - 1;
}

// Spectral radius of a square FP32 matrix by 24 power-iteration steps.
double spec_radius_est(qpinv_ctx* c, const QMat& M) {
  const int steps = 24;
  float* sc = (float*)buf(c, "rho.v", sizeof(float) * 8 * (size_t)M.rows + 256);
  double* ds = (double*)buf(c, "rho.d", sizeof(double) * power_radius_doubles(M.rows, steps));
  double rho = 0.0;
  const long long before = g_kernel_launches;
  ck(c, power_radius(fview(M), M.rows, steps, sc, ds, c->h_pin, c->st, &rho), "spectral radius estimate");
  c->stats.kernel_launches += g_kernel_launches - before;
  return rho;
}

// Network prediction y = log(alpha * theta_1) for one feature vector.
double predict_one(qpinv_ctx* c, const float* feat) {
  const int NW = alpha_nweights();
  float* dW = (float*)buf(c, "alpha.W", sizeof(float) * NW);
  float* dX = (float*)buf(c, "alpha.x1", sizeof(float) * 32);
  float* sc = (float*)buf(c, "alpha.s1", sizeof(float) * alpha_scratch_floats(1) + 64);
  float* dy = (float*)buf(c, "alpha.y1", sizeof(float) * 4);
  ck(c, cudaMemcpyAsync(dW, c->alpha_w.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, c->st), "weights");
  ck(c, cudaMemcpyAsync(dX, feat, sizeof(float) * 32, cudaMemcpyHostToDevice, c->st), "features");
  timed(c, EV_EW, 0, 0, 0, [&] { return alpha_forward(dW, dX, 1, sc, dy, c->st); });
  float y = 0.f;
  ck(c, cudaMemcpyAsync(c->h_pin, dy, sizeof(float), cudaMemcpyDeviceToHost, c->st), "read");
  ck(c, cudaStreamSynchronize(c->st), "sync");
  memcpy(&y, c->h_pin, sizeof(float));
  return (double)y;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

void qpinv_default_options(qpinv_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = QPINV_PREC_MIXED;
  o->split_level = 0;
  o->polish_iters = 2;
  o->alpha_mode = QPINV_ALPHA_SAFE;
  o->alpha_user = 0.0;
  o->qrapid_N = 5;
  o->side = QPINV_SIDE_AUTO;
  o->stop_rule = QPINV_STOP_REL_PLATEAU;
  o->penrose = 1;
  o->profile = 0;
  o->batched_tile = -1;
  o->hyper_order = 19;
  o->fuse_epilogue = 1;
  o->emu_pair = -1;
  o->tc_broad = -1;
}

static int check_opts(const qpinv_options* o) {
  if (o->precision < 0 || o->precision > 3) return 0;
  if (o->split_level < 0 || o->split_level > 3) return 0;
  if (o->polish_iters < 0 || o->polish_iters > 100) return 0;
  if (o->alpha_mode < 0 || o->alpha_mode > 4) return 0;
  if (o->alpha_mode == QPINV_ALPHA_USER && !(o->alpha_user > 0.0 && std::isfinite(o->alpha_user))) return 0;
  if (o->qrapid_N < 0 || o->qrapid_N > 30) return 0;
  if (o->side < 0 || o->side > 2 || o->stop_rule < 0 || o->stop_rule > 1) return 0;
  if (o->batched_tile < -1 || o->batched_tile >= qp::BATCH_TILES) return 0;
  if (o->hyper_order < 2 || o->hyper_order > 64) return 0;
  if (o->fuse_epilogue < 0 || o->fuse_epilogue > 1) return 0;
  if (o->emu_pair < -1 || o->emu_pair > 1) return 0;
  if (o->tc_broad < -1 || o->tc_broad > 1) return 0;
  return 1;
}

int qpinv_init(qpinv_ctx** out, int device, const qpinv_options* opt) {
  if (!out) return QPINV_E_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return QPINV_E_CUDA;
  }
  if (opt && !check_opts(opt)) return QPINV_E_INVALID;
  qpinv_ctx* c = new qpinv_ctx();
  c->device = device;
  qpinv_default_options(&c->opt);
  if (opt) c->opt = *opt;
  memset(&c->stats, 0, sizeof(c->stats));
  const char* tr = getenv("QPINV_TRACE");
  c->trace = tr && tr[0] == '1';
  DeviceGuard g(device);
  if (cudaMalloc(&c->d_err, sizeof(int)) != cudaSuccess || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_pin, sizeof(double) * 64) != cudaSuccess) {
    cudaGetLastError();
    qpinv_free(c);
    return QPINV_E_NOMEM;
  }
  init_constants();
  *out = c;
  return QPINV_OK;
}

int qpinv_set_options(qpinv_ctx* c, const qpinv_options* opt) {
  if (!c || !opt) return QPINV_E_INVALID;
  if (!check_opts(opt)) return fail(c, QPINV_E_INVALID, "invalid options");
  c->opt = *opt;
  return QPINV_OK;
}

void qpinv_free(qpinv_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  flush_events(c);
  for (auto& kv : c->bufs)
    if (kv.second.p) cudaFree(kv.second.p);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  if (c->d_err) cudaFree(c->d_err);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  for (void* p : c->bh_buf)
    if (p) cudaFreeHost(p);
  if (c->bmaps_host) cudaFreeHost(c->bmaps_host);
  if (c->bgraph.exec) cudaGraphExecDestroy(c->bgraph.exec);
  if (c->bgraph.stream) cudaStreamDestroy(c->bgraph.stream);
  delete c;
}

const char* qpinv_last_error(qpinv_ctx* c) { return c ? c->err.c_str() : "null context"; }

int qpinv_get_stats(qpinv_ctx* c, qpinv_stats* s) {
  if (!c || !s) return QPINV_E_INVALID;
  DeviceGuard g(c->device);
  flush_events(c);
  *s = c->stats;
  return QPINV_OK;
}

int qpinv_reset_stats(qpinv_ctx* c) {
  if (!c) return QPINV_E_INVALID;
  DeviceGuard g(c->device);
  flush_events(c);
  memset(&c->stats, 0, sizeof(c->stats));
  return QPINV_OK;
}

static bool planes_ok(const double* const P[4]) {
  if (!P) return false;
  for (int t = 0; t < 4; t++)
    if (!P[t]) return false;
  return true;
}

int qpinv_solve(qpinv_ctx* c, void* stream, int m, int n, const double* const A[4], long lda, qpinv_method method,
                double tol, int max_iter, double* const X[4], long ldx, qpinv_result* out) {
  if (!c) return QPINV_E_INVALID;
  if (m <= 0 || n <= 0 || lda < n || ldx < m || !planes_ok(A) || !planes_ok((const double* const*)X) ||
      max_iter < 1 || !(tol >= 0.0) || (int)method < 0 || (int)method > 4)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  const auto t_start = std::chrono::steady_clock::now();
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  const qpinv_options& o = c->opt;
  qpinv_result res;
  memset(&res, 0, sizeof(res));
  try {
    const bool fp64 = o.precision == QPINV_PREC_FP64;
    // A residual forced onto the larger side has eigenvalue 1 on the
    // complement of the range, where rounding noise grows by the method's
    // order each step (as for rank-deficient A): such solves run with
    // FP64-accurate products throughout.
    const bool wrong_side = (o.side == QPINV_SIDE_RIGHT && m > n) || (o.side == QPINV_SIDE_LEFT && m < n);
    bool emu = o.precision == QPINV_PREC_EMU || (!fp64 && wrong_side);
    if (!fp64 && !tc_supported()) return fail(c, QPINV_E_UNSUPPORTED, "tcgen05 path needs an sm_103 device");
    long long gemms_before = 0;
    // A solve started from a learned alpha that does not contract is
    // restarted once from the safe alpha (north of Thm. 1's bound the
    // iteration diverges along the top singular direction, which the
    // features' Lanczos estimate theta_1 <= sigma_1^2 may have missed).
    bool force_safe = false;
    // A MIXED solve whose result fails the Penrose check is repeated with
    // FP64-accurate products: rank-deficient A (and A beyond the tensor-core
    // phase's conditioning reach) amplifies BF16 rounding in the complement of
    // the range by the method's order every step.
    for (int attempt = 0;; attempt++) {
    res.precision = fp64 ? QPINV_PREC_FP64 : emu ? QPINV_PREC_EMU : o.precision;
    Solver S;
    S.c = c;
    S.m = m;
    S.n = n;
    S.left = o.side == QPINV_SIDE_LEFT || (o.side == QPINV_SIDE_AUTO && m > n);
    S.s = S.left ? n : m;
    res.side = S.left ? QPINV_SIDE_LEFT : QPINV_SIDE_RIGHT;
    S.A = mat(c, "A", m, n, MST_D | MST_F, !S.left, S.left);
    load_planes(c, A, lda, m, n, S.A);
    Planes<const double> a = dview(S.A);
    double bad = 0.0;
    const double a_f2 = fro2(c, a, nullptr, m, n, &bad);
    if (bad > 0.0 || !std::isfinite(a_f2)) return fail(c, QPINV_E_NONFINITE, "A contains NaN or Inf");
    // ---- norms and alpha (Thm. 1) ----
    double* rs = (double*)buf(c, "rowsum", sizeof(double) * (size_t)(m + n) + 64);
    double* mx = (double*)buf(c, "maxes", sizeof(double) * 4);
    timed(c, EV_EW, 0, 0, 64.0 * m * n, [&] { return launch_abs_sums(a, m, n, rs, rs + m, (double*)buf(c, "colpart", sizeof(double) * (size_t)COL_SCRATCH(n) + 64), c->st); });
    timed(c, EV_EW, 0, 0, 8.0 * m, [&] { return launch_max(rs, m, mx, c->st); });
    timed(c, EV_EW, 0, 0, 8.0 * n, [&] { return launch_max(rs + m, n, mx + 1, c->st); });
    double hm[2];
    read_back(c, mx, 2, hm);
    const double norm_inf = hm[0], norm_1 = hm[1];
    const double a2est = std::sqrt(norm_1 * norm_inf);  // >= sigma_1
    double alpha = 0.0;
    int amode = o.alpha_mode;
    if (amode == QPINV_ALPHA_LEARNED) {
      // Network prediction, accepted only if it passes Thm. 1's contraction
      // condition alpha sigma_1^2 < 2 with a 5% margin for the Lanczos
      // estimate theta_1 <= sigma_1^2; otherwise the safe alpha is used.
      // The solve itself then checks that the residual contracts.
      amode = QPINV_ALPHA_SAFE;
      res.alpha_fallback = 1;
      if (!force_safe && !c->alpha_w.empty() && a_f2 > 0.0) {
        ck(c, launch_f64_to_f32(a, m, n, S.A.f, c->st), "A to fp32");
        float feat[32];
        double theta1 = 0.0;
        features_of(c, S.A, a_f2, norm_1, norm_inf, feat, &theta1);
        const double y = predict_one(c, feat);
        const double al = std::exp(y) / theta1;
        if (std::isfinite(al) && al > 0.0 && al * theta1 * 1.05 < 2.0) {
          alpha = al;
          amode = QPINV_ALPHA_LEARNED;
          res.alpha_fallback = 0;
        }
      }
    }
    if (amode == QPINV_ALPHA_LEARNED) {
      // alpha set above
    } else if (a_f2 == 0.0) {
      alpha = 0.0;
    } else if (amode == QPINV_ALPHA_SAFE) {
      alpha = 1.0 / (norm_1 * norm_inf);
    } else if (amode == QPINV_ALPHA_FRO) {
      alpha = 1.0 / a_f2;
    } else if (amode == QPINV_ALPHA_USER) {
      alpha = o.alpha_user;
    } else {  // SPECTRAL: power iteration on A^H A with FP64 matrix-vector products
      QMat AH = mat(c, "AH", n, m, MST_D, false, false);
      ck(c, launch_init_x0(a, m, n, 1.0, AH.d, c->st), "adjoint");
      QMat v = mat(c, "pv", n, 1, MST_D, false, false), w = mat(c, "pw", m, 1, MST_D, false, false);
      std::vector<double> hv(4 * (size_t)n);
      for (int i = 0; i < 4 * n; i++) hv[i] = 1.0 / (1.0 + 0.37 * (i % 7) + 0.11 * i);
      ck(c, cudaMemcpyAsync(v.d.p, hv.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice, c->st), "copy");
      double lam = 0.0;
      Solver P;
      P.c = c;
      P.dbl = true;
      P.L = 0;
      for (int it = 0; it < 300; it++) {
        const double nv = std::sqrt(fro2(c, dview(v), nullptr, n, 1));
        CombineArgs ca = P.base_args(n, 1, nullptr);
        P.aux(ca, 0, v);
        P.out(ca, v, "f", 0.0).caux[0] = 1.0 / nv;
        P.run(ca);
        timed(c, EV_F64, 32.0 * m * n, 32.0 * m * n, 0,
              [&] { return launch_qgemm_f64(m, n, 1, a, dview(v), w.d, c->st); });
        timed(c, EV_F64, 32.0 * m * n, 32.0 * m * n, 0,
              [&] { return launch_qgemm_f64(n, m, 1, dview(AH), dview(w), v.d, c->st); });
        const double lam_new = std::sqrt(fro2(c, dview(v), nullptr, n, 1));
        if (it > 10 && std::fabs(lam_new - lam) <= 1e-13 * lam_new) {
          lam = lam_new;
          break;
        }
        lam = lam_new;
      }
      alpha = 1.0 / lam;
    }
    res.alpha = alpha;
    res.alpha_source = amode;
    // ---- X_0 = alpha A^H (FP64), with the FP32 copies of A and X_0 ----
    S.X[0] = mat(c, "X0", n, m, MST_D | MST_F, true, true);
    S.X[1] = mat(c, "X1", n, m, MST_D | MST_F, true, true);
    S.cur = 0;
    ck(c, launch_init_x0(a, m, n, alpha, S.X[0].d, c->st), "init X0");
    const int Lr = o.split_level ? o.split_level : 2;
    bool polish = fp64 || emu;  // these forms run in their final precision from the start
    if (fp64 || emu) {
      S.dbl = true;
      S.L = 0;
      S.xmode = S.rmode = fp64 ? PM_F64 : PM_EMU;
      S.xS = 8;
    } else {
      S.dbl = false;
      S.L = 3;
      S.Lr = Lr;
      // X-products on 2-term splits for square MIXED solves: at K in the
      // thousands the tensor cores' FP32 accumulation error (about 3e-5
      // relative) already exceeds what a third term would add, and the polish
      // iterations remove the rest.  TC precision keeps 3 terms (its output is
      // the tensor-core iterate), and so does rectangular A, whose
      // out-of-space component starts at the level of the FP32 phase.
      const bool square_mixed = o.precision == QPINV_PREC_MIXED && m == n;
      S.Lx = square_mixed ? 2 : 3;
      S.xSu = square_mixed ? 3 : 4;
      S.L = std::max(S.Lx, Lr);  // BF16 terms the operand forms need: no more are written
      S.xmode = PM_TC;
      ck(c, launch_f64_to_f32(a, m, n, S.A.f, c->st), "A to fp32");
      ck(c, launch_f64_to_f32(dview(S.X[0]), n, m, S.X[0].f, c->st), "X0 to fp32");
      S.forms(S.A, !S.left, S.left);
      S.forms(S.X[0], true, true);
    }
    int polish_done = 0, tc_done = 0;
    double prev_rel = INFINITY, xnorm = std::sqrt(a_f2) * alpha;
    double prev_rnorm = INFINITY;  // ||R_{j-1}||_F (contraction check of a learned alpha)
    bool learned_failed = false;
    res.status = QPINV_NOT_CONVERGED;
    res.iters = 0;
    for (int j = 0; j < max_iter; j++) {
      if (!polish && !emu) {
        // X-products: BF16 splits while their error, amplified by about
        // ||A|| ||X||, stays small; exact 4-slice products beyond.
        const double kappa_est = a2est * xnorm;
        if (kappa_est * 1e-5 > 1e-2) {
          S.xmode = PM_EMU;
          S.xS = 4;
        } else {
          S.xmode = PM_TC;
        }
      }
      // R-products on single BF16 terms while the residual still has
      // unresolved directions (relative step > 0.5): the rounding they leave in
      // t puts resolved directions back at a residual of about 1e-2, which the
      // next step's power of R removes; 2-term splits after (automatic
      // split_level only).
      if (!polish && !emu && o.split_level == 0) S.Lr = prev_rel > 0.5 ? 1 : Lr;
      S.xSp = 0;
      if (o.precision == QPINV_PREC_MIXED && polish && polish_done >= 1) {
        // Later polish steps: form the residual of X_j first.  The step
        // changes X by about ||X t|| <= ||X|| ||t||, ||t|| ~ ||R_j||, so when
        // ||R_j||_F is at the rounding floor of the update (or within the
        // relative tolerance) the step is not taken; otherwise the update
        // product X t needs only enough exact slices for FP64 accuracy of
        // X + X t: 53 + log2(4 ||R_j||_F) bits, plus one slice of guard.
        S.pre_R = S.residual(S.X[S.cur], "R", "fab", true);
        S.pre_res = true;
        double hr[8];
        read_back(c, (const double*)buf(c, "red", sizeof(double) * 8), 6, hr);
        const double rn = std::sqrt(hr[4]);
        const double floor_rel = 0x1p-53 * a2est * xnorm;
        if (c->trace) fprintf(stderr, "qpinv it %d polish residual |R|_F %.3e floor %.3e\n", j, rn, floor_rel);
        if (o.stop_rule != QPINV_STOP_PAPER_ABS && (rn <= tol || rn <= floor_rel)) {
          S.pre_res = false;
          res.status = rn <= tol ? QPINV_CONVERGED : QPINV_PLATEAU;
          res.delta_rel = rn;  // the predicted relative step
          break;
        }
        if (rn > 0.0) {
          const int bits = 53 + (int)std::ceil(std::log2(4.0 * rn));
          S.xSp = std::min(8, std::max(3, (bits + 6) / 7 + 1));
        }
      }
      switch (method) {
        case QPINV_NS: S.step_ns(); break;
        case QPINV_QSAI: S.step_qsai((1.0 + std::sqrt(5.0)) / 2.0, (1.0 - std::sqrt(5.0)) / 2.0); break;
        case QPINV_QRAPID: S.step_qrapid(o.qrapid_N); break;
        case QPINV_QHPIM: S.step_qhpim(o.hyper_order); break;
        default: S.step_qhpi19(hpi19_k); break;
      }
      if (!fp64) check_kernel_error(c);
      double h[8];
      read_back(c, (const double*)buf(c, "red", sizeof(double) * 8), 6, h);
      const double rnorm = std::sqrt(h[4]);  // ||R_j||_F of this step's residual
      const double d = std::sqrt(h[0]), nx = std::sqrt(h[1]);
      if (c->trace)
        fprintf(stderr, "qpinv it %d %s xmode %d xS %d Lr %d delta %.3e |X| %.3e rel %.3e |R|_F %.3e\n", j,
                polish ? "polish" : "tc", S.xmode, S.xS, S.Lr, d, nx, nx > 0 ? d / nx : d, rnorm);
      if (h[2] > 0.0 || !std::isfinite(d) || !std::isfinite(nx)) {
        res.status = QPINV_DIVERGED;
        break;  // X[cur] is the last finite iterate
      }
      if (amode == QPINV_ALPHA_LEARNED) {
        // First-step contraction check (and the next few steps): in exact
        // arithmetic R_{j+1} = R_j^p with the spectrum of R_0 in (-1, 1] when
        // alpha sigma_1^2 < 2, so ||R_j||_F cannot grow; a growth beyond
        // rounding (5 %) while the residual is still O(1)-ish means
        // alpha sigma_1^2 > 2.  Later divergence shows up as DIVERGED.
        if (j <= 4 && rnorm > 1.05 * prev_rnorm && prev_rnorm > 1e-4) {
          learned_failed = true;
          break;
        }
        prev_rnorm = rnorm;
      }
      const double drel = nx > 0 ? d / nx : d;
      res.delta = d;
      res.delta_rel = drel;
      if (polish && !fp64 && !emu) polish_done++;
      else if (!fp64 && !emu) tc_done++;
      bool accept = true, stop = false;
      const bool final_phase = polish || o.precision == QPINV_PREC_TC;  // (FP64 and EMU: polish)
      if (o.stop_rule == QPINV_STOP_PAPER_ABS) {
        if (d < tol && final_phase) stop = true, res.status = QPINV_CONVERGED;
      } else {
        if (drel <= tol && final_phase) {
          stop = true;
          res.status = QPINV_CONVERGED;
        } else if (prev_rel < 1e-3 && drel >= prev_rel && final_phase) {
          stop = true;
          accept = false;
          res.status = QPINV_PLATEAU;
        }
      }
      if (accept) {
        S.cur ^= 1;
        res.iters = j + 1;
        xnorm = nx;
      }
      if (stop) break;
      // Rectangular A: the low-precision phase leaves X with a component
      // outside the pseudoinverse's row (or column) space, of relative size
      // delta ~ 1e-7, that no residual sees.  After the first polish iteration
      // (range part at the FP64 level) an FP64-accurate projection takes it to
      // second order, delta^2 kappa; the range error the projection itself
      // adds (about kappa times the FP64 level) is what the following polish
      // iterations correct.
      if (o.precision == QPINV_PREC_MIXED && m != n && polish && polish_done == 1 && o.polish_iters >= 2)
        S.range_projection();
      if (o.precision == QPINV_PREC_MIXED && !polish) {
        // Leave the tensor-core phase once the step stops shrinking fast or
        // is below the FP32 level: switch to FP64 masters and FP64-accurate
        // X-products for the polish iterations.
        const bool stalled = prev_rel < INFINITY && drel > 0.05 * prev_rel && drel < 1e-2;
        // In exact arithmetic the residual after this step is R_j^p (p the
        // method's order) and after the polish iterations R_j^(p^(1+P)), P =
        // polish_iters.  Leave the tensor-core phase once that is negligible:
        // ||R_j||_F < lim bounds it directly; when the relative step (a cheap
        // proxy for ||R_j||) already predicts it, a power-iteration estimate
        // of the spectral radius of R_j (2 % margin) confirms it, which
        // catches residuals that still have unresolved directions (the step
        // dips between clusters of singular values, while R ~ 1 there).  The
        // 2-norm is not used for that: R is not normal, and after single-term
        // R-products its 2-norm exceeds 1 while the iteration converges.
        const double order = method == QPINV_NS      ? 2.0
                             : method == QPINV_QSAI  ? 10.0
                             : method == QPINV_QRAPID ? 5.0
                             : method == QPINV_QHPIM  ? (double)o.hyper_order
                                                      : 19.0;
        const double expo = std::pow(order, 1.0 + o.polish_iters);
        const double lim = std::pow(1e-20, 1.0 / expo);  // largest ||R_j|| that qualifies
        bool resolved = rnorm < lim;
        if (!resolved && std::pow(drel, order) < 1e-6) {
          const double rho = spec_radius_est(c, mat(c, "R", S.s, S.s, MST_F, false, false));
          resolved = 1.02 * rho < lim;
          if (c->trace) fprintf(stderr, "qpinv it %d rho(R) ~ %.4f (limit %.4f)\n", j, rho, lim);
        }
        if (stalled || resolved || drel < 1e-6 || (o.stop_rule == QPINV_STOP_PAPER_ABS && d < tol)) {
          polish = true;
          S.Lr = Lr;  // polish R-products on the full split, whatever the last step used
          ck(c, launch_f32_to_f64(fview(S.X[S.cur]), n, m, S.X[S.cur].d, c->st), "X to fp64");
          S.dbl = true;
          S.xmode = PM_EMU;
          S.xS = 8;
          prev_rel = INFINITY;  // the plateau rule compares polish steps only with each other
          continue;
        }
      } else if (o.precision == QPINV_PREC_MIXED && polish && polish_done >= o.polish_iters) {
        // After the polish iterations: CONVERGED if the stop rule holds,
        // PLATEAU if the relative step is at the FP64 rounding floor of the
        // update (unit roundoff times sqrt(||A||_1 ||A||_inf) ||X||_F, an
        // upper estimate of the condition number), NOT_CONVERGED otherwise.
        const bool conv = o.stop_rule == QPINV_STOP_PAPER_ABS ? d < tol : drel <= tol;
        const double floor_rel = 0x1p-53 * a2est * nx;
        res.status = conv ? QPINV_CONVERGED : drel <= floor_rel ? QPINV_PLATEAU : QPINV_NOT_CONVERGED;
        if (res.status == QPINV_NOT_CONVERGED) {
          // The last step may have been large only because it corrected the
          // range error of a projection (rectangular A) or the R-product
          // rounding of the first polish step: judge the returned X by the
          // step its residual predicts, as in the polish steps above.  The
          // absolute rule uses the bound ||X t||_F <= ||X||_F r / (1 - r),
          // r = ||R||_F, t = R + R^2 + ... (every method's t is a polynomial
          // in R of this kind with coefficients at most 1 in modulus).
          S.residual(S.X[S.cur], "R", "fab", true);
          double hr[8];
          read_back(c, (const double*)buf(c, "red", sizeof(double) * 8), 6, hr);
          const double rn = std::sqrt(hr[4]);
          const bool next_ok = o.stop_rule == QPINV_STOP_PAPER_ABS ? rn < 1.0 && nx * rn / (1.0 - rn) < tol
                                                                   : rn <= tol;
          if (next_ok) res.status = QPINV_CONVERGED;
          else if (rn <= floor_rel) res.status = QPINV_PLATEAU;
        }
        break;
      }
      prev_rel = drel;
    }
    if (amode == QPINV_ALPHA_LEARNED && !force_safe &&
        (learned_failed || res.status == QPINV_DIVERGED || res.status == QPINV_NOT_CONVERGED)) {
      if (c->trace) fprintf(stderr, "qpinv: learned alpha %.6e did not contract; restart from the safe alpha\n", alpha);
      gemms_before += S.gemms;
      force_safe = true;
      continue;
    }
    res.tc_iters = tc_done;
    res.polish_iters = polish_done;
    if (!S.dbl) {
      ck(c, launch_f32_to_f64(fview(S.X[S.cur]), n, m, S.X[S.cur].d, c->st), "X to fp64");
      S.dbl = true;
    }
    // TC precision (no polish iterations): the projection is the last step.
    if (o.precision == QPINV_PREC_TC && m != n && res.status != QPINV_DIVERGED) S.range_projection();
    QMat& Xf = S.X[S.cur];
    if (o.penrose) {
      const bool reuse = S.res_cur == S.cur;
      penrose(c, S.A, Xf, fp64 ? PM_F64 : PM_EMU, res.E, res.E_rel, nullptr, reuse ? &S.res_R : nullptr, S.left);
      if (reuse) c->stats.penrose_reused++;
      if (!fp64) check_kernel_error(c);
    }
    res.gemms = gemms_before + S.gemms;
    if (c->trace)
      fprintf(stderr, "qpinv: attempt %d precision %d status %d iters %d E1_rel %.3e\n", attempt, res.precision,
              res.status, res.iters, res.E_rel[0]);
    // The stated tolerance of an FP64-polished result is E1/||A|| <= 1e-10;
    // where the mixed schedule works it lands at 1e-11 .. 1e-14, so a result
    // above 1e-9 is a failure of the schedule (rank deficiency, or a
    // rectangular A whose complement error the projection did not reach).
    if (o.precision == QPINV_PREC_MIXED && !emu && o.penrose && !(res.E_rel[0] <= 1e-9)) {
      gemms_before = res.gemms;
      emu = true;
      continue;
    }
    store_planes(c, Xf, X, ldx, n, m);
    break;
    }
    ck(c, cudaStreamSynchronize(c->st), "stream sync");
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  res.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (out) *out = res;
  return QPINV_OK;
}

int qpinv_qgemm(qpinv_ctx* c, void* stream, int m, int k, int n, const double* const A[4], long lda,
                const double* const B[4], long ldb, double* const C[4], long ldc, int precision, int split_level) {
  if (!c) return QPINV_E_INVALID;
  if (m <= 0 || n <= 0 || k < 0 || lda < k || ldb < n || ldc < n || !planes_ok(A) || !planes_ok(B) ||
      !planes_ok((const double* const*)C) ||
      (precision != QPINV_PREC_FP64 && precision != QPINV_PREC_TC && precision != QPINV_PREC_EMU) ||
      (precision == QPINV_PREC_TC && (split_level < 1 || split_level > 3)) ||
      (precision == QPINV_PREC_EMU && (split_level < 2 || split_level > 8)))
    return fail(c, QPINV_E_INVALID, "invalid argument");
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    if (precision != QPINV_PREC_FP64 && !tc_supported())
      return fail(c, QPINV_E_UNSUPPORTED, "tcgen05 path needs an sm_103 device");
    const int kk = k > 0 ? k : 1;
    QMat a = mat(c, "gA", m, kk, MST_D, precision == QPINV_PREC_TC, false);
    QMat b = mat(c, "gB", kk, n, MST_D, false, precision == QPINV_PREC_TC);
    QMat cc = mat(c, "gC", m, n, MST_D, false, false);
    if (k == 0) {
      ck(c, cudaMemsetAsync(cc.d.p, 0, sizeof(double) * 4 * cc.d.ps, c->st), "memset");
    } else {
      load_planes(c, A, lda, m, k, a);
      load_planes(c, B, ldb, k, n, b);
      Solver S;
      S.c = c;
      S.dbl = true;
      S.L = precision == QPINV_PREC_TC ? split_level : 0;
      S.Lcur = split_level;
      S.xS = split_level;
      if (precision == QPINV_PREC_TC) {
        S.forms(a, true, false);
        S.forms(b, false, true);
      }
      Solver::Acc acc = S.prod(a, b, precision == QPINV_PREC_FP64 ? PM_F64 : (precision == QPINV_PREC_TC ? PM_TC : PM_EMU));
      S.L = 0;
      CombineArgs args = S.base_args(m, n, &acc);
      S.out(args, cc, "f", 1.0);
      S.run(args);
      if (precision != QPINV_PREC_FP64) check_kernel_error(c);
    }
    store_planes(c, cc, C, ldc, m, n);
    ck(c, cudaStreamSynchronize(c->st), "stream sync");
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_penrose(qpinv_ctx* c, void* stream, int m, int n, const double* const A[4], long lda,
                  const double* const X[4], long ldx, double* E, double* E_rel) {
  if (!c) return QPINV_E_INVALID;
  if (m <= 0 || n <= 0 || lda < n || ldx < m || !planes_ok(A) || !planes_ok(X) || !E || !E_rel)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    const int mode = c->opt.precision == QPINV_PREC_FP64 ? PM_F64 : PM_EMU;
    if (mode == PM_EMU && !tc_supported()) return fail(c, QPINV_E_UNSUPPORTED, "tcgen05 path needs an sm_103 device");
    QMat a = mat(c, "A", m, n, MST_D, false, false), x = mat(c, "X0", n, m, MST_D, false, false);
    load_planes(c, A, lda, m, n, a);
    load_planes(c, X, ldx, n, m, x);
    penrose(c, a, x, mode, E, E_rel, nullptr);
    if (mode == PM_EMU) check_kernel_error(c);
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_cur_complete(qpinv_ctx* c, void* stream, int m, int n, const double* const M[4], long ldm,
                       const unsigned char* mask, long ldmask, int r, int iters, const int* I, const int* J, int form,
                       qpinv_method method, double tol, int max_iter, double sigma, double* const C[4], long ldc,
                       qpinv_cur_result* out) {
  if (!c) return QPINV_E_INVALID;
  if (m <= 0 || n <= 0 || r < 1 || r > std::min(m, n) || iters < 1 || ldm < n || ldmask < n || ldc < n ||
      !planes_ok(M) || !planes_ok((const double* const*)C) || !mask || !I || !J || (form != 0 && form != 1) ||
      (int)method < 0 || (int)method > 4 || !(tol >= 0.0) || max_iter < 1 || !(sigma >= 0.0) ||
      std::ceil(2.0 * sigma) > kMaxGaussRadius)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  for (long t = 0; t < (long)iters * r; t++)
    if (I[t] < 0 || I[t] >= m || J[t] < 0 || J[t] >= n) return fail(c, QPINV_E_INVALID, "index out of range");
  const auto t_start = std::chrono::steady_clock::now();
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  c->st = st;
  qpinv_cur_result res;
  memset(&res, 0, sizeof(res));
  try {
    const bool fp64 = c->opt.precision == QPINV_PREC_FP64;
    if (!fp64 && !tc_supported()) return fail(c, QPINV_E_UNSUPPORTED, "tcgen05 path needs an sm_103 device");
    // caller data (device or host) into contiguous workspace planes
    QMat Mo = mat(c, "cur.M", m, n, MST_D, false, false);
    load_planes(c, M, ldm, m, n, Mo);
    unsigned char* dmask = (unsigned char*)buf(c, "cur.mask", (size_t)m * n + 64);
    ck(c, cudaMemcpy2DAsync(dmask, n, mask, ldmask, n, m, is_device_ptr(mask) ? cudaMemcpyDeviceToDevice
                                                                               : cudaMemcpyHostToDevice, st),
       "copy mask");
    int* didx = (int*)buf(c, "cur.idx", sizeof(int) * 2 * (size_t)iters * r + 64);
    ck(c, cudaMemcpyAsync(didx, I, sizeof(int) * (size_t)iters * r, cudaMemcpyHostToDevice, st), "copy I");
    ck(c, cudaMemcpyAsync(didx + (size_t)iters * r, J, sizeof(int) * (size_t)iters * r, cudaMemcpyHostToDevice, st),
       "copy J");
    QMat Cm = mat(c, "cur.C", m, n, MST_D, false, false), Xm = mat(c, "cur.X", m, n, MST_D, false, false);
    QMat CJ = mat(c, "cur.CJ", m, r, MST_D, false, false), RI = mat(c, "cur.RI", r, n, MST_D, false, false);
    QMat W = mat(c, "cur.W", r, r, MST_D, false, false), U = mat(c, "cur.U", r, r, MST_D, false, false);
    QMat CJp = mat(c, "cur.CJp", r, m, MST_D, false, false), RIp = mat(c, "cur.RIp", n, r, MST_D, false, false);
    QMat T1 = mat(c, "cur.T1", r, n, MST_D, false, false), T2 = mat(c, "cur.T2", m, r, MST_D, false, false);
    const double bytes_mn = 32.0 * m * n;
    CurFill f;
    for (int q = 0; q < 4; q++) f.M[q] = Mo.d.p + q * Mo.d.ps;
    f.ldm = n;
    f.mask = dmask;
    f.ldk = n;
    f.C = Cm.d.p;
    f.m = m;
    f.n = n;
    timed(c, EV_EW, 0, 0, bytes_mn * 2, [&] { return launch_cur_fill(f, st); });  // C^(0): missing = 0
    GaussTaps taps;
    if (sigma > 0.0) {  // sampled Gaussian on |x| <= ceil(2 sigma), normalised
      taps.radius = (int)std::ceil(2.0 * sigma);
      double sum = 0.0;
      for (int a = -taps.radius; a <= taps.radius; a++) sum += taps.w[a + taps.radius] = std::exp(-a * a / (2.0 * sigma * sigma));
      for (int a = 0; a <= 2 * taps.radius; a++) taps.w[a] /= sum;
    }
    // C = P Q on the tensor cores (FP64-accurate exact slices), or the FP64 kernel
    auto gemm = [&](const QMat& P, const QMat& Q, const QMat& R) {
      Solver S;
      S.c = c;
      S.dbl = true;
      S.L = 0;
      S.xS = 8;
      Solver::Acc acc = S.prod(P, Q, fp64 ? PM_F64 : PM_EMU);
      CombineArgs a = S.base_args(R.rows, R.cols, &acc);
      S.out(a, R, "f", 1.0);
      S.run(a);
      if (!fp64) check_kernel_error(c);
    };
    auto planes = [](const QMat& Q, double* p[4]) {
      for (int q = 0; q < 4; q++) p[q] = Q.d.p + q * Q.d.ps;
    };
    // pseudoinverse of P (rows x cols) into Pp (cols x rows) by the chosen iteration
    auto pinv = [&](const QMat& P, const QMat& Pp) {
      double* a[4];
      double* x[4];
      planes(P, a);
      planes(Pp, x);
      qpinv_result pr;
      const int rc = qpinv_solve(c, stream, P.rows, P.cols, a, P.cols, method, tol, max_iter, x, P.rows, &pr);
      if (rc != QPINV_OK) throw QpError{rc, "pseudoinverse: " + c->err};
      res.pinv_solves++;
      res.pinv_iters += pr.iters;
      res.pinv_worst_status = std::max(res.pinv_worst_status, pr.status);
      res.pinv_max_E1_rel = std::max(res.pinv_max_E1_rel, pr.E_rel[0]);
    };
    for (int t = 0; t < iters; t++) {
      const int* It = didx + (size_t)t * r;
      const int* Jt = didx + (size_t)iters * r + (size_t)t * r;
      timed(c, EV_EW, 0, 0, 64.0 * r * (m + n + r),
            [&] { return launch_cur_gather(Cm.d.p, m, n, r, It, Jt, CJ.d.p, RI.d.p, form ? W.d.p : nullptr, st); });
      if (form == 0) {  // U = C_J^dagger C R_I^dagger (eq. Uopt with A the filled matrix)
        pinv(CJ, CJp);
        pinv(RI, RIp);
        gemm(CJp, Cm, T1);
        gemm(T1, RIp, U);
      } else {  // U = W^dagger (eq. Ucross)
        pinv(W, U);
      }
      gemm(CJ, U, T2);
      gemm(T2, RI, Xm);  // X^(t) = C_J U R_I
      f.X = Xm.d.p;
      if (sigma > 0.0) {
        timed(c, EV_EW, 0, 0, bytes_mn * 2, [&] { return launch_cur_gauss(Xm.d.p, Cm.d.p, m, n, taps, st); });
        f.X = Cm.d.p;  // filtered X; the fill below overwrites it in place
      }
      timed(c, EV_EW, 0, 0, bytes_mn * 2.5, [&] { return launch_cur_fill(f, st); });  // C^(t+1)
    }
    store_planes(c, Cm, C, ldc, m, n);
    ck(c, cudaStreamSynchronize(st), "stream sync");
  } catch (const std::bad_alloc&) {
    cudaGetLastError();
    return fail(c, QPINV_E_NOMEM, "host allocation failed");
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  res.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (out) *out = res;
  return QPINV_OK;
}

int qpinv_toeplitz_filter(qpinv_ctx* c, void* stream, int N, const double* const x[4], const double* const s[4],
                          int p, int t0, qpinv_method method, double tol, int max_iter, double* const h[4],
                          double* const s_hat[4], qpinv_result* pinv_out, double* err) {
  if (!c) return QPINV_E_INVALID;
  if (N < 1 || p < 0 || t0 - p < 0 || t0 + p >= N || !planes_ok(x) || !planes_ok(s) ||
      !planes_ok((const double* const*)h) || !planes_ok((const double* const*)s_hat) || (int)method < 0 ||
      (int)method > 4 || !(tol >= 0.0) || max_iter < 1)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  c->st = st;
  try {
    const bool fp64 = c->opt.precision == QPINV_PREC_FP64;
    if (!fp64 && !tc_supported()) return fail(c, QPINV_E_UNSUPPORTED, "tcgen05 path needs an sm_103 device");
    const int n = p + 1;
    QMat xs = mat(c, "flt.x", 1, N, MST_D, false, false), ss = mat(c, "flt.s", 1, N, MST_D, false, false);
    load_planes(c, x, N, 1, N, xs);
    load_planes(c, s, N, 1, N, ss);
    QMat X = mat(c, "flt.X", n, n, MST_D, false, false), Xp = mat(c, "flt.Xp", n, n, MST_D, false, false);
    QMat S = mat(c, "flt.S", n, 1, MST_D, false, false), H = mat(c, "flt.h", n, 1, MST_D, false, false);
    QMat Sh = mat(c, "flt.sh", n, 1, MST_D, false, false);
    timed(c, EV_EW, 0, 0, 32.0 * n * n, [&] { return launch_toeplitz(xs.d.p, xs.d.ps, p, t0, X.d.p, st); });
    for (int q = 0; q < 4; q++)  // s(t0 + i), i = 0..p
      ck(c, cudaMemcpyAsync(S.d.p + q * S.d.ps, ss.d.p + q * ss.d.ps + t0, sizeof(double) * n,
                            cudaMemcpyDeviceToDevice, st),
         "copy target");
    double* a[4];
    double* xp[4];
    for (int q = 0; q < 4; q++) {
      a[q] = X.d.p + q * X.d.ps;
      xp[q] = Xp.d.p + q * Xp.d.ps;
    }
    qpinv_result pr;
    const int rc = qpinv_solve(c, stream, n, n, a, n, method, tol, max_iter, xp, n, &pr);
    if (rc != QPINV_OK) throw QpError{rc, "pseudoinverse: " + c->err};
    auto gemm = [&](const QMat& P, const QMat& Q, const QMat& R) {  // FP64-accurate R = P Q
      Solver S2;
      S2.c = c;
      S2.dbl = true;
      S2.L = 0;
      S2.xS = 8;
      Solver::Acc acc = S2.prod(P, Q, fp64 ? PM_F64 : PM_EMU);
      CombineArgs ca = S2.base_args(R.rows, R.cols, &acc);
      S2.out(ca, R, "f", 1.0);
      S2.run(ca);
      if (!fp64) check_kernel_error(c);
    };
    gemm(Xp, S, H);   // h = X^dagger s
    gemm(X, H, Sh);   // s_hat = X h
    const Planes<const double> sv = dview(S);  // eps = ||s_hat - s|| / ||s||
    const double num = fro2(c, dview(Sh), &sv, n, 1), den = fro2(c, sv, nullptr, n, 1);
    store_planes(c, H, h, 1, n, 1);
    store_planes(c, Sh, s_hat, 1, n, 1);
    ck(c, cudaStreamSynchronize(st), "stream sync");
    if (err) *err = den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
    if (pinv_out) *pinv_out = pr;
  } catch (const std::bad_alloc&) {
    cudaGetLastError();
    return fail(c, QPINV_E_NOMEM, "host allocation failed");
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_global_krylov(qpinv_ctx* c, void* stream, int n, int m, const double* const A[4], long lda,
                        const double* const B[4], long ldb, int kind, int restart, int precond_iters, double tol,
                        int max_iter, double* const X[4], long ldx, qpinv_krylov_result* out) {
  if (!c) return QPINV_E_INVALID;
  if (n < 1 || m < 1 || lda < n || ldb < m || ldx < m || !planes_ok(A) || !planes_ok(B) ||
      !planes_ok((const double* const*)X) || (kind != 0 && kind != 1) || restart < 0 || precond_iters < 0 ||
      precond_iters > 100 || !(tol >= 0.0) || max_iter < 1 || max_iter > 100000)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  // the basis and the Hessenberg matrix of one cycle grow with its length:
  // (cycle + 1) blocks and (cycle + 1) x cycle doubles, on the device and the host
  if ((restart > 0 ? std::min(restart, max_iter) : max_iter) > 10000)
    return fail(c, QPINV_E_INVALID, "cycle longer than 10000 steps: give restart <= 10000");
  const auto t_start = std::chrono::steady_clock::now();
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  c->st = st;
  qpinv_krylov_result res;
  memset(&res, 0, sizeof(res));
  try {
    const long L = 4L * n * m;
    QMat Ao = mat(c, "kry.A", n, n, MST_D, false, false), Bo = mat(c, "kry.B", n, m, MST_D, false, false);
    load_planes(c, A, lda, n, n, Ao);
    load_planes(c, B, ldb, n, m, Bo);
    QMat As = Ao, Bs = Bo;  // the system solved: A X = B, or M A X = M B
    auto f64 = [&](const QMat& P, const QMat& Q, const QMat& R) {
      const double fl = 32.0 * P.rows * P.cols * Q.cols;
      timed(c, EV_F64, fl, fl, 0, [&] {
        return skinny_ok(Q.cols) ? launch_qgemm_skinny(P.rows, P.cols, Q.cols, dview(P), dview(Q), R.d, st)
                                 : launch_qgemm_f64(P.rows, P.cols, Q.cols, dview(P), dview(Q), R.d, st);
      });
    };
    if (precond_iters > 0) {
      // M = X_k of QSAI (Alg. 2) from X_0 = alpha A^H, safe alpha, FP64 products
      QMat M = mat(c, "kry.M", n, n, MST_D, false, false);
      const qpinv_options saved = c->opt;
      c->opt.precision = QPINV_PREC_FP64;
      c->opt.penrose = 0;
      c->opt.stop_rule = QPINV_STOP_PAPER_ABS;
      c->opt.alpha_mode = QPINV_ALPHA_SAFE;
      c->opt.side = QPINV_SIDE_AUTO;
      double* a[4];
      double* x[4];
      for (int q = 0; q < 4; q++) {
        a[q] = Ao.d.p + q * Ao.d.ps;
        x[q] = M.d.p + q * M.d.ps;
      }
      qpinv_result pr;
      const int rc = qpinv_solve(c, stream, n, n, a, n, QPINV_QSAI, 0.0, precond_iters, x, n, &pr);
      c->opt = saved;
      c->st = st;
      if (rc != QPINV_OK) throw QpError{rc, "preconditioner: " + c->err};
      As = mat(c, "kry.MA", n, n, MST_D, false, false);
      Bs = mat(c, "kry.MB", n, m, MST_D, false, false);
      f64(M, Ao, As);
      f64(M, Bo, Bs);
    }
    const int cycle = restart > 0 ? std::min(restart, max_iter) : max_iter;
    double* V = (double*)buf(c, "kry.V", sizeof(double) * (size_t)(cycle + 1) * L + 64);
    QMat Xm = mat(c, "kry.X", n, m, MST_D, false, false), R = mat(c, "kry.R", n, m, MST_D, false, false);
    QMat Wm = mat(c, "kry.W", n, m, MST_D, false, false);
    // device: h scratch | norm | Hessenberg columns (rotated in place) | c | s | g | residual estimates
    const size_t hstride = (size_t)cycle + 1;
    double* dh = (double*)buf(c, "kry.h", sizeof(double) * ((size_t)cycle + 2 + hstride * cycle + 4 * hstride) + 64);
    double* dnrm = dh + cycle + 1;
    double* dH = dh + cycle + 2;
    double* dcs = dH + hstride * cycle;
    double* dsn = dcs + hstride;
    double* dg = dsn + hstride;
    double* dres = dg + hstride;
    ck(c, cudaMemsetAsync(Xm.d.p, 0, sizeof(double) * L, st), "memset");
    ck(c, cudaMemcpyAsync(R.d.p, Bs.d.p, sizeof(double) * L, cudaMemcpyDeviceToDevice, st), "copy");  // X_0 = 0
    timed(c, EV_EW, 0, 0, 8.0 * L, [&] { return launch_norm_scale(R.d.p, L, dnrm, nullptr, st); });
    double r0 = 0.0;
    read_back(c, dnrm, 1, &r0);
    // host copies: rotated columns (upper triangle), c, g, residual estimates
    std::vector<double> H(hstride * cycle), cs(cycle), gv(hstride), rs(cycle), y(cycle);
    constexpr int kCheck = 16;  // steps launched between host checks of the residual estimates
    int steps = 0;
    bool converged = r0 == 0.0;
    double beta = r0;
    while (steps < max_iter && !converged) {
      if (beta / r0 <= tol) {
        converged = true;
        break;
      }
      // V_0 = R / beta; g = beta e_1
      timed(c, EV_EW, 0, 0, 16.0 * L, [&] { return launch_norm_scale(R.d.p, L, dnrm, V, st); });
      ck(c, cudaMemsetAsync(dg, 0, sizeof(double) * hstride, st), "memset");
      c->h_pin[0] = beta;
      ck(c, cudaMemcpyAsync(dg, c->h_pin, sizeof(double), cudaMemcpyHostToDevice, st), "copy beta");
      // Steps are launched kCheck at a time without host synchronisation; the
      // host then finds the first step whose residual estimate meets the
      // tolerance (or whose h_{j+1,j} is 0).  Steps launched beyond it are
      // discarded: the GMRES / FOM iterate of step k uses columns 0..k-1 only.
      int k = 0, j = 0;
      bool done = false;
      while (!done) {
        const int j0 = j, nb = std::min({kCheck, cycle - j, max_iter - steps});  // >= 1: not done
        for (int b = 0; b < nb; b++, j++) {
          double* Vj = V + (size_t)j * L;
          Planes<const double> vj{Vj, (long)m, (long)n * m};
          Planes<double> w{Wm.d.p, (long)m, (long)n * m};
          timed(c, EV_F64, 32.0 * n * n * m, 32.0 * n * n * m, 0, [&] {
            return skinny_ok(m) ? launch_qgemm_skinny(n, n, m, dview(As), vj, w, st)
                                : launch_qgemm_f64(n, n, m, dview(As), vj, w, st);
          });
          double* hcol = dH + hstride * j;  // Hessenberg column j (j + 2 entries)
          ck(c, cudaMemsetAsync(hcol, 0, sizeof(double) * (j + 2), st), "memset");
          for (int pass = 0; pass < 2; pass++) {  // classical Gram-Schmidt, applied twice
            timed(c, EV_EW, 0, 0, 8.0 * L * (j + 2), [&] { return launch_block_dot(V, j + 1, Wm.d.p, L, dh, st); });
            timed(c, EV_EW, 0, 0, 8.0 * L * (j + 3),
                  [&] { return launch_block_sub(Wm.d.p, V, dh, j + 1, L, hcol, st); });
          }
          double* Vn = V + (size_t)(j + 1) * L;  // V_{j+1} = W / h_{j+1,j}
          timed(c, EV_EW, 0, 0, 16.0 * L, [&] { return launch_norm_scale(Wm.d.p, L, hcol + j + 1, Vn, st); });
          timed(c, EV_EW, 0, 0, 8.0 * (3 * j + 8),
                [&] { return launch_givens(hcol, dcs, dsn, dg, j, kind, dres, st); });
        }
        // the new columns' rows 0 .. j (rotated R and raw h_{j+1,j}), c, g, estimates
        ck(c, cudaMemcpy2DAsync(H.data() + hstride * j0, sizeof(double) * hstride, dH + hstride * j0,
                                sizeof(double) * hstride, sizeof(double) * (j + 1), nb, cudaMemcpyDeviceToHost, st),
           "read columns");
        ck(c, cudaMemcpyAsync(cs.data() + j0, dcs + j0, sizeof(double) * nb, cudaMemcpyDeviceToHost, st), "read c");
        ck(c, cudaMemcpyAsync(rs.data() + j0, dres + j0, sizeof(double) * nb, cudaMemcpyDeviceToHost, st), "read r");
        ck(c, cudaMemcpyAsync(gv.data(), dg, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st), "read g");
        ck(c, cudaStreamSynchronize(st), "stream sync");
        for (int t = j0; t < j; t++) {
          steps++;
          k = t + 1;
          if (rs[t] / r0 <= tol || steps >= max_iter || H[hstride * t + t + 1] == 0.0 || !(rs[t] == rs[t])) {
            done = true;
            break;
          }
        }
        if (j >= cycle) done = true;
      }
      // y: GMRES R y = g (upper triangular); FOM H_k y = beta e_1, which is
      // the same triangular system with the last rotation undone
      // (last diagonal times c_k, last right-hand side divided by c_k).
      for (int i = k - 1; i >= 0; i--) {
        double d = H[hstride * i + i], rhs = gv[i];
        if (kind == 1 && i == k - 1) {
          d *= cs[k - 1];
          rhs = cs[k - 1] != 0.0 ? rhs / cs[k - 1] : 0.0;
        }
        for (int l = i + 1; l < k; l++) rhs -= H[hstride * l + i] * y[l];
        y[i] = d != 0.0 ? rhs / d : 0.0;
      }
      ck(c, cudaMemcpyAsync(dh, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st), "copy y");
      timed(c, EV_EW, 0, 0, 8.0 * L * (k + 2), [&] { return launch_basis_add(Xm.d.p, V, dh, k, L, st); });
      ck(c, cudaStreamSynchronize(st), "sync");  // y is pageable host memory read by the copy above
      // explicit residual R = B' - A' X
      f64(As, Xm, Wm);
      timed(c, EV_EW, 0, 0, 24.0 * L, [&] { return launch_sub(R.d.p, Bs.d.p, Wm.d.p, L, st); });
      timed(c, EV_EW, 0, 0, 8.0 * L, [&] { return launch_norm_scale(R.d.p, L, dnrm, nullptr, st); });
      read_back(c, dnrm, 1, &beta);
      converged = beta / r0 <= tol;
    }
    res.iters = steps;
    res.converged = converged ? 1 : 0;
    res.rel_res = r0 > 0.0 ? beta / r0 : 0.0;
    // true residual ||B - A X|| / ||B||
    f64(Ao, Xm, Wm);
    timed(c, EV_EW, 0, 0, 24.0 * L, [&] { return launch_sub(R.d.p, Bo.d.p, Wm.d.p, L, st); });
    double tn = 0.0, bn = 0.0;
    timed(c, EV_EW, 0, 0, 8.0 * L, [&] { return launch_norm_scale(R.d.p, L, dnrm, nullptr, st); });
    read_back(c, dnrm, 1, &tn);
    timed(c, EV_EW, 0, 0, 8.0 * L, [&] { return launch_norm_scale(Bo.d.p, L, dnrm, nullptr, st); });
    read_back(c, dnrm, 1, &bn);
    res.true_rel_res = bn > 0.0 ? tn / bn : tn;
    store_planes(c, Xm, X, ldx, n, m);
    ck(c, cudaStreamSynchronize(st), "stream sync");
  } catch (const std::bad_alloc&) {
    cudaGetLastError();
    return fail(c, QPINV_E_NOMEM, "host allocation failed");
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  res.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (out) *out = res;
  return QPINV_OK;
}

int qpinv_solve_batched(qpinv_ctx* c, void* stream, int batch, const int* m, const int* n, const double* const* A,
                        const long* lda, qpinv_method method, double tol, int max_iter, double* const* X,
                        const long* ldx, qpinv_result* out) {
  if (!c) return QPINV_E_INVALID;
  if (batch < 1 || !m || !n || !A || !X || !lda || !ldx || max_iter < 1 || !(tol >= 0.0) || (int)method < 0 ||
      (int)method > 4)
    return fail(c, QPINV_E_INVALID, "invalid argument");
  const int maxd = batched_max_dim();
  for (int b = 0; b < batch; b++) {
    if (m[b] < 1 || n[b] < 1 || m[b] > maxd || n[b] > maxd || lda[b] < n[b] || ldx[b] < m[b])
      return fail(c, QPINV_E_INVALID, "batched matrix " + std::to_string(b) + ": shape outside [1, 256] or bad ld");
    for (int q = 0; q < 4; q++)
      if (!A[4 * b + q] || !X[4 * b + q] || !is_device_ptr(A[4 * b + q]) || !is_device_ptr(X[4 * b + q]))
        return fail(c, QPINV_E_INVALID, "batched matrix " + std::to_string(b) + ": planes must be device pointers");
  }
  const auto t_start = std::chrono::steady_clock::now();
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    int nsm = 0;
    ck(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device), "device attribute");
    int max_slots = 0;
    for (int t = 0; t < BATCH_TILES; t++) max_slots = std::max(max_slots, nsm * batched_slots_per_sm(t));
    max_slots = std::min(max_slots, batch);
    BatchRun run;
    run.ws = buf(c, "batch.ws", batched_slot_bytes() * (size_t)max_slots);
    run.dev_items = buf(c, "batch.items", batched_item_bytes() * (size_t)batch + 64);
    run.dev_order = buf(c, "batch.order", sizeof(int) * (size_t)batch + 64);
    run.dev_results = buf(c, "batch.results", batched_result_bytes() * (size_t)batch + 64);
    run.dev_counter = (int*)buf(c, "batch.counter", 64);
    // tensor-core engine: slice scratch and TMA maps for one slot per SM
    run.tc_ws = buf(c, "batch.tcws", batched_tc_slot_bytes() * (size_t)nsm);
    run.tc_maps = buf(c, "batch.tcmaps", sizeof(CUtensorMap) * 2 * (size_t)nsm + 64);
    if (!c->bmaps_host) ck(c, cudaMallocHost(&c->bmaps_host, sizeof(CUtensorMap) * 2 * (size_t)nsm + 64), "pinned maps");
    run.host_maps = c->bmaps_host;
    run.err = c->d_err;
    const size_t need[3] = {batched_item_bytes() * (size_t)batch, sizeof(int) * (size_t)batch,
                            batched_result_bytes() * (size_t)batch};
    for (int t = 0; t < 3; t++)
      if (c->bh_cap[t] < need[t]) {
        if (c->bh_buf[t]) cudaFreeHost(c->bh_buf[t]);
        c->bh_buf[t] = nullptr;
        c->bh_cap[t] = 0;
        ck(c, cudaMallocHost(&c->bh_buf[t], need[t] + 64), "pinned staging");
        c->bh_cap[t] = need[t];
      }
    run.host_items = c->bh_buf[0];
    run.host_order = c->bh_buf[1];
    run.host_results = c->bh_buf[2];
    if (!c->bgraph.stream) ck(c, cudaStreamCreateWithFlags(&c->bgraph.stream, cudaStreamNonBlocking), "stream");
    std::vector<BatchResultHost> res;
    const int amode = c->opt.alpha_mode == QPINV_ALPHA_USER ? QPINV_ALPHA_USER
                      : c->opt.alpha_mode == QPINV_ALPHA_FRO ? QPINV_ALPHA_FRO
                                                              : QPINV_ALPHA_SAFE;
    const int mparam = method == QPINV_QHPIM ? c->opt.hyper_order : c->opt.qrapid_N;
    auto solve_with = [&](int tile, int cnt, const int* mm, const int* nn, const double* const* AA,
                          const long* la, double* const* XX, const long* lx, BatchGraph* graph, int iters) {
      run.tile = tile;
      run.slots = std::min(cnt, nsm * batched_slots_per_sm(tile));
      ck(c, run_batched(cnt, mm, nn, AA, la, XX, lx, (int)method, tol, iters, mparam, c->opt.stop_rule,
                        amode, c->opt.alpha_user, hpi19_k, run, graph, res, c->st),
         "batched solve");
    };
    int tile = c->opt.batched_tile;
    if (tile < 0) {
      // Autotuner: a batch signature (method, count, shape histogram) maps to
      // the tile that ran three iterations on an evenly spaced sample of its
      // matrices (one per SM) fastest.
      unsigned long long sig = 0x51ED270B27A5B49Dull ^ ((unsigned long long)method << 40) ^
                               ((unsigned long long)mparam << 48) ^ (unsigned long long)batch;
      int hist[16] = {0};
      for (int b = 0; b < batch; b++) hist[(std::max(m[b], n[b]) - 1) / 16]++;
      for (int t = 0; t < 16; t++) sig = (sig ^ (unsigned long long)hist[t]) * 0x100000001B3ull;
      auto hit = c->tile_of.find(sig);
      if (hit != c->tile_of.end()) {
        tile = hit->second;
      } else {
        const auto t0 = std::chrono::steady_clock::now();
        const int cnt = std::min(batch, nsm);
        std::vector<int> sm(cnt), sn(cnt);
        std::vector<long> sla(cnt), slx(cnt);
        std::vector<const double*> sa(4 * (size_t)cnt);
        std::vector<double*> sx(4 * (size_t)cnt);
        for (int k = 0; k < cnt; k++) {
          const int b = (int)((long long)k * batch / cnt);
          sm[k] = m[b];
          sn[k] = n[b];
          sla[k] = lda[b];
          slx[k] = ldx[b];
          for (int q = 0; q < 4; q++) {
            sa[4 * k + q] = A[4 * b + q];
            sx[4 * k + q] = X[4 * b + q];
          }
        }
        double best = INFINITY;
        tile = 1;
        for (int t = 0; t < BATCH_TILES; t++) {
          ck(c, cudaStreamSynchronize(c->st), "sync");
          const auto a0 = std::chrono::steady_clock::now();
          // three iterations per matrix: the tiles' relative speed, not a converged solve
          solve_with(t, cnt, sm.data(), sn.data(), sa.data(), sla.data(), sx.data(), slx.data(), nullptr,
                     std::min(max_iter, 3));
          check_kernel_error(c);
          const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a0).count();
          if (c->trace)
            fprintf(stderr, "qpinv batched tile %s: %.2f ms on %d sampled matrices\n", batched_tile_name(t), ms, cnt);
          if (ms < best) {
            best = ms;
            tile = t;
          }
        }
        c->tile_of[sig] = tile;
        c->stats.batched_tune_ms +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      }
    }
    c->stats.batched_tile = tile;
    const int replays = c->bgraph.replays;
    timed(c, EV_EW, 0, 0, 0, [&] {
      solve_with(tile, batch, m, n, A, lda, X, ldx, &c->bgraph, max_iter);
      return cudaSuccess;
    });
    check_kernel_error(c);  // bounded waits of the tensor-core engine
    if (c->bgraph.replays > replays && c->bgraph.replays > 1) c->stats.batched_graph_replays++;
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (out) {
      for (int b = 0; b < batch; b++) {
        qpinv_result& r = out[b];
        memset(&r, 0, sizeof(r));
        r.status = res[b].status < 0 ? QPINV_NONFINITE_INPUT : res[b].status;
        r.iters = res[b].iters;
        r.alpha = res[b].alpha;
        r.alpha_source = amode;
        r.side = res[b].side;
        r.precision = QPINV_PREC_DF32;
        r.delta = res[b].delta;
        r.delta_rel = res[b].delta_rel;
        for (int q = 0; q < 4; q++) {
          r.E[q] = res[b].E[q];
          r.E_rel[q] = res[b].E_rel[q];
        }
        r.gemms = res[b].gemms;
        r.time_ms = ms;
      }
    }
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_alpha_features(qpinv_ctx* c, void* stream, int m, int n, const double* const A[4], long lda, float* feat,
                         double* theta1) {
  if (!c) return QPINV_E_INVALID;
  if (m <= 0 || n <= 0 || lda < n || !planes_ok(A) || !feat) return fail(c, QPINV_E_INVALID, "invalid argument");
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    QMat a = mat(c, "A", m, n, MST_D | MST_F, false, false);
    load_planes(c, A, lda, m, n, a);
    Planes<const double> av = dview(a);
    double bad = 0.0;
    const double f2 = fro2(c, av, nullptr, m, n, &bad);
    if (bad > 0.0) return fail(c, QPINV_E_NONFINITE, "A contains NaN or Inf");
    double* rs = (double*)buf(c, "rowsum", sizeof(double) * (size_t)(m + n) + 64);
    double* mx = (double*)buf(c, "maxes", sizeof(double) * 4);
    ck(c, launch_abs_sums(av, m, n, rs, rs + m, (double*)buf(c, "colpart", sizeof(double) * (size_t)COL_SCRATCH(n) + 64), c->st), "abs sums");
    ck(c, launch_max(rs, m, mx, c->st), "max");
    ck(c, launch_max(rs + m, n, mx + 1, c->st), "max");
    double hm[2];
    read_back(c, mx, 2, hm);
    ck(c, launch_f64_to_f32(av, m, n, a.f, c->st), "A to fp32");
    double t1 = 0.0;
    features_of(c, a, f2, hm[1], hm[0], feat, &t1);
    if (theta1) *theta1 = t1;
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_alpha_weights(qpinv_ctx* c, float* w, int count, int set) {
  if (!c || !w || count != alpha_nweights()) return c ? fail(c, QPINV_E_INVALID, "weight count mismatch") : QPINV_E_INVALID;
  if (set) {
    c->alpha_w.assign(w, w + count);
  } else {
    if (c->alpha_w.empty()) return fail(c, QPINV_E_INVALID, "the network is untrained");
    memcpy(w, c->alpha_w.data(), sizeof(float) * count);
  }
  return QPINV_OK;
}

int qpinv_alpha_gradient(qpinv_ctx* c, void* stream, int count, const float* feat, const float* label, float* grad,
                         double* loss) {
  if (!c || count < 1 || !feat || !label || !grad || c->alpha_w.empty())
    return c ? fail(c, QPINV_E_INVALID, "invalid argument or untrained network") : QPINV_E_INVALID;
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    const int NW = alpha_nweights(), NT = alpha_ntrain();
    float* dW = (float*)buf(c, "alpha.W", sizeof(float) * NW);
    float* dX = (float*)buf(c, "alpha.X", sizeof(float) * 32 * (size_t)count);
    float* dT = (float*)buf(c, "alpha.T", sizeof(float) * (size_t)count);
    float* dG = (float*)buf(c, "alpha.G", sizeof(float) * NT);
    float* sc = (float*)buf(c, "alpha.sc", sizeof(float) * alpha_scratch_floats(count) + 64);
    double* dl = (double*)buf(c, "alpha.loss", sizeof(double) * 2);
    ck(c, cudaMemcpyAsync(dW, c->alpha_w.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, c->st), "copy");
    ck(c, cudaMemcpyAsync(dX, feat, sizeof(float) * 32 * count, cudaMemcpyHostToDevice, c->st), "copy");
    ck(c, cudaMemcpyAsync(dT, label, sizeof(float) * count, cudaMemcpyHostToDevice, c->st), "copy");
    timed(c, EV_EW, 0, 0, 0, [&] { return alpha_gradient(dW, dX, dT, count, sc, dG, dl, c->st); });
    ck(c, cudaMemcpyAsync(grad, dG, sizeof(float) * NT, cudaMemcpyDeviceToHost, c->st), "copy");
    double hl = 0.0;
    read_back(c, dl, 1, &hl);
    if (loss) *loss = hl;
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_alpha_train(qpinv_ctx* c, void* stream, int count, const float* feat, const float* label, int epochs,
                      int batch, float lr, unsigned long long seed, double* loss) {
  if (!c || count < 2 || !feat || !label || epochs < 1 || batch < 1 || !(lr > 0.f))
    return c ? fail(c, QPINV_E_INVALID, "invalid argument") : QPINV_E_INVALID;
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    const int NW = alpha_nweights(), NT = alpha_ntrain();
    std::vector<float> W(NW);
    alpha_init_weights(W.data(), seed);
    // input standardisation from the training set (mu, sd stored with the weights)
    for (int j = 0; j < 32; j++) {
      double mu = 0, v = 0;
      for (int i = 0; i < count; i++) mu += feat[(size_t)i * 32 + j];
      mu /= count;
      for (int i = 0; i < count; i++) v += (feat[(size_t)i * 32 + j] - mu) * (feat[(size_t)i * 32 + j] - mu);
      W[NW - 64 + j] = (float)mu;
      W[NW - 32 + j] = (float)std::max(std::sqrt(v / count), 1e-3);
    }
    if (batch > count) batch = count;
    float* dW = (float*)buf(c, "alpha.W", sizeof(float) * NW);
    float* dX = (float*)buf(c, "alpha.X", sizeof(float) * 32 * (size_t)count);
    float* dT = (float*)buf(c, "alpha.T", sizeof(float) * (size_t)count);
    float* dG = (float*)buf(c, "alpha.G", sizeof(float) * NT);
    float* dM1 = (float*)buf(c, "alpha.M1", sizeof(float) * NT);
    float* dM2 = (float*)buf(c, "alpha.M2", sizeof(float) * NT);
    float* sc = (float*)buf(c, "alpha.sc", sizeof(float) * alpha_scratch_floats(std::max(batch, count)) + 64);
    double* dl = (double*)buf(c, "alpha.loss", sizeof(double) * 2);
    ck(c, cudaMemcpyAsync(dW, W.data(), sizeof(float) * NW, cudaMemcpyHostToDevice, c->st), "copy");
    ck(c, cudaMemsetAsync(dM1, 0, sizeof(float) * NT, c->st), "memset");
    ck(c, cudaMemsetAsync(dM2, 0, sizeof(float) * NT, c->st), "memset");
    std::vector<int> perm(count);
    for (int i = 0; i < count; i++) perm[i] = i;
    std::vector<float> px((size_t)count * 32), pt(count);
    unsigned long long st = seed * 0x9E3779B97F4A7C15ull + 1;
    int step = 0;
    for (int ep = 0; ep < epochs; ep++) {
      for (int i = count - 1; i > 0; i--) {  // Fisher-Yates with splitmix64
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        std::swap(perm[i], perm[(int)(z % (unsigned long long)(i + 1))]);
      }
      for (int i = 0; i < count; i++) {
        memcpy(&px[(size_t)i * 32], &feat[(size_t)perm[i] * 32], sizeof(float) * 32);
        pt[i] = label[perm[i]];
      }
      ck(c, cudaMemcpyAsync(dX, px.data(), sizeof(float) * 32 * count, cudaMemcpyHostToDevice, c->st), "copy");
      ck(c, cudaMemcpyAsync(dT, pt.data(), sizeof(float) * count, cudaMemcpyHostToDevice, c->st), "copy");
      for (int b0 = 0; b0 + batch <= count; b0 += batch) {
        step++;
        timed(c, EV_EW, 0, 0, 0,
              [&] { return alpha_gradient(dW, dX + (size_t)b0 * 32, dT + b0, batch, sc, dG, dl, c->st); });
        timed(c, EV_EW, 0, 0, 0, [&] { return alpha_adam(dW, dG, dM1, dM2, step, lr, c->st); });
      }
      ck(c, cudaStreamSynchronize(c->st), "sync");  // host buffers px, pt are reused next epoch
    }
    timed(c, EV_EW, 0, 0, 0, [&] { return alpha_gradient(dW, dX, dT, count, sc, dG, dl, c->st); });
    double hl = 0.0;
    read_back(c, dl, 1, &hl);
    if (loss) *loss = hl;
    ck(c, cudaMemcpyAsync(W.data(), dW, sizeof(float) * NW, cudaMemcpyDeviceToHost, c->st), "copy");
    ck(c, cudaStreamSynchronize(c->st), "sync");
    c->alpha_w = W;
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

int qpinv_alpha_predict(qpinv_ctx* c, void* stream, const float* feat, double* y) {
  if (!c || !feat || !y || c->alpha_w.empty())
    return c ? fail(c, QPINV_E_INVALID, "invalid argument or untrained network") : QPINV_E_INVALID;
  DeviceGuard g(c->device);
  c->st = (cudaStream_t)stream;
  try {
    *y = predict_one(c, feat);
  } catch (const QpError& e) {
    cudaGetLastError();
    return fail(c, e.code, e.msg);
  }
  return QPINV_OK;
}

}  // extern "C"
