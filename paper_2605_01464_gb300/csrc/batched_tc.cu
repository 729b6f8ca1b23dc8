// batched_tc.cu -- the tensor-core engine of qpinv_solve_batched.
//
// Same persistent kernel structure as the CUDA-core engine (batched_impl.cuh:
// one CTA per matrix at a time from an atomic work counter, the solve end to
// end with double-FP32 "df" masters in a global workspace slot), but every
// CTA-level quaternion product runs on the tcgen05 tensor cores as an
// exact-slice product, the scheme of the dense FP64-accurate kernel
// (qgemm_emu.cu) applied inside one CTA:
//   1. per-row exponents of P and per-column exponents of Q (integer bit
//      operations on the df high parts);
//   2. every df entry v = hi + lo, scaled by 2^-e of its row (P) or column
//      (Q), becomes S balanced 7-bit digits -- exact BF16 values -- in the
//      slot's slice scratch (P row-major, Q transposed: both K-major), zero
//      padded in K to a multiple of 32;
//   3. warp-specialised tensor-core phase over the product's 128 x 64
//      quaternion tiles: TMA stages the slice planes (64-byte swizzle), one
//      thread issues the 16 signed MMAs per K step, level d = s + t sums the
//      pairs (s, t) in K chunks short enough for exact FP32 partial sums in
//      TMEM, the epilogue warps add each chunk exactly into an int32 level
//      sum in TMEM and each finished level into an int64 fixed-point
//      accumulator (global, L2-resident);
//   4. all threads turn the int64 sums back into df values (exact two-term
//      split) and apply the pass's epilogue (scale, aux terms, diagonal,
//      stop-test norms).
// With S = 7 slices (49 bits) the products carry the df masters' accuracy
// (about 2^-46), which rank-deficient blocks need: rounding that reaches the
// complement of the range is multiplied by the method's order every step.
//
// Roles inside a product (256 threads): warp 0 lane 0 TMA, warp 1 lane 0
// MMA (warp 1 owns TMEM: 512 columns, FP32 chunk buffer + int32 level sums),
// warps 4-7 the TMEM epilogue (TMEM lane quarter = warp % 4); every phase in
// between uses all warps.  mbarrier phases continue across products.  Every
// wait is bounded (2 s): on expiry the kernel raises an error word, stops
// issuing tensor-core work, drains its copies and frees TMEM.
#define QP_BATCHED_TILE 5
#define QP_BATCHED_TC_UNIT 1
#include "batched_impl.cuh"
#include "tc_ptx.cuh"

namespace qp {
namespace {

constexpr int TBM = 128, TBN = 64, TBK = 32, TSWB = 64;
constexpr int TSTAGES = 4;
constexpr int TA_PLANE = TBM * TBK * 2;            // 8 KB
constexpr int TB_PLANE = TBN * TBK * 2;            // 4 KB
constexpr int TSTAGE = 4 * (TA_PLANE + TB_PLANE);  // 48 KB
constexpr int TSTAGING = 4 * 32 * 33 * 8;          // slicing transpose, aliased with stage 0
constexpr int TSMEM = TSTAGES * TSTAGE + 1024;
static_assert(TSTAGING <= TSTAGE, "the slicing staging fits in one idle stage");
constexpr int TKP = MAXD;   // K pitch of the slice scratch (elements)
constexpr int TMAXS = 8;    // slice planes reserved per operand
constexpr uint32_t TIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);
static_assert(TSMEM + 4096 <= 227 * 1024, "shared memory per CTA");
constexpr int TMMA_WARPS = 2;               // MMA issuers: components 0-1 and 2-3
constexpr int TEPI0 = 1 + TMMA_WARPS;        // first of the 8 epilogue warps (two per TMEM lane quarter)
constexpr int TTHREADS = 32 * (TEPI0 + 8);   // 352
static_assert(TTHREADS <= TPB_MAX, "shared per-matrix state sized for the block");

// slice scratch per slot: A-form and B-form [TMAXS][4][MAXD][TKP] BF16, then
// the int64 accumulator [4][MAXD][MAXD]
constexpr size_t TC_SLICE_BYTES = (size_t)TMAXS * 4 * MAXD * TKP * sizeof(bf16);
constexpr size_t TC_C64_BYTES = (size_t)4 * MAXD * MAXD * sizeof(long long);
constexpr size_t TC_SLOT_BYTES = 2 * TC_SLICE_BYTES + TC_C64_BYTES;

struct TcShared {
  uint64_t full[TSTAGES], empty[TSTAGES], acc_full[2], acc_empty[2];
  uint32_t tmem;
  int abort_flag;
  int u, w, issued;  // stage uses and chunks so far (mbarrier phases); loads issued
  int eP[MAXD], eQ[MAXD];
};

// Binary exponent e with |v| < 2^e from the bits (-100000 for zero / subnormal).
__device__ __forceinline__ int fexp(float v) {
  const int ex = (int)((__float_as_uint(v) >> 23) & 0xFF);
  return ex == 0 ? -100000 : ex - 126;
}
// round(v * 2^sh) as an integer from the bits of v (|v * 2^sh| < 2^62).
__device__ __forceinline__ long long ffixed(float v, int sh) {
  const unsigned b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 0xFF);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0x7FFFFFu) | (1u << 23));
  const int k = ex - 150 + sh;
  long long F;
  if (k >= 0) F = mant << k;
  else if (k <= -26) F = 0;
  else F = (mant + (1ll << (-k - 1))) >> (-k);
  return (b >> 31) ? -F : F;
}
// S balanced base-128 digits of (hi + lo) * 2^(7S - e), slice l at
// base[l * lstride]: slice l = digit_l * 2^-7(l+1) (the top digit may reach 128).
__device__ __forceinline__ void slice_df(bf16* base, long lstride, int S, dfv v, int e) {
  const int sh = 7 * S - e;
  long long F = ffixed(v.hi, sh) + ffixed(v.lo, sh);
  for (int l = S - 1; l >= 1; l--) {
    int d = (int)(F & 127);
    if (d >= 64) d -= 128;
    F = (F - d) >> 7;
    base[l * lstride] = __float2bfloat16_rn(ldexpf((float)d, -7 * (l + 1)));
  }
  base[0] = __float2bfloat16_rn(ldexpf((float)F, -7));
}

// The same for 8 consecutive entries of one row (one exponent), written as
// 16-byte stores per slice plane (base 16-byte aligned).
__device__ __forceinline__ void slice_df8(bf16* base, long lstride, int S, const dfv* v, int e) {
  const int sh = 7 * S - e;
  long long F[8];
#pragma unroll
  for (int q = 0; q < 8; q++) F[q] = ffixed(v[q].hi, sh) + ffixed(v[q].lo, sh);
  for (int l = S - 1; l >= 0; l--) {
    uint32_t pk[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      float x[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (l > 0) {
          int d = (int)(F[q + h] & 127);
          if (d >= 64) d -= 128;
          F[q + h] = (F[q + h] - d) >> 7;
          x[h] = ldexpf((float)d, -7 * (l + 1));
        } else {
          x[h] = ldexpf((float)F[q + h], -7);
        }
      }
      pk[q >> 1] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[0])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[1])) << 16);
    }
    *reinterpret_cast<uint4*>(base + l * lstride) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// The tensor-core CTA GEMM: C = epilogue(P Q) for df matrices (P M x K, Q K x N).
struct TcGemm {
  Shared* sh;
  TcShared* ts;
  uint8_t* smem;  // 1024-aligned: TSTAGES stages (the first doubles as staging outside the tensor-core phase)
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  bf16* sa;  // A-form slices [TMAXS][4][MAXD][TKP]
  bf16* sb;  // B-form slices [TMAXS][4][MAXD][TKP] (row j = column j of Q)
  long long* c64;  // [4][MAXD][MAXD]
  int S;
  int* err;

  __device__ void operator()(const DM& P, const DM& Q, const DM& C, const Epi& e, double* norms);
  // the phases, each its own function (own register allocation)
  __device__ void exponents(const DM& P, const DM& Q);
  __device__ void slices(const DM& P, const DM& Q);
  __device__ void products(int M, int N, int K, int shift, int u0, int w0);
  __device__ void combine(int M, int N, int K, int shift, const DM& C, const Epi& e, double* norms);
};

__device__ __noinline__ void TcGemm::exponents(const DM& P, const DM& Q) {
  const int K = P.cols, M = P.rows, N = Q.cols;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)warp;
  (void)lane;
  // ---- 1. exponents ----
  for (int i = warp; i < M; i += TTHREADS / 32) {
    int ex = -100000;
    for (int k = lane; k < K; k += 32)
#pragma unroll
      for (int c = 0; c < 4; c++) ex = max(ex, fexp(P.at(c, i, k).hi));
    for (int o = 16; o > 0; o >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, o));
    if (lane == 0) ts->eP[i] = ex;
  }
  {
    // columns of Q: lanes walk 32 consecutive columns, warps split the rows;
    // per-warp maxima meet in the shared staging area
    int* part = reinterpret_cast<int*>(smem);  // [warps][MAXD], in the idle stage ring
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      int ex = -100000;
      if (j < N)
        for (int k = warp; k < K; k += TTHREADS / 32)
#pragma unroll
          for (int c = 0; c < 4; c++) ex = max(ex, fexp(Q.at(c, k, j).hi));
      part[warp * MAXD + j] = ex;  // j < j0 + 32 <= MAXD
    }
    __syncthreads();
    for (int j = tid; j < N; j += TTHREADS) {
      int ex = part[j];
#pragma unroll
      for (int w = 1; w < TTHREADS / 32; w++) ex = max(ex, part[w * MAXD + j]);
      ts->eQ[j] = ex;
    }
  }
  __syncthreads();
}

__device__ __noinline__ void TcGemm::slices(const DM& P, const DM& Q) {
  const int K = P.cols, M = P.rows, N = Q.cols;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)warp;
  (void)lane;
  // ---- 2. exact slices (zero padded in K to a multiple of TBK) ----
  const int KP = (K + TBK - 1) / TBK * TBK;
  const long lstride = 4L * MAXD * TKP;
  const int KP8 = KP / 8;
  for (long t = tid; t < (long)M * KP8; t += TTHREADS) {
    const int i = (int)(t / KP8), k = (int)(t % KP8) * 8;
    // two planes' 16 loads in flight before any is used (the slot's
    // matrices live in L2 / HBM and one CTA per SM has few warps to hide it)
    const int e = ts->eP[i];
#pragma unroll
    for (int c0 = 0; c0 < 4; c0 += 2) {
      dfv v[2][8];
#pragma unroll
      for (int c = 0; c < 2; c++)
#pragma unroll
        for (int q = 0; q < 8; q++) v[c][q] = k + q < K ? P.at(c0 + c, i, k + q) : dfv{0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 2; c++) slice_df8(sa + ((long)(c0 + c) * MAXD + i) * TKP + k, lstride, S, v[c], e);
    }
  }
  {
    // Q transposed through shared memory: reads along j, writes along k (the
    // first 256 threads: 8 rows of 32 per pass)
    dfv(*st)[32][33] = reinterpret_cast<dfv(*)[32][33]>(smem);  // the idle stage ring
    const int tx = tid & 31, ty = tid >> 5;
    for (int k0 = 0; k0 < KP; k0 += 32)
      for (int j0 = 0; j0 < N; j0 += 32) {
        if (tid < 256) {
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int k = k0 + ty + 8 * q, j = j0 + tx;
#pragma unroll
            for (int c = 0; c < 4; c++) st[c][ty + 8 * q][tx] = (k < K && j < N) ? Q.at(c, k, j) : dfv{0.f, 0.f};
          }
        }
        __syncthreads();
        if (tid < 256) {
          // 32 columns x 4 groups of 8 k: thread (jl, g) = (tid / 4 % 32, tid % 4), one plane pass each
          const int jl = (tid >> 2) & 31, g = tid & 3, j = j0 + jl, k = k0 + 8 * g;
          if (j < N)
#pragma unroll 1
            for (int c = 0; c < 4; c++) {
              if ((tid >> 7) != (c & 1)) continue;  // threads 0..127 planes 0, 2; 128..255 planes 1, 3
              dfv v[8];
#pragma unroll
              for (int q = 0; q < 8; q++) v[q] = st[c][8 * g + q][jl];
              slice_df8(sb + ((long)c * MAXD + j) * TKP + k, lstride, S, v, ts->eQ[j]);
            }
        }
        __syncthreads();
      }
  }
  // the slices are read by TMA (async proxy)
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();

}

__device__ __noinline__ void TcGemm::products(int M, int N, int K, int shift, int u0, int w0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)warp;
  (void)lane;
  const bool aborted = false;
  // ---- 3. tensor-core phase ----
  int kc[TMAXS];
#pragma unroll
  for (int d = 0; d < TMAXS; d++) {
    int c0 = K;
    if (d <= S - 3) {
      const int lim = d == 0 ? 256 : 1024 / (d + 3);
      c0 = (lim / TBK) * TBK;
    }
    kc[d] = c0 < K ? c0 : K;
  }
  const int Mt = (M + TBM - 1) / TBM, Nt = (N + TBN - 1) / TBN;
  if (!aborted) {
    if (warp == 0) {
      // ---------------- TMA producer ----------------
      if (lane == 0) {
        int u = u0;
        bool ok = true;
        for (int tile = 0; tile < Mt * Nt && ok; tile++) {
          const int m0 = (tile % Mt) * TBM, n0 = (tile / Mt) * TBN;
          for (int d = S - 1; d >= 0 && ok; d--) {
            for (int k0 = 0; k0 < K && ok; k0 += kc[d]) {
              const int kb0 = k0 / TBK, kb1 = (min(K, k0 + kc[d]) + TBK - 1) / TBK;
              for (int kb = kb0; kb < kb1 && ok; kb++) {
                for (int s = 0; s <= d; s++, u++) {
                  const int st = u % TSTAGES;
                  if (u >= TSTAGES && !mbar_wait(smem_u32(&ts->empty[st]), ((u / TSTAGES) - 1) & 1,
                                                 &ts->abort_flag, err, 21)) {
                    ok = false;
                    break;
                  }
                  const uint32_t fb = smem_u32(&ts->full[st]);
                  mbar_expect_tx(fb, TSTAGE);
                  uint8_t* sp = smem + (size_t)st * TSTAGE;
                  for (int c = 0; c < 4; c++)
                    tma_load_3d(smem_u32(sp + c * TA_PLANE), mapA, kb * TBK, m0, s * 4 + c, fb);
                  for (int c = 0; c < 4; c++)
                    tma_load_3d(smem_u32(sp + 4 * TA_PLANE + c * TB_PLANE), mapB, kb * TBK, n0, (d - s) * 4 + c, fb);
                  ts->issued = u + 1;
                }
              }
            }
          }
        }
        if (ok) ts->u = u;
      }
    } else if (warp < TEPI0) {
      // ---------------- MMA issuers: warp 1 components 0, 1; warp 2 components 2, 3 ----------------
      if (lane == 0) {
        const bool lo = warp == 1;
        int u = u0, w = w0;
        bool ok = true;
        for (int tile = 0; tile < Mt * Nt && ok; tile++) {
          for (int d = S - 1; d >= 0 && ok; d--) {
            for (int k0 = 0; k0 < K && ok; k0 += kc[d], w++) {
              const int b = w & 1;  // FP32 buffer of this chunk, free once chunk w - 2 was drained
              if (w >= 2 && !mbar_wait(smem_u32(&ts->acc_empty[b]), ((w >> 1) - 1) & 1, &ts->abort_flag, err, 22)) {
                ok = false;
                break;
              }
              fence_after();
              const uint32_t dacc = ts->tmem + b * 256;
              const int kb0 = k0 / TBK, kb1 = (min(K, k0 + kc[d]) + TBK - 1) / TBK;
              bool first = true;
              for (int kb = kb0; kb < kb1 && ok; kb++) {
                for (int s = 0; s <= d; s++, u++) {
                  const int st = u % TSTAGES;
                  if (!mbar_wait(smem_u32(&ts->full[st]), (u / TSTAGES) & 1, &ts->abort_flag, err, 23)) {
                    ok = false;
                    break;
                  }
                  fence_after();
                  uint8_t* sp = smem + (size_t)st * TSTAGE;
                  const uint64_t ad0 = smem_desc_sw<TSWB>(smem_u32(sp)),
                                 bd0 = smem_desc_sw<TSWB>(smem_u32(sp + 4 * TA_PLANE));
#pragma unroll
                  for (int kk = 0; kk < TBK / 16; kk++) {
                    if (lo)
                      qmma_k16_half<TA_PLANE, TB_PLANE, 0>(dacc, TBN, ad0 + kk * 2, bd0 + kk * 2, TIDESC,
                                                          first && kk == 0);
                    else
                      qmma_k16_half<TA_PLANE, TB_PLANE, 2>(dacc, TBN, ad0 + kk * 2, bd0 + kk * 2, TIDESC,
                                                          first && kk == 0);
                  }
                  first = false;
                  mma_commit(smem_u32(&ts->empty[st]));
                }
              }
              if (ok) mma_commit(smem_u32(&ts->acc_full[b]));
            }
          }
        }
        if (ok && lo) ts->w = w;
      }
    } else {
      // ---------------- epilogue: FP32 chunk -> int32 level sums (registers) -> int64 (global) ----------------
      // Warp e = warp - TEPI0 reads TMEM lane quarter warp % 4 and column half e / 4
      // (components 2h, 2h + 1): 128 int32 level sums per thread.
      const int e8 = warp - TEPI0, quarter = warp & 3, half = e8 >> 2;
      const uint32_t tb0 = ts->tmem + ((uint32_t)(quarter * 32) << 16) + half * 128;
      int w = w0;
      bool ok = true;
      int acc[128];
      for (int tile = 0; tile < Mt * Nt && ok; tile++) {
        const int m0 = (tile % Mt) * TBM, n0 = (tile / Mt) * TBN;
        const int row = m0 + quarter * 32 + lane;
        for (int d = S - 1; d >= 0 && ok; d--) {
          const float scale = ldexpf(1.0f, 7 * (d + 2));
          const int shd = shift - 7 * (d + 2);
          for (int k0 = 0; k0 < K && ok; k0 += kc[d], w++) {
            const int b = w & 1;
            const uint32_t tb = tb0 + b * 256;
            int have = 1;
            if (lane == 0)
              have = mbar_wait(smem_u32(&ts->acc_full[b]), (w >> 1) & 1, &ts->abort_flag, err, 24) ? 1 : 0;
            have = __shfl_sync(0xffffffffu, have, 0);
            if (!have) {
              ok = false;
              break;
            }
            fence_after();
            const bool first = k0 == 0;
#pragma unroll
            for (int p = 0; p < 8; p++) {
              uint32_t f[16];
              tmem_ld16u(tb + p * 16, f);
              tmem_wait_ld();
#pragma unroll
              for (int t = 0; t < 16; t++) {
                const int x = __float2int_rn(__uint_as_float(f[t]) * scale);
                acc[p * 16 + t] = first ? x : acc[p * 16 + t] + x;
              }
            }
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&ts->acc_empty[b]));
            if (k0 + kc[d] < K || row >= M) continue;
            // level done: int64 accumulator (+)= int32 sum * 2^shd, this
            // thread's row, components 2 half and 2 half + 1 (16-byte accesses;
            // a column past N in a pair lands in the row's padding, never read)
#pragma unroll
            for (int p = 0; p < 4; p++) {
              const int c = 2 * half + (p >> 1), j0 = n0 + (p & 1) * 32;
              long long* dst = c64 + ((long)c * MAXD + row) * MAXD + j0;
#pragma unroll
              for (int t = 0; t < 32; t += 2) {
                if (j0 + t >= N) break;
                const long long x0 = (long long)acc[p * 32 + t], x1 = (long long)acc[p * 32 + t + 1];
                longlong2 y;
                y.x = shd >= 0 ? (x0 << shd) : ((x0 + (1LL << (-shd - 1))) >> (-shd));
                y.y = shd >= 0 ? (x1 << shd) : ((x1 + (1LL << (-shd - 1))) >> (-shd));
                longlong2* dp = reinterpret_cast<longlong2*>(dst + t);
                if (d != S - 1) {
                  const longlong2 g0 = *dp;
                  y.x += g0.x;
                  y.y += g0.y;
                }
                *dp = y;
              }
            }
          }
        }
      }
    }
  }
}

__device__ __noinline__ void TcGemm::combine(int M, int N, int K, int shift, const DM& C, const Epi& e,
                                             double* norms) {
  (void)K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)warp;
  (void)lane;
  fence_before();
  __syncthreads();
  fence_after();

  // ---- 4. int64 -> df, the pass's epilogue ----
  float nd = 0.f, nx = 0.f;
  for (long t = tid; t < (long)M * N; t += TTHREADS) {
    const int i = (int)(t / N), j = (int)(t % N);
    const int ex = ts->eP[i] + ts->eQ[j] - shift;
    // loads first (the stores to C may alias an aux plane at this very entry only)
    long long q[4];
    dfv ax[3][4], rf[4];
#pragma unroll
    for (int c = 0; c < 4; c++) q[c] = c64[((long)c * MAXD + i) * MAXD + j];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) ax[a][c] = e.aux[a] ? e.aux[a]->at(c, i, j) : dfv{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 4; c++) rf[c] = e.ref ? e.ref->at(c, i, j) : dfv{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      const float h = __ll2float_rn(q[c]);
      const float l = __ll2float_rn(q[c] - (long long)h);
      dfv v = df_quick(ldexpf(h, ex), ldexpf(l, ex));
      v = df_mul(e.ca, v);
#pragma unroll
      for (int a = 0; a < 3; a++)
        if (e.aux[a]) v = df_fma(e.ct[a], ax[a][c], v);
      if (c == 0 && i == j) v = df_add(v, e.diag);
      if (e.ref) {
        const dfv dd = df_add(v, df_neg(rf[c]));
        nd += dd.hi * dd.hi;
        nx += v.hi * v.hi;
      }
      C.at(c, i, j) = v;
    }
  }
  if (e.ref) {
    norms[0] = block_sum((double)nd, *sh, 0);
    norms[1] = block_sum((double)nx, *sh, 1);
  } else {
    __syncthreads();
  }
}


__device__ __noinline__ void TcGemm::operator()(const DM& P, const DM& Q, const DM& C, const Epi& e, double* norms) {
  const int M = P.rows, K = P.cols, N = Q.cols;
  const int u0 = ts->u, w0 = ts->w;  // read before this product's first barrier
  const bool aborted = ts->abort_flag != 0;
  int lg = 0;
  while ((1L << lg) < 4L * K) lg++;
  const int shift = 61 - lg;  // |sum| < 4K in normalized units
  exponents(P, Q);
  slices(P, Q);
  if (!aborted) products(M, N, K, shift, u0, w0);
  combine(M, N, K, shift, C, e, norms);
}

__global__ void __launch_bounds__(TTHREADS, 1) k_batched_tc(BatchParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ Shared sh;
  __shared__ TcShared ts;
  __shared__ int next;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    ts.abort_flag = 0;
    ts.u = ts.w = ts.issued = 0;
    for (int s = 0; s < TSTAGES; s++) {
      mbar_init(smem_u32(&ts.full[s]), 1);
      mbar_init(smem_u32(&ts.empty[s]), TMMA_WARPS);  // one commit per MMA issuer
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&ts.acc_full[b]), TMMA_WARPS);
      mbar_init(smem_u32(&ts.acc_empty[b]), 8);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ts.tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();

  char* slot = P.tc_ws + (long)blockIdx.x * P.tc_slot_bytes;
  TcGemm g;
  g.sh = &sh;
  g.ts = &ts;
  g.smem = smem;
  g.mapA = P.tc_maps + 2 * blockIdx.x;
  g.mapB = P.tc_maps + 2 * blockIdx.x + 1;
  g.sa = reinterpret_cast<bf16*>(slot);
  g.sb = reinterpret_cast<bf16*>(slot + TC_SLICE_BYTES);
  g.c64 = reinterpret_cast<long long*>(slot + 2 * TC_SLICE_BYTES);
  g.S = P.tc_slices;
  g.err = P.err;
  if (threadIdx.x == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(g.mapA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(g.mapB)) : "memory");
  }
  Ctx c;
  c.P = &P;
  c.sh = &sh;
  c.base = P.ws + (long)blockIdx.x * P.slot_elems;
  for (;;) {
    if (threadIdx.x == 0) next = ts.abort_flag ? P.count : atomicAdd(P.counter, 1);
    __syncthreads();
    const int item = next;
    __syncthreads();
    if (item >= P.count) break;
    solve_item(P, c, g, P.order[item]);
  }

  fence_before();
  __syncthreads();
  // after an abort: wait (bounded) for the copies this CTA still has in flight
  if (threadIdx.x == 0 && ts.abort_flag) {
    for (int u = (ts.issued > TSTAGES ? ts.issued - TSTAGES : 0); u < ts.issued; u++)
      (void)mbar_wait(smem_u32(&ts.full[u % TSTAGES]), (u / TSTAGES) & 1, &ts.abort_flag, nullptr, 0);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(ts.tmem), "r"(512) : "memory");
  }
}

}  // namespace

cudaError_t batched_launch_tc(int slots, const BatchParams& P, cudaStream_t st) {
  if (P.tc_slices < 2 || P.tc_slices > TMAXS || !P.tc_maps || !P.tc_ws || !P.err) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k_batched_tc, TSMEM, attr_done)) return e;
  k_batched_tc<<<slots, TTHREADS, TSMEM, st>>>(P);
  return cudaGetLastError();
}

size_t batched_tc_slot_bytes() { return TC_SLOT_BYTES; }

// Two TMA maps per slot over its slice scratch: A-form and B-form planes
// [TMAXS * 4][MAXD rows][TKP], boxes of 32 K-elements x 128 (A) / 64 (B) rows.
cudaError_t batched_tc_maps(char* tc_ws, int slots, CUtensorMap* host_maps, void* dev_maps, cudaStream_t st) {
  for (int s = 0; s < slots; s++) {
    char* slot = tc_ws + (size_t)s * TC_SLOT_BYTES;
    const bf16* sa = reinterpret_cast<const bf16*>(slot);
    const bf16* sb = reinterpret_cast<const bf16*>(slot + TC_SLICE_BYTES);
    if (!make_map(&host_maps[2 * s], sa, TKP, MAXD, 4 * TMAXS, TKP, (long)MAXD * TKP, TBM, TBK) ||
        !make_map(&host_maps[2 * s + 1], sb, TKP, MAXD, 4 * TMAXS, TKP, (long)MAXD * TKP, TBN, TBK))
      return cudaErrorInvalidValue;
  }
  return cudaMemcpyAsync(dev_maps, host_maps, sizeof(CUtensorMap) * 2 * (size_t)slots, cudaMemcpyHostToDevice, st);
}

}  // namespace qp
