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
//      (Q), becomes S = 7 balanced base-128 digits, each stored as the BF16
//      value of the digit itself (an integer of at most 8 bits: exact), in
//      the slot's slice scratch (P row-major, Q transposed: both K-major),
//      zero padded in K to a multiple of 32;
//   3. warp-specialised tensor-core phase over the product's 128 x 64
//      quaternion tiles: TMA stages the slice planes (64-byte swizzle), two
//      threads issue the 16 signed MMAs per K step, level d = s + t sums the
//      pairs (s, t) in K chunks short enough for exact FP32 partial sums in
//      TMEM (integers: the digits are unscaled), the epilogue warps add each
//      chunk exactly into int32 level sums in registers and store each
//      finished level to its own int32 plane (through a per-warp shared
//      transposition tile, so that the stores are coalesced; stores only);
//   4. all threads sum each entry's level planes in 64-bit fixed point, turn
//      the sum into a df value (exact two-term split) and apply the pass's
//      epilogue (scale, aux terms, diagonal, stop-test norms).
// With S = 7 slices (49 bits) the products carry the df masters' accuracy
// (about 2^-46), which rank-deficient blocks need: rounding that reaches the
// complement of the range is multiplied by the method's order every step.
//
// Roles inside a product (352 threads): warp 0 lane 0 TMA, warps 1-2 lane 0
// MMA (components 0-1 and 2-3; warp 1 owns TMEM: 512 columns, two FP32 chunk
// buffers), warps 3-10 the TMEM epilogue (TMEM lane quarter = warp % 4,
// column half = (warp - 3) / 4); exponents, slicing and the combine use all
// warps.  mbarrier phases continue across products.  Every wait is bounded
// (2 s): on expiry the kernel raises an error word, stops issuing tensor-core
// work, drains its copies and frees TMEM.
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
// per epilogue warp: a 32-row x 16-column int32 transposition tile (row
// pitch 20 words: 16-byte aligned rows, conflict-free 16-byte stores)
constexpr int TXP = 20;
constexpr int TXTILE = 32 * TXP * 4;  // bytes
constexpr int TSMEM = TSTAGES * TSTAGE + 8 * TXTILE + 1024;
constexpr int TKP = MAXD;   // K pitch of the slice scratch (elements)
constexpr int TMAXS = 8;    // slice planes reserved per operand
constexpr int TS = 7;       // slices formed per operand (49 bits)
static_assert(TS >= 2 && TS <= TMAXS, "slice count");
constexpr uint32_t TIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);
static_assert(TSMEM + 4096 <= 227 * 1024, "shared memory per CTA");
constexpr int TMMA_WARPS = 2;               // MMA issuers: components 0-1 and 2-3
constexpr int TEPI0 = 1 + TMMA_WARPS;        // first of the 8 epilogue warps (two per TMEM lane quarter)
constexpr int TTHREADS = 32 * (TEPI0 + 8);   // 352
constexpr int TSTAGING = (TTHREADS / 32) * MAXD * (int)sizeof(int);  // column-exponent partials, in stage 0
static_assert(TSTAGING <= TSTAGE, "the exponent staging fits in one idle stage");
static_assert(TTHREADS <= TPB_MAX, "shared per-matrix state sized for the block");

// slice scratch per slot: A-form and B-form [TMAXS][4][MAXD][TKP] BF16, then
// the int32 level sums [TS][4][MAXD][MAXD]
constexpr size_t TC_SLICE_BYTES = (size_t)TMAXS * 4 * MAXD * TKP * sizeof(bf16);
constexpr size_t TC_LVL_BYTES = (size_t)TS * 4 * MAXD * MAXD * sizeof(int);
constexpr size_t TC_SLOT_BYTES = 2 * TC_SLICE_BYTES + TC_LVL_BYTES;

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
// 2^a as a float for a in [-126, 127] (exponent bits).
__device__ __forceinline__ float pow2f(int a) { return __int_as_float((a + 127) << 23); }

// v * 2^x for an exponent x of any size: two exact power-of-two factors
// (each clamped to the float range; a result below it is zero anyway).
__device__ __forceinline__ float scale2(float v, int x) {
  const int a = min(max(x >> 1, -126), 127), b = min(max(x - (x >> 1), -126), 127);
  return v * pow2f(a) * pow2f(b);
}

// Factors s1 s2 = 2^(7 TS - e) that bring a row (column) with exponent e to
// |v 2^(7 TS - e)| <= 2^(7 TS); zero for a row of zeros / subnormals.
__device__ __forceinline__ void slice_scale(int e, float& s1, float& s2) {
  if (e < -10000) {
    s1 = s2 = 0.f;
    return;
  }
  const int sh = min(max(7 * TS - e, -252), 252);
  s1 = pow2f(sh >> 1);
  s2 = pow2f(sh - (sh >> 1));
}

// Balanced base-128 digits: with F = round(v 2^(7 TS - e)), |F| <= 2^(7 TS),
// and G = F + 64 (1 + 2^7 + ... + 2^(7 (TS - 2))), the digit of weight
// 2^(7 q) is ((G >> 7 q) & 127) - 64 for q < TS - 1, and the top one is
// G >> 7 (TS - 1), in [-128, 128].  Slice p (p = 0 the top) holds the digit of
// weight 2^(7 (TS - 1 - p)), so that v 2^-e = sum_p digit_p 2^-7(p+1).
constexpr long long digit_bias_of(int n) { return n == 0 ? 0 : (64LL << (7 * (n - 1))) + digit_bias_of(n - 1); }
constexpr long long DIGIT_BIAS = digit_bias_of(TS - 1);
__device__ __forceinline__ long long biased_fixed(dfv v, float s1, float s2) {
  // each part scaled exactly, rounded to an integer (|part| <= 2^(7 TS))
  return __float2ll_rn(v.hi * s1 * s2) + __float2ll_rn(v.lo * s1 * s2) + DIGIT_BIAS;
}
// Digit p of a biased value as a float, exactly: 2^23 + u - (2^23 + 64) for
// the low digits (u the 7-bit field), 2^23 + (t + 128) - (2^23 + 128) for the
// top one.
template <int p>
__device__ __forceinline__ float digit_f(long long G) {
  if constexpr (p == 0) {
    return __int_as_float(0x4B000000 | (int)((G >> (7 * (TS - 1))) + 128)) - 8388736.0f;
  } else {
    return __int_as_float(0x4B000000u | ((unsigned)(G >> (7 * (TS - 1 - p))) & 127u)) - 8388672.0f;
  }
}
// Slice plane p of 8 consecutive biased values: 8 BF16 digits (the upper
// halves of the exact floats) in one 16-byte store.
template <int p>
__device__ __forceinline__ void store_plane8(bf16* dst, const long long* G) {
  uint32_t pk[4];
#pragma unroll
  for (int q = 0; q < 4; q++)
    pk[q] = __byte_perm(__float_as_uint(digit_f<p>(G[2 * q])), __float_as_uint(digit_f<p>(G[2 * q + 1])), 0x7632);
  *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}
template <int p>
__device__ __forceinline__ void store_planes8(bf16* base, long lstride, const long long* G) {
  store_plane8<p>(base + p * lstride, G);
  if constexpr (p + 1 < TS) store_planes8<p + 1>(base, lstride, G);
}
// The TS slices of 8 consecutive entries sharing one scale (base 16-byte aligned).
__device__ __forceinline__ void slice8(bf16* base, long lstride, const dfv* v, float s1, float s2) {
  long long G[8];
#pragma unroll
  for (int q = 0; q < 8; q++) G[q] = biased_fixed(v[q], s1, s2);
  store_planes8<0>(base, lstride, G);
}

// Epilogue: drain FP32 chunk w (TMEM buffer w % 2) into the thread's int32
// level sums and release the buffer.  The level's first chunk assigns the
// sums, later chunks add: the sums are dead between levels.
template <bool FIRST>
__device__ __forceinline__ bool drain_chunk(int (&acc)[128], int& w, uint32_t tb0, int lane, TcShared* ts, int* err) {
  const int b = w & 1;
  const uint32_t tb = tb0 + b * 256;
  int have = 1;
  if (lane == 0) have = mbar_wait(smem_u32(&ts->acc_full[b]), (w >> 1) & 1, &ts->abort_flag, err, 24) ? 1 : 0;
  have = __shfl_sync(0xffffffffu, have, 0);
  if (!have) return false;
  fence_after();
#pragma unroll
  for (int p = 0; p < 8; p++) {
    uint32_t f[16];
    tmem_ld16u(tb + p * 16, f);
    tmem_wait_ld();
    // the chunk's FP32 sums are integers (products of unscaled digits)
#pragma unroll
    for (int t = 0; t < 16; t++) {
      const int x = __float2int_rn(__uint_as_float(f[t]));
      if constexpr (FIRST) acc[p * 16 + t] = x;
      else acc[p * 16 + t] += x;
    }
  }
  fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(smem_u32(&ts->acc_empty[b]));
  w++;
  return true;
}

// The tensor-core CTA GEMM: C = epilogue(P Q) for df matrices (P M x K, Q K x N).
struct TcGemm {
  Shared* sh;
  TcShared* ts;
  uint8_t* smem;  // 1024-aligned: TSTAGES stages (the first doubles as the exponent staging), then the
                  // epilogue warps' transposition tiles
  const CUtensorMap* mapA;
  const CUtensorMap* mapB;
  bf16* sa;  // A-form slices [TMAXS][4][MAXD][TKP]
  bf16* sb;  // B-form slices [TMAXS][4][MAXD][TKP] (row j = column j of Q)
  int* lvl;  // int32 level sums [TS][4][MAXD][MAXD]
  int* err;

  __device__ void operator()(const DM& P, const DM& Q, const DM& C, const Epi& e, double* norms);
  // the phases, each its own function (own register allocation)
  __device__ void exponents(const DM& P, const DM& Q);
  __device__ void slices(const DM& P, const DM& Q);
  __device__ void products(int M, int N, int K, int u0, int w0);
  __device__ void combine(int M, int N, int shift, const DM& C, const Epi& e, double* norms);
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
  const int tid = threadIdx.x;
  // exact slices, zero padded in K to a multiple of TBK; units of 8
  // consecutive k of one (component, row) for P and one (component, column)
  // for Q, two units per thread in flight (their 16 loads issued first)
  const int KP = (K + TBK - 1) / TBK * TBK;
  const long lstride = 4L * MAXD * TKP;
  const int KP8 = KP / 8;
  {
    const long units = 4L * M * KP8;
    for (long t0 = tid; t0 < units; t0 += 2 * TTHREADS) {
      dfv v[2][8];
      int ci[2], ii[2], kk[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const long t = t0 + h * TTHREADS;
        const bool ok = t < units;
        const long r = ok ? t : 0;
        kk[h] = (int)(r % KP8) * 8;
        ii[h] = (int)((r / KP8) % M);
        ci[h] = (int)(r / ((long)KP8 * M));
#pragma unroll
        for (int q = 0; q < 8; q++)
          v[h][q] = ok && kk[h] + q < K ? P.at(ci[h], ii[h], kk[h] + q) : dfv{0.f, 0.f};
      }
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (t0 + h * TTHREADS >= units) break;
        float s1, s2;
        slice_scale(ts->eP[ii[h]], s1, s2);
        slice8(sa + ((long)ci[h] * MAXD + ii[h]) * TKP + kk[h], lstride, v[h], s1, s2);
      }
    }
  }
  {
    // Q: lanes 0-15 take 16 consecutive columns at one group of 8 k, lanes
    // 16-31 the same columns at the next group (coalesced loads along j; the
    // two 16-byte stores of a column meet in one 32-byte sector)
    const int NB = (N + 15) / 16, KP16 = KP / 16;
    const long lanes_total = 4L * NB * KP16 * 32;  // (component, 16-column block, 16 k) x 32 lanes
    for (long t0 = tid; t0 < lanes_total; t0 += 2 * TTHREADS) {
      dfv v[2][8];
      int ci[2], jj[2], kk[2];
      bool ok[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const long t = t0 + h * TTHREADS;
        const int jl = (int)(t & 15), kp = (int)((t >> 4) & 1);
        long r = t >> 5;
        const int k16 = (int)(r % KP16);
        r /= KP16;
        const int jb = (int)(r % NB);
        ci[h] = (int)(r / NB);
        jj[h] = jb * 16 + jl;
        kk[h] = k16 * 16 + kp * 8;
        ok[h] = t < lanes_total && jj[h] < N;
#pragma unroll
        for (int q = 0; q < 8; q++)
          v[h][q] = ok[h] && kk[h] + q < K ? Q.at(ci[h], kk[h] + q, jj[h]) : dfv{0.f, 0.f};
      }
#pragma unroll
      for (int h = 0; h < 2; h++) {
        if (!ok[h]) continue;
        float s1, s2;
        slice_scale(ts->eQ[jj[h]], s1, s2);
        slice8(sb + ((long)ci[h] * MAXD + jj[h]) * TKP + kk[h], lstride, v[h], s1, s2);
      }
    }
  }
  // the slices are read by TMA (async proxy), which also overwrites the
  // stage ring the exponent phase used
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
}

__device__ __noinline__ void TcGemm::products(int M, int N, int K, int u0, int w0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  (void)warp;
  (void)lane;
  // ---- 3. tensor-core phase ----
  int kc[TMAXS];
#pragma unroll
  for (int d = 0; d < TMAXS; d++) {
    int c0 = K;
    if (d <= TS - 3) {
      const int lim = d == 0 ? 256 : 1024 / (d + 3);
      c0 = (lim / TBK) * TBK;
    }
    kc[d] = c0 < K ? c0 : K;
  }
  const int Mt = (M + TBM - 1) / TBM, Nt = (N + TBN - 1) / TBN;
  {
    if (warp == 0) {
      // ---------------- TMA producer ----------------
      if (lane == 0) {
        int u = u0;
        bool ok = true;
        for (int tile = 0; tile < Mt * Nt && ok; tile++) {
          const int m0 = (tile % Mt) * TBM, n0 = (tile / Mt) * TBN;
          for (int d = TS - 1; d >= 0 && ok; d--) {
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
          for (int d = TS - 1; d >= 0 && ok; d--) {
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
      // ---------------- epilogue: FP32 chunk -> int32 level sums (registers) -> int64 (global) -> C ----------------
      // Warp e = warp - TEPI0 reads TMEM lane quarter warp % 4 and column half e / 4
      // (components 2h, 2h + 1): 128 int32 level sums per thread.
      const int e8 = warp - TEPI0, quarter = warp & 3, half = e8 >> 2;
      const uint32_t tb0 = ts->tmem + ((uint32_t)(quarter * 32) << 16) + half * 128;
      int w = w0;
      int acc[128];
      int* xt = reinterpret_cast<int*>(smem + TSTAGES * TSTAGE + e8 * TXTILE);
      const int rr = lane >> 4, cc = lane & 15;
      for (int tile = 0; tile < Mt * Nt; tile++) {
        const int m0 = (tile % Mt) * TBM, n0 = (tile / Mt) * TBN;
        const int row0 = m0 + quarter * 32;  // this warp's rows row0 .. row0 + 31 (TMEM lanes)
        for (int d = TS - 1; d >= 0; d--) {
          // a failed wait (abort) leaves the loops at once (no path from it
          // reads the level sums: they stay dead across the combine call)
          if (!drain_chunk<true>(acc, w, tb0, lane, ts, err)) goto epilogue_done;
          for (int k0 = kc[d]; k0 < K; k0 += kc[d])
            if (!drain_chunk<false>(acc, w, tb0, lane, ts, err)) goto epilogue_done;
          // level done: this warp's 32 rows x 128 sums go to the level's
          // int32 plane, 16 columns at a time through the warp's shared tile
          // (each lane writes its row, then reads lane-consecutive columns),
          // so that every global store instruction covers two 64-byte row
          // segments; stores only (no read-modify-write: the combine sums the
          // levels)
#pragma unroll
          for (int p = 0; p < 8; p++) {
            const int c = 2 * half + (p >> 2), j = n0 + (p & 3) * 16 + cc;
            int4* trow = reinterpret_cast<int4*>(xt + lane * TXP);
#pragma unroll
            for (int q = 0; q < 4; q++)
              trow[q] = make_int4(acc[p * 16 + 4 * q], acc[p * 16 + 4 * q + 1], acc[p * 16 + 4 * q + 2],
                                  acc[p * 16 + 4 * q + 3]);
            __syncwarp();
            int* dst = lvl + (((long)d * 4 + c) * MAXD + row0) * MAXD + j;
            if (j < N)
#pragma unroll 4
              for (int i = 0; i < 16; i++) {
                const int r = 2 * i + rr;
                if (row0 + r < M) dst[(long)r * MAXD] = xt[r * TXP + cc];
              }
            __syncwarp();
          }
        }
      }
    epilogue_done:;
    }
  }
}

// All level planes written: every thread takes entries (i, j) in row-major
// order (coalesced).  An entry's TS int32 level sums are shifted to the
// common 64-bit fixed point (value 2^(eP + eQ - shift) times the integer) and
// summed exactly, the sum split exactly in two floats, then
// out = ca v + sum_a ct_a aux_a + diag I is stored to C, with the stop-test
// partials against ref.  An entry's loads precede its store (C may alias an
// aux plane at that entry only).
__device__ __noinline__ void TcGemm::combine(int M, int N, int shift, const DM& C, const Epi& e, double* norms) {
  const int tid = threadIdx.x;
  const bool has_ref = e.ref != nullptr;
  const long lplane = 4L * MAXD * MAXD;
  float nd = 0.f, nx = 0.f;
  for (long t = tid; t < (long)M * N; t += TTHREADS) {
    const int i = (int)(t / N), j = (int)(t % N);
    const int ex = ts->eP[i] + ts->eQ[j] - shift;
    int L[4][TS];
    dfv ax[4][3], rf[4];
#pragma unroll
    for (int c = 0; c < 4; c++)
#pragma unroll
      for (int d = 0; d < TS; d++) L[c][d] = lvl[d * lplane + ((long)c * MAXD + i) * MAXD + j];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int c = 0; c < 4; c++) ax[c][a] = e.aux[a] ? e.aux[a]->at(c, i, j) : dfv{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 4; c++) rf[c] = has_ref ? e.ref->at(c, i, j) : dfv{0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 4; c++) {
      long long q = 0;
#pragma unroll
      for (int d = 0; d < TS; d++) {
        const int shd = shift - 7 * (d + 2);
        const long long x = (long long)L[c][d];
        q += shd >= 0 ? (x << shd) : ((x + (1LL << (-shd - 1))) >> (-shd));
      }
      const float hq = __ll2float_rn(q);
      const float lq = __ll2float_rn(q - (long long)hq);
      const dfv v = epi_entry(e, df_quick(scale2(hq, ex), scale2(lq, ex)), ax[c], c, i, j, C);
      if (has_ref) {
        const dfv dd = df_add(v, df_neg(rf[c]));
        nd += dd.hi * dd.hi;
        nx += v.hi * v.hi;
      }
    }
  }
  if (has_ref) {
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
  if (!aborted) products(M, N, K, u0, w0);
  // every level plane written and visible to every thread
  fence_before();
  __syncthreads();
  fence_after();
  combine(M, N, shift, C, e, norms);
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
  g.lvl = reinterpret_cast<int*>(slot + 2 * TC_SLICE_BYTES);
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
  if (P.tc_slices != TS || !P.tc_maps || !P.tc_ws || !P.err) return cudaErrorInvalidValue;
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
