// qgemm_tc.cu -- quaternion GEMM on the sm_103a tensor cores (tcgen05 + TMEM + TMA).
//
// The quaternion product C = A B (Hamilton product, Sec. 2) is one real
// contraction [C0 C1 C2 C3] = [A0 A1 A2 A3] M(B), where block (r, c) of the
// 4K x 4N matrix M(B) is +-B_{r xor c}:
//     c=0    c=1    c=2    c=3
//   r=0 +B0   +B1    +B2    +B3
//   r=1 -B1   +B0    -B3    +B2
//   r=2 -B2   +B3    +B0    -B1
//   r=3 -B3   -B2    +B1    +B0
// M(B) is never formed: per K step the kernel stages the four A planes and
// the four B planes of a tile in shared memory (TMA; 64-byte swizzle for the
// two-CTA-per-SM shape, 128-byte for the two-accumulator shape) and
// issues the 16 (r, c) products as separate tcgen05.mma instructions, each
// reading plane r xor c of B and taking its sign from the instruction
// descriptor's negate-A bit.  The four output components accumulate in FP32
// in TMEM (128 lanes x 4*BN columns).
//
// Split operands: A and B are sums of BF16 terms (A = A_0 + A_1 + ...); the
// kernel accumulates A_i B_j over a list of (i, j) pairs, giving products
// accurate to about 2^-8 (1 term), 2^-16 (3 pairs) or 2^-24 (6 pairs).
//
// Roles (192 threads): warp 0 issues TMA loads, warp 1 owns TMEM and issues
// the MMAs (one elected lane), warps 2-5 drain TMEM to global memory through
// a shared-memory transpose (coalesced rows).
// Every wait is bounded (2 s of globaltimer); on expiry the kernel records
// an error code, stops issuing work, drains what it started and frees TMEM.
#include <cuda.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qp {
namespace {

constexpr int BM = 128;  // output rows per CTA = TMEM lanes
constexpr int BN = 64;   // quaternion output columns per CTA (per component)
constexpr int ACC_COLS = 4 * BN;  // TMEM columns of one accumulator (four output components)
constexpr int GROUP_M = 16;       // CTA rasterization: 16 row tiles per group share B tiles in L2

// Stage shape.  BK BF16 K-elements per stage = one swizzle row of 2*BK bytes.
//   Wide: BK = 32 (64-byte swizzle), 48 KB per stage, two CTAs per SM, so one
//         CTA's epilogue overlaps the other's main loop (one accumulator).
//   Deep: BK = 64 (128-byte swizzle), 96 KB per stage, one CTA per SM (two
//         accumulators take all 512 TMEM columns).
template <int BK_, int SWB_, int MINB_>
struct Cfg {
  static constexpr int BK = BK_;
  static constexpr int SWB = SWB_;
  static constexpr int MINB = MINB_;
  static constexpr int STAGES = 2;
  static constexpr int A_PLANE = BM * BK * 2;
  static constexpr int B_PLANE = BN * BK * 2;
  static constexpr int STAGE = 4 * (A_PLANE + B_PLANE);
  static constexpr int SMEM = STAGES * STAGE + 1024;
};
using CfgWide = Cfg<32, 64, 2>;
using CfgDeep = Cfg<64, 128, 1>;
static_assert(CfgWide::SMEM * 2 <= 227 * 1024, "two wide CTAs per SM");
static_assert(CfgDeep::SMEM * 2 > 228 * 1024, "one deep CTA per SM");
constexpr int THREADS = 192;

static_assert(ACC_COLS == 256, "TMEM allocations must be powers of two (256 or 512 columns)");

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = BM, N = BN.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);

struct KParams {
  int M, N;
  int Mt, Nt;    // tile counts
  int kb0, kb1;  // K blocks [kb0, kb1) of BK elements
  int npairs;
  int pi[16], pj[16];
  int pacc[16];   // accumulator (0 or 1) of each pair
  int pfirst[16]; // 1 if the pair is the first of its accumulator
  int nacc;       // 1 or 2 accumulators (2 only with int64 output)
  Planes<float> C;
  long long* C64;  // non-null: int64 fixed-point accumulation
  long ld64, ps64;
  float scale;     // 2^shift
  int* err;
};

template <class C>
__global__ void __launch_bounds__(THREADS, C::MINB)
    k_qgemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, KParams P) {
  constexpr int BK = C::BK, STAGES = C::STAGES, A_PLANE_BYTES = C::A_PLANE, B_PLANE_BYTES = C::B_PLANE,
                STAGE_BYTES = C::STAGE;
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES], bar_acc;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // grouped rasterization: consecutive CTAs walk GROUP_M row tiles, then the next column tile
  const int per_group = GROUP_M * P.Nt, group = blockIdx.x / per_group, local = blockIdx.x % per_group;
  const int gm = min(GROUP_M, P.Mt - group * GROUP_M);
  const int m0 = (group * GROUP_M + local % gm) * BM, n0 = (local / gm) * BN;
  const int nunits = (P.kb1 - P.kb0) * P.npairs;
  const uint32_t tmem_cols = P.nacc == 2 ? 2 * ACC_COLS : ACC_COLS;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_acc), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;  // producer: units whose loads were issued

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      for (int u = 0; u < nunits; u++) {
        const int s = u % STAGES;
        if (u >= STAGES && !mbar_wait(smem_u32(&bar_empty[s]), ((u / STAGES) - 1) & 1, &abort_flag, P.err, 1))
          break;
        const int kb = P.kb0 + u / P.npairs, pr = u % P.npairs;
        const uint32_t fb = smem_u32(&bar_full[s]);
        mbar_expect_tx(fb, STAGE_BYTES);
        uint8_t* st = smem + (size_t)s * STAGE_BYTES;
        for (int c = 0; c < 4; c++)
          tma_load_3d(smem_u32(st + c * A_PLANE_BYTES), &tmA, kb * BK, m0, P.pi[pr] * 4 + c, fb);
        for (int c = 0; c < 4; c++)
          tma_load_3d(smem_u32(st + 4 * A_PLANE_BYTES + c * B_PLANE_BYTES), &tmB, kb * BK, n0, P.pj[pr] * 4 + c,
                      fb);
        issued = u + 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one lane) ----------------
    if (lane == 0) {
      for (int u = 0; u < nunits; u++) {
        const int s = u % STAGES;
        if (!mbar_wait(smem_u32(&bar_full[s]), (u / STAGES) & 1, &abort_flag, P.err, 2)) break;
        fence_after();
        uint8_t* st = smem + (size_t)s * STAGE_BYTES;
        const uint32_t a_base = smem_u32(st), b_base = smem_u32(st + 4 * A_PLANE_BYTES);
        const int pr = u % P.npairs;
        const uint32_t dacc = tmem + (uint32_t)(P.pacc[pr] * ACC_COLS);
        const bool fresh = u < P.npairs && P.pfirst[pr];  // first K block of this accumulator
#pragma unroll
        for (int kk = 0; kk < BK / 16; kk++) {
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const uint64_t ad = smem_desc_sw<C::SWB>(a_base + r * A_PLANE_BYTES + kk * 32);
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const int bp = r ^ c;
              const bool neg = (r == 1 && (c == 0 || c == 2)) || (r == 2 && (c == 0 || c == 3)) ||
                               (r == 3 && (c == 0 || c == 1));
              const uint64_t bd = smem_desc_sw<C::SWB>(b_base + bp * B_PLANE_BYTES + kk * 32);
              const uint32_t acc = (!fresh || kk > 0 || r > 0) ? 1u : 0u;
              mma_bf16(dacc + c * BN, ad, bd, neg ? IDESC_NEG_A : IDESC, acc);
            }
          }
        }
        mma_commit(smem_u32(&bar_empty[s]));
        if (u == nunits - 1) mma_commit(smem_u32(&bar_acc));
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> global ----------------
    // Each warp owns 32 accumulator rows (its TMEM lane quarter).  A 32 x 32
    // block read from TMEM (one row per thread) is transposed through shared
    // memory -- the pipeline stages are idle once the last MMA has completed --
    // so that every global access of the warp covers 32 consecutive columns
    // of one row.
    const int quarter = warp & 3;
    const int row0 = m0 + quarter * 32;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
    int have = 1;
    if (nunits > 0) {
      if (lane == 0) have = mbar_wait(smem_u32(&bar_acc), 0, &abort_flag, P.err, 3) ? 1 : 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      fence_after();
    }
    if (have) {
      long long* st64 = reinterpret_cast<long long*>(smem) + (warp - 2) * (32 * 33);
      float* st32 = reinterpret_cast<float*>(st64);
#pragma unroll 1
      for (int c = 0; c < 4; c++) {
#pragma unroll 1
        for (int ch = 0; ch < BN / 32; ch++) {
          float v[32], v2[32];
          if (nunits > 0) {
            tmem_ld32(tbase + c * BN + ch * 32, v);
            if (P.nacc == 2) tmem_ld32(tbase + ACC_COLS + c * BN + ch * 32, v2);
          } else {
#pragma unroll
            for (int t = 0; t < 32; t++) v[t] = v2[t] = 0.f;
          }
          const int col = n0 + ch * 32 + lane;
          const int nrow = min(32, P.M - row0);
          if (P.C64) {
            if (P.nacc == 2) {
#pragma unroll
              for (int t = 0; t < 32; t++)
                st64[lane * 33 + t] = __float2ll_rn(v[t] * P.scale) + __float2ll_rn(v2[t] * P.scale);
            } else {
#pragma unroll
              for (int t = 0; t < 32; t++) st64[lane * 33 + t] = __float2ll_rn(v[t] * P.scale);
            }
            __syncwarp();
            if (col < P.N) {
              long long* dst = P.C64 + c * P.ps64 + (long)row0 * P.ld64 + col;
              rmw_rows64(dst, P.ld64, nrow, st64 + lane);
            }
          } else {
#pragma unroll
            for (int t = 0; t < 32; t++) st32[lane * 33 + t] = v[t];
            __syncwarp();
            if (col < P.N) {
              float* dst = P.C.p + c * P.C.ps + (long)row0 * P.C.ld + col;
              store_rows32(dst, P.C.ld, nrow, st32 + lane);
            }
          }
          __syncwarp();
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  // Drain: if the producer stopped early, wait (bounded) for loads it issued.
  if (warp == 0 && lane == 0 && abort_flag) {
    for (int u = (issued > STAGES ? issued - STAGES : 0); u < issued; u++)
      (void)mbar_wait(smem_u32(&bar_full[u % STAGES]), (u / STAGES) & 1, &abort_flag, nullptr, 0);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

template <class C>
cudaError_t launch_cfg(const TcGemmArgs& a, KParams& P, cudaStream_t st) {
  constexpr int BK = C::BK;
  if ((a.k0 % BK) != 0 || (a.k1 != a.K && (a.k1 % BK) != 0) || a.k0 < 0 || a.k1 > a.K || a.k0 > a.k1)
    return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A->a, a.K, a.M, 4 * a.A->levels, a.A->lda, a.A->psa, BM, BK)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.B->b, a.K, a.N, 4 * a.B->levels, a.B->ldb, a.B->psb, BN, BK)) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_qgemm_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  P.kb0 = a.k0 / BK;
  P.kb1 = (a.k1 + BK - 1) / BK;
  P.Mt = (a.M + BM - 1) / BM;
  P.Nt = (a.N + BN - 1) / BN;
  k_qgemm_tc<C><<<P.Mt * P.Nt, THREADS, C::SMEM, st>>>(mA, mB, P);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace

bool tc_supported() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  return p.major == 10 && p.minor == 3 && get_encode() != nullptr;
}

cudaError_t launch_qgemm_tc(const TcGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.npairs < 1 || a.npairs > 16 || !a.A || !a.B || !a.A->a || !a.B->b) return cudaErrorInvalidValue;
  if ((a.A->lda % 8) || (a.A->psa % 8) || (a.B->ldb % 8) || (a.B->psb % 8)) return cudaErrorInvalidValue;
  int nacc = 1;
  for (int p = 0; p < a.npairs; p++) {
    if (a.pair_i[p] < 0 || a.pair_i[p] >= a.A->levels || a.pair_j[p] < 0 || a.pair_j[p] >= a.B->levels ||
        a.pair_acc[p] < 0 || a.pair_acc[p] > 1)
      return cudaErrorInvalidValue;
    if (a.pair_acc[p] == 1) nacc = 2;
  }
  if (nacc == 2 && !a.C64) return cudaErrorInvalidValue;  // two accumulators only sum into int64
  KParams P;
  P.M = a.M;
  P.N = a.N;
  P.npairs = a.npairs;
  bool seen[2] = {false, false};
  for (int p = 0; p < 16; p++) {
    P.pi[p] = p < a.npairs ? a.pair_i[p] : 0;
    P.pj[p] = p < a.npairs ? a.pair_j[p] : 0;
    P.pacc[p] = p < a.npairs ? a.pair_acc[p] : 0;
    P.pfirst[p] = 0;
    if (p < a.npairs && !seen[P.pacc[p]]) {
      P.pfirst[p] = 1;
      seen[P.pacc[p]] = true;
    }
  }
  P.nacc = nacc;
  P.C = a.C;
  P.C64 = a.C64;
  P.ld64 = a.ld64;
  P.ps64 = a.ps64;
  P.scale = ldexpf(1.0f, a.shift);
  P.err = a.err;
  return nacc == 2 ? launch_cfg<CfgDeep>(a, P, st) : launch_cfg<CfgWide>(a, P, st);
}

}  // namespace qp
