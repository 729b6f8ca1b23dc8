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
// the four B planes of a tile in shared memory (TMA, 128-byte swizzle) and
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
// the MMAs (one elected lane), warps 2-5 drain TMEM to global memory.
// Every wait is bounded (2 s of globaltimer); on expiry the kernel records
// an error code, stops issuing work, drains what it started and frees TMEM.
#include <cuda.h>

#include "common.cuh"

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
  static constexpr unsigned long long LAYOUT = SWB == 128 ? 2ull : 4ull;  // descriptor swizzle code
  static constexpr unsigned SBO = 8 * SWB;                               // bytes between 8-row groups
};
using CfgWide = Cfg<32, 64, 2>;
using CfgDeep = Cfg<64, 128, 1>;
static_assert(CfgWide::SMEM * 2 <= 227 * 1024, "two wide CTAs per SM");
static_assert(CfgDeep::SMEM * 2 > 228 * 1024, "one deep CTA per SM");
constexpr int THREADS = 192;
constexpr unsigned long long WAIT_NS = 2000000000ull;

static_assert(ACC_COLS == 256, "TMEM allocations must be powers of two (256 or 512 columns)");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the abort flag is raised or WAIT_NS elapses (then
// raises the flag and records `code` in *err).
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err, int code) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 0) {
      if (*abort_flag) return false;
      if (gtime() - t0 > WAIT_NS) {
        *abort_flag = 1;
        if (err) atomicCAS(err, 0, code);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, swizzled rows of 2*BK bytes, 8-row groups SBO bytes apart.
template <class C>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(C::SBO >> 4) << 32) |
         ((uint64_t)1 << 46) | (C::LAYOUT << 61);
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = BM, N = BN.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 32; t++) v[t] = __uint_as_float(r[t]);
}

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
            const uint64_t ad = smem_desc<C>(a_base + r * A_PLANE_BYTES + kk * 32);
#pragma unroll
            for (int c = 0; c < 4; c++) {
              const int bp = r ^ c;
              const bool neg = (r == 1 && (c == 0 || c == 2)) || (r == 2 && (c == 0 || c == 3)) ||
                               (r == 3 && (c == 0 || c == 1));
              const uint64_t bd = smem_desc<C>(b_base + bp * B_PLANE_BYTES + kk * 32);
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
    // ---------------- epilogue: TMEM -> FP32 global ----------------
    const int quarter = warp & 3;
    const int row = m0 + quarter * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16);
    int have = 1;
    if (nunits > 0) {
      if (lane == 0) have = mbar_wait(smem_u32(&bar_acc), 0, &abort_flag, P.err, 3) ? 1 : 0;
      have = __shfl_sync(0xffffffffu, have, 0);
      fence_after();
    }
    if (have) {
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
          if (row < P.M && P.C64) {
            long long* dst = P.C64 + c * P.ps64 + (long)row * P.ld64 + n0 + ch * 32;
            const int ncol = min(32, P.N - (n0 + ch * 32));
            if (P.nacc == 2) {
              for (int t = 0; t < ncol; t++) dst[t] += __float2ll_rn(v[t] * P.scale) + __float2ll_rn(v2[t] * P.scale);
            } else {
              for (int t = 0; t < ncol; t++) dst[t] += __float2ll_rn(v[t] * P.scale);
            }
          } else if (row < P.M) {
            float* dst = P.C.p + c * P.C.ps + (long)row * P.C.ld + n0 + ch * 32;
            const int ncol = min(32, P.N - (n0 + ch * 32));
            if (ncol == 32 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
              for (int t = 0; t < 32; t += 4)
                *reinterpret_cast<float4*>(dst + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
            } else {
              for (int t = 0; t < ncol; t++) dst[t] = v[t];
            }
          }
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D map over [planes][rows][K] BF16 with a box of (bk, box_rows, 1) and a 2*bk-byte swizzle.
bool make_map(CUtensorMap* map, const bf16* base, int K, int rows, int planes, long ld, long ps, int box_rows,
              int bk) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)ps * 2};
  cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
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
