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

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qp {
namespace {

constexpr int BM = 128;  // output rows per CTA = TMEM lanes
constexpr int BN = 64;   // quaternion output columns per CTA (per component) of the 64-column shapes
constexpr int ACC_COLS = 4 * BN;  // TMEM columns of one 64-column accumulator (four output components)
constexpr int GROUP_M = 16;       // CTA rasterization: 16 row tiles per group share B tiles in L2

// Stage shape.  BK BF16 K-elements per stage = one swizzle row of 2*BK bytes.
//   Wide: BK = 32 (64-byte swizzle), 48 KB per stage, two CTAs per SM, so one
//         CTA's epilogue overlaps the other's main loop (one accumulator).
//   Deep: BK = 64 (128-byte swizzle), 96 KB per stage, one CTA per SM (two
//         accumulators take all 512 TMEM columns).
//   Broad: BK = 32, 128 columns per CTA (a 512-column accumulator), three
//         64 KB stages, one CTA per SM: twice the MMA work per operand tile
//         read of the wide shape.
template <int BK_, int SWB_, int MINB_, int BN_ = 64, int STAGES_ = 2>
struct Cfg {
  static constexpr int BK = BK_;
  static constexpr int SWB = SWB_;
  static constexpr int MINB = MINB_;
  static constexpr int BN = BN_;
  static constexpr int ACC = 4 * BN_;  // TMEM columns of one accumulator
  static constexpr int STAGES = STAGES_;
  static constexpr int A_PLANE = BM * BK * 2;
  static constexpr int B_PLANE = BN * BK * 2;
  static constexpr int STAGE = 4 * (A_PLANE + B_PLANE);
  static constexpr int SMEM = STAGES * STAGE + 1024;
  // Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = BM, N = BN.
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                    ((uint32_t)(BM >> 4) << 24);
};
using CfgWide = Cfg<32, 64, 2>;
using CfgDeep = Cfg<64, 128, 1>;
using CfgBroad = Cfg<32, 64, 1, 128, 3>;
static_assert(CfgWide::SMEM * 2 <= 227 * 1024, "two wide CTAs per SM");
static_assert(CfgDeep::SMEM * 2 > 228 * 1024, "one deep CTA per SM");
static_assert(CfgBroad::SMEM <= 227 * 1024 && CfgBroad::ACC == 512, "one broad CTA per SM, all TMEM columns");
constexpr int THREADS = 192;

static_assert(ACC_COLS == 256, "TMEM allocations must be powers of two (256 or 512 columns)");


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
  EpiArgs E;       // E.nout > 0: fused combine epilogue (FP32 output only)
  long long* C64;  // non-null: int64 fixed-point accumulation
  long ld64, ps64;
  float scale;     // 2^shift
  int* err;
};

__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Fused combine for 16 consecutive columns j0.. of row i (this lane), plane c:
// v = the product's values; see EpiArgs.  nc = valid columns (1..16, the
// same for the whole warp); rok = row i exists (the whole warp calls this:
// the transposed B-form goes through `stg`, this warp's 16 x 32 BF16 block
// of shared memory, so that each lane writes 16-byte pieces of B-form rows).
// T is the master type of the aux inputs and the output masters (float, or
// double when E.f64: the combine's arithmetic then runs in FP64 and the split
// forms are taken from the FP32 rounding of the result, as in the combine
// kernel).
template <typename T>
__device__ __forceinline__ void epi_piece_t(const EpiArgs& E, int c, int i, bool rok, int row0, int M, int j0, int nc,
                                            const float* v, bf16* stg, float& sdx, float& sx, int& bad) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int o = 0; o < E.nout; o++) {
    const EpiOut& O = E.out[o];
    T w[16];
    const T cacc = (T)O.cacc;
#pragma unroll
    for (int t = 0; t < 16; t++)  // +-1 as a sign flip (the combine kernel's arithmetic)
      w[t] = cacc == (T)0 ? (T)0 : cacc == (T)1 ? (T)v[t] : cacc == (T)-1 ? -(T)v[t] : cacc * (T)v[t];
#pragma unroll 1
    for (int a = 0; a < 4; a++) {
      if (!rok || !E.aux[a] || O.caux[a] == 0.0) continue;
      const T* ap = reinterpret_cast<const T*>(E.aux[a]) + c * E.ps_aux[a] + (long)i * E.ld_aux[a] + j0;
      const T ca = (T)O.caux[a];
      if (sizeof(T) == 4 && nc == 16 && al16(ap)) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const float4 u = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(ap))[q];
          w[4 * q] += ca * u.x;
          w[4 * q + 1] += ca * u.y;
          w[4 * q + 2] += ca * u.z;
          w[4 * q + 3] += ca * u.w;
        }
      } else if (sizeof(T) == 8 && nc == 16 && al16(ap)) {
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const double2 u = reinterpret_cast<const double2*>(reinterpret_cast<const double*>(ap))[q];
          w[2 * q] += ca * u.x;
          w[2 * q + 1] += ca * u.y;
        }
      } else {
#pragma unroll
        for (int t = 0; t < 16; t++)
          if (t < nc) w[t] += ca * ap[t];
      }
    }
    if (c == 0 && O.diag != 0.0) {
#pragma unroll
      for (int t = 0; t < 16; t++)
        if (i == j0 + t) w[t] += (T)O.diag;
    }
    if (o == 0 && E.partials && rok) {
      const T* xp = E.aux[0] ? reinterpret_cast<const T*>(E.aux[0]) + c * E.ps_aux[0] + (long)i * E.ld_aux[0] + j0
                             : nullptr;
#pragma unroll
      for (int t = 0; t < 16; t++)
        if (t < nc) {
          const float x0 = xp ? (float)(w[t] - xp[t]) : (float)w[t];
          sdx += x0 * x0;
          sx += (float)w[t] * (float)w[t];
          bad += isfinite(w[t]) ? 0 : 1;
        }
    }
    if (O.mp && rok) {
      T* dst = reinterpret_cast<T*>(O.mp) + c * O.mps + (long)i * O.mld + j0;
      if (sizeof(T) == 4 && nc == 16 && al16(dst)) {
#pragma unroll
        for (int q = 0; q < 4; q++)
          reinterpret_cast<float4*>(reinterpret_cast<float*>(dst))[q] =
              make_float4((float)w[4 * q], (float)w[4 * q + 1], (float)w[4 * q + 2], (float)w[4 * q + 3]);
      } else if (sizeof(T) == 8 && nc == 16 && al16(dst)) {
#pragma unroll
        for (int q = 0; q < 8; q++)
          reinterpret_cast<double2*>(reinterpret_cast<double*>(dst))[q] =
              make_double2((double)w[2 * q], (double)w[2 * q + 1]);
      } else {
#pragma unroll
        for (int t = 0; t < 16; t++)
          if (t < nc) dst[t] = w[t];
      }
    }
    if (O.a || O.b) {
      float r[16];
#pragma unroll
      for (int t = 0; t < 16; t++) r[t] = (float)w[t];
#pragma unroll 1
      for (int l = 0; l < O.levels; l++) {
        bf16 h[16];
#pragma unroll
        for (int t = 0; t < 16; t++) {
          h[t] = __float2bfloat16_rn(r[t]);
          r[t] -= __bfloat162float(h[t]);
        }
        if (O.a && rok) {
          bf16* dst = O.a + (long)l * 4 * O.psa + c * O.psa + (long)i * O.lda + j0;
          if (nc == 16 && al16(dst)) {
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; q++)
              pk[q] = (uint32_t)__bfloat16_as_ushort(h[2 * q]) | ((uint32_t)__bfloat16_as_ushort(h[2 * q + 1]) << 16);
            reinterpret_cast<uint4*>(dst)[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            reinterpret_cast<uint4*>(dst)[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
          } else {
#pragma unroll
            for (int t = 0; t < 16; t++)
              if (t < nc) dst[t] = h[t];
          }
        }
        if (O.b) {
          // B-form row j holds column j of the output (rows row0 .. row0 + 31
          // contiguous): transpose the warp's 32 x 16 block through shared
          // memory, then lane q writes 8 rows of column q / 4 (16 bytes), twice
#pragma unroll
          for (int t = 0; t < 16; t++) stg[t * 32 + lane] = h[t];
          __syncwarp();
          bf16* bl = O.b + (long)l * 4 * O.psb + c * O.psb;
#pragma unroll
          for (int k = 0; k < 2; k++) {
            const int q = lane + 32 * k, t = q >> 2, part = q & 3;
            const int r0 = row0 + part * 8;
            if (t < nc && r0 < M) {
              bf16* dst = bl + (long)(j0 + t) * O.ldb + r0;
              const bf16* src = stg + t * 32 + part * 8;
              if (r0 + 8 <= M && al16(dst)) {
                *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
              } else {
                for (int x = 0; x < 8 && r0 + x < M; x++) dst[x] = src[x];
              }
            }
          }
          __syncwarp();
        }
      }
    }
  }
}

__device__ __forceinline__ void epi_piece(const EpiArgs& E, int c, int i, bool rok, int row0, int M, int j0, int nc,
                                          const float* v, bf16* stg, float& sdx, float& sx, int& bad) {
  if (E.f64)
    epi_piece_t<double>(E, c, i, rok, row0, M, j0, nc, v, stg, sdx, sx, bad);
  else
    epi_piece_t<float>(E, c, i, rok, row0, M, j0, nc, v, stg, sdx, sx, bad);
}

template <class C>
__global__ void __launch_bounds__(THREADS, C::MINB)
    k_qgemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, KParams P) {
  constexpr int BK = C::BK, STAGES = C::STAGES, A_PLANE_BYTES = C::A_PLANE, B_PLANE_BYTES = C::B_PLANE,
                STAGE_BYTES = C::STAGE, BN = C::BN, ACC_COLS = C::ACC;
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
        const uint64_t ad0 = smem_desc_sw<C::SWB>(smem_u32(st)),
                       bd0 = smem_desc_sw<C::SWB>(smem_u32(st + 4 * A_PLANE_BYTES));
        const int pr = u % P.npairs;
        const uint32_t dacc = tmem + (uint32_t)(P.pacc[pr] * ACC_COLS);
        const bool fresh = u < P.npairs && P.pfirst[pr];  // first K block of this accumulator
#pragma unroll
        for (int kk = 0; kk < BK / 16; kk++)
          qmma_k16<A_PLANE_BYTES, B_PLANE_BYTES>(dacc, BN, ad0 + kk * 2, bd0 + kk * 2, C::IDESC, fresh && kk == 0);
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
    if (have && P.E.nout > 0) {
      // fused combine: one row per lane, 16 columns at a time, straight from TMEM;
      // the idle pipeline stages give each warp 1 KB for the B-form transpose
      const int i = row0 + lane;
      bf16* stg = reinterpret_cast<bf16*>(smem) + (warp - 2) * 512;
      float sdx = 0.f, sx = 0.f;
      int bad = 0;
#pragma unroll 1
      for (int c = 0; c < 4; c++) {
#pragma unroll 1
        for (int ch = 0; ch < BN / 16; ch++) {
          float v[16];
          if (nunits > 0) {
            tmem_ld16(tbase + c * BN + ch * 16, v);
          } else {
#pragma unroll
            for (int t = 0; t < 16; t++) v[t] = 0.f;
          }
          const int j0 = n0 + ch * 16;
          const int nc = min(16, P.N - j0);
          if (nc > 0) epi_piece(P.E, c, i, i < P.M, row0, P.M, j0, nc, v, stg, sdx, sx, bad);
        }
      }
      if (P.E.partials) {
        double d0 = sdx, d1 = sx, d2 = bad;
        for (int o = 16; o > 0; o >>= 1) {
          d0 += __shfl_xor_sync(0xffffffffu, d0, o);
          d1 += __shfl_xor_sync(0xffffffffu, d1, o);
          d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        }
        if (lane == 0) {
          double* pp = P.E.partials + 3 * ((long)blockIdx.x * 4 + quarter);
          pp[0] = d0;
          pp[1] = d1;
          pp[2] = d2;
        }
      }
    } else if (have) {
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

// Persistent shape for products with the fused combine epilogue: work items
// (128 x 128 tile, component pair), one CTA per SM, two accumulators of 256
// TMEM columns (the pair's two components x 128 columns) used by items in
// turn, so the epilogue warps run the combine of one item while the MMA
// warp accumulates the next.  Each 128 x 128 x 16 MMA reads a 128 x 16 A and
// a 128 x 16 B tile (one operand wavefront per pipe cycle, against 1.5 for
// the 64-column shape); an item takes all four A and B planes of a K step
// (each output component uses every plane once).  Same MMAs per output
// entry in the same order as the other shapes: bit-identical products.
constexpr int CP_BN = 128, CP_BK = 32, CP_STAGES = 3;
constexpr int CP_A_PLANE = BM * CP_BK * 2, CP_B_PLANE = CP_BN * CP_BK * 2;
constexpr int CP_STAGE = 4 * (CP_A_PLANE + CP_B_PLANE);  // 64 KB
constexpr int CP_EPI_WARPS = 8;                          // two per TMEM lane quarter: one per component
constexpr int CP_THREADS = 32 * (2 + CP_EPI_WARPS);      // TMA warp, MMA warp, epilogue warps
constexpr int CP_STG = CP_EPI_WARPS * 1024;              // the epilogue warps' B-form transpose tiles
constexpr int CP_SMEM = CP_STAGES * CP_STAGE + CP_STG + 1024;
constexpr uint32_t CP_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CP_BN >> 3) << 17) |
                              ((uint32_t)(BM >> 4) << 24);
static_assert(CP_SMEM <= 227 * 1024, "shared memory per CTA");

// The 4 signed MMAs of one K = 16 step into output component c (accumulator at d_tmem).
__device__ __forceinline__ void qmma_k16_one(uint32_t d_tmem, int c, uint64_t ad0, uint64_t bd0, bool fresh) {
  constexpr uint32_t NEG_A = 1u << 13;
#pragma unroll
  for (int r = 0; r < 4; r++)
    mma_bf16(d_tmem, ad0 + ((r * CP_A_PLANE) >> 4), bd0 + (((r ^ c) * CP_B_PLANE) >> 4),
             qsign_neg(r, c) ? CP_IDESC | NEG_A : CP_IDESC, (fresh && r == 0) ? 0u : 1u);
}

__global__ void __launch_bounds__(CP_THREADS, 1)
    k_qgemm_tc_pairs(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, KParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[CP_STAGES], bar_empty[CP_STAGES], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = (P.kb1 - P.kb0) * P.npairs;  // (K block, split pair) units per item
  const int items = P.Mt * P.Nt * 2;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < CP_STAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&bar_acc_full[b]), 1);
      mbar_init(smem_u32(&bar_acc_empty[b]), CP_EPI_WARPS);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;

  auto item_origin = [&](int item, int& m0, int& n0, int& c0) {
    const int t = item >> 1;
    c0 = 2 * (item & 1);
    const int per_group = GROUP_M * P.Nt, group = t / per_group, local = t % per_group;
    const int gm = min(GROUP_M, P.Mt - group * GROUP_M);
    m0 = (group * GROUP_M + local % gm) * BM;
    n0 = (local / gm) * CP_BN;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int u = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        int m0, n0, c0;
        item_origin(item, m0, n0, c0);
        for (int x = 0; x < units; x++, u++) {
          const int s = u % CP_STAGES;
          if (u >= CP_STAGES &&
              !mbar_wait(smem_u32(&bar_empty[s]), ((u / CP_STAGES) - 1) & 1, &abort_flag, P.err, 41)) {
            ok = false;
            break;
          }
          const int kb = P.kb0 + x / P.npairs, pr = x % P.npairs;
          const uint32_t fb = smem_u32(&bar_full[s]);
          mbar_expect_tx(fb, CP_STAGE);
          uint8_t* st = smem + (size_t)s * CP_STAGE;
          for (int c = 0; c < 4; c++)
            tma_load_3d(smem_u32(st + c * CP_A_PLANE), &tmA, kb * CP_BK, m0, P.pi[pr] * 4 + c, fb);
          for (int c = 0; c < 4; c++)
            tma_load_3d(smem_u32(st + 4 * CP_A_PLANE + c * CP_B_PLANE), &tmB, kb * CP_BK, n0, P.pj[pr] * 4 + c, fb);
          issued = u + 1;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (one lane): both components of the item's pair ----------------
    if (lane == 0) {
      int u = 0, w = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < items && ok; item += gridDim.x, w++) {
        int m0, n0, c0;
        item_origin(item, m0, n0, c0);
        const int b = w & 1;
        if (w >= 2 && !mbar_wait(smem_u32(&bar_acc_empty[b]), ((w >> 1) - 1) & 1, &abort_flag, P.err, 42)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t dacc = tmem + b * 256;
        for (int x = 0; x < units && ok; x++, u++) {
          const int s = u % CP_STAGES;
          if (!mbar_wait(smem_u32(&bar_full[s]), (u / CP_STAGES) & 1, &abort_flag, P.err, 43)) {
            ok = false;
            break;
          }
          fence_after();
          uint8_t* st = smem + (size_t)s * CP_STAGE;
          const uint64_t ad0 = smem_desc_sw<64>(smem_u32(st)), bd0 = smem_desc_sw<64>(smem_u32(st + 4 * CP_A_PLANE));
          const bool fresh = x < P.npairs && P.pfirst[x % P.npairs];  // first K block of the accumulator
#pragma unroll
          for (int kk = 0; kk < CP_BK / 16; kk++) {
            qmma_k16_one(dacc, c0, ad0 + kk * 2, bd0 + kk * 2, fresh && kk == 0);
            qmma_k16_one(dacc + CP_BN, c0 + 1, ad0 + kk * 2, bd0 + kk * 2, fresh && kk == 0);
          }
          mma_commit(smem_u32(&bar_empty[s]));
        }
        if (ok) mma_commit(smem_u32(&bar_acc_full[b]));
      }
    }
  } else {
    // ---------------- epilogue: the fused combine of each item, one row per lane ----------------
    // warp e = warp - 2: TMEM lane quarter warp % 4, component c0 + e / 4 of the item's pair
    const int quarter = warp & 3, e8 = warp - 2, h = e8 >> 2;
    const uint32_t tq = tmem + ((uint32_t)(quarter * 32) << 16);
    bf16* stg = reinterpret_cast<bf16*>(smem + CP_STAGES * CP_STAGE) + e8 * 512;
    float sdx = 0.f, sx = 0.f;
    int bad = 0;
    int w = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, w++) {
      int m0, n0, c0;
      item_origin(item, m0, n0, c0);
      const int b = w & 1;
      int have = 1;
      if (units > 0) {
        if (lane == 0) have = mbar_wait(smem_u32(&bar_acc_full[b]), (w >> 1) & 1, &abort_flag, P.err, 44) ? 1 : 0;
        have = __shfl_sync(0xffffffffu, have, 0);
        fence_after();
      }
      if (!have) break;
      const int row0 = m0 + quarter * 32, i = row0 + lane;
#pragma unroll 1
      for (int ch = 0; ch < CP_BN / 16; ch++) {
        float v[16];
        if (units > 0) {
          tmem_ld16(tq + b * 256 + h * CP_BN + ch * 16, v);
        } else {
#pragma unroll
          for (int t = 0; t < 16; t++) v[t] = 0.f;
        }
        const int j0 = n0 + ch * 16;
        const int nc = min(16, P.N - j0);
        if (nc > 0) epi_piece(P.E, c0 + h, i, i < P.M, row0, P.M, j0, nc, v, stg, sdx, sx, bad);
      }
      // the accumulator is read: release it to the MMA warp
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty[b]));
    }
    if (P.E.partials) {
      double d0 = sdx, d1 = sx, d2 = bad;
      for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      }
      if (lane == 0) {
        double* pp = P.E.partials + 3 * ((long)blockIdx.x * CP_EPI_WARPS + e8);
        pp[0] = d0;
        pp[1] = d1;
        pp[2] = d2;
      }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && abort_flag) {
    for (int u = (issued > CP_STAGES ? issued - CP_STAGES : 0); u < issued; u++)
      (void)mbar_wait(smem_u32(&bar_full[u % CP_STAGES]), (u / CP_STAGES) & 1, &abort_flag, nullptr, 0);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

int sm_count() {
  static int nsm[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (!nsm[dev] && cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return nsm[dev];
}

// Grid of the persistent component-pair shape: one CTA per SM at most.
int pairs_grid(int M, int N) {
  const int items = ((M + BM - 1) / BM) * ((N + CP_BN - 1) / CP_BN) * 2;
  return std::min(items, std::max(1, sm_count()));
}

cudaError_t launch_pairs(const TcGemmArgs& a, KParams& P, cudaStream_t st) {
  if ((a.k0 % CP_BK) != 0 || (a.k1 != a.K && (a.k1 % CP_BK) != 0) || a.k0 < 0 || a.k1 > a.K || a.k0 > a.k1)
    return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A->a, a.K, a.M, 4 * a.A->levels, a.A->lda, a.A->psa, BM, CP_BK)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.B->b, a.K, a.N, 4 * a.B->levels, a.B->ldb, a.B->psb, CP_BN, CP_BK))
    return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k_qgemm_tc_pairs, CP_SMEM, attr_done)) return e;
  P.kb0 = a.k0 / CP_BK;
  P.kb1 = (a.k1 + CP_BK - 1) / CP_BK;
  P.Mt = (a.M + BM - 1) / BM;
  P.Nt = (a.N + CP_BN - 1) / CP_BN;
  const int grid = pairs_grid(a.M, a.N);
  if (grid < 1) return cudaErrorInvalidValue;
  k_qgemm_tc_pairs<<<grid, CP_THREADS, CP_SMEM, st>>>(mA, mB, P);
  ++g_kernel_launches;
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_cfg(const TcGemmArgs& a, KParams& P, cudaStream_t st) {
  constexpr int BK = C::BK;
  if ((a.k0 % BK) != 0 || (a.k1 != a.K && (a.k1 % BK) != 0) || a.k0 < 0 || a.k1 > a.K || a.k0 > a.k1)
    return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A->a, a.K, a.M, 4 * a.A->levels, a.A->lda, a.A->psa, BM, BK)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.B->b, a.K, a.N, 4 * a.B->levels, a.B->ldb, a.B->psb, C::BN, BK)) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k_qgemm_tc<C>, C::SMEM, attr_done)) return e;
  P.kb0 = a.k0 / BK;
  P.kb1 = (a.k1 + BK - 1) / BK;
  P.Mt = (a.M + BM - 1) / BM;
  P.Nt = (a.N + C::BN - 1) / C::BN;
  k_qgemm_tc<C><<<P.Mt * P.Nt, THREADS, C::SMEM, st>>>(mA, mB, P);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace

// One-accumulator products with M, N >= 128 take a 128-column shape unless
// broad = 0: without a fused epilogue the broad shape (one tile per CTA,
// 128 x 128, all four components; plain products gain 10-19 %), with one
// the persistent component-pair shape (broad = -1), whose epilogue overlaps
// the MMAs of the CTA's next item -- the broad shape's one tile per CTA
// would expose it (measured: no gain on the 2048^2 solve).  broad = 1 takes
// the broad shape for both.  The fused epilogue's partials follow the shape
// chosen: one set per (CTA, epilogue warp).
enum TcShape { SHAPE_WIDE, SHAPE_BROAD, SHAPE_PAIRS };
static TcShape tc_shape(int broad, bool fused, int M, int N) {
  if (broad == 0 || N < 128 || M < 128) return SHAPE_WIDE;
  if (broad == 1 || !fused) return SHAPE_BROAD;
  return SHAPE_PAIRS;
}
int tc_partial_blocks(int M, int N, int broad) {
  switch (tc_shape(broad, true, M, N)) {
    case SHAPE_PAIRS: return pairs_grid(M, N) * CP_EPI_WARPS;
    case SHAPE_BROAD: return ((M + BM - 1) / BM) * ((N + CfgBroad::BN - 1) / CfgBroad::BN) * 4;
    default: return ((M + BM - 1) / BM) * ((N + CfgWide::BN - 1) / CfgWide::BN) * 4;
  }
}

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
  P.E = a.epi;
  if (P.E.nout < 0 || P.E.nout > kMaxOut || (P.E.nout > 0 && (a.C64 || nacc == 2)) || (P.E.f64 && P.E.partials))
    return cudaErrorInvalidValue;
  P.C64 = a.C64;
  P.ld64 = a.ld64;
  P.ps64 = a.ps64;
  P.scale = ldexpf(1.0f, a.shift);
  P.err = a.err;
  if (nacc == 2) return launch_cfg<CfgDeep>(a, P, st);
  switch (tc_shape(a.broad, P.E.nout > 0, a.M, a.N)) {
    case SHAPE_PAIRS: return launch_pairs(a, P, st);
    case SHAPE_BROAD: return launch_cfg<CfgBroad>(a, P, st);
    default: return launch_cfg<CfgWide>(a, P, st);
  }
}

}  // namespace qp
