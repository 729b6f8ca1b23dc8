// qgemm_emu.cu -- FP64-accurate quaternion GEMM from exact BF16 slices in ONE
// tensor-core launch.
//
// Operands arrive as S exact slices per entry (row / column power-of-two
// scaling, balanced 7-bit digits; see slice_store in elementwise.cu), so
// A B = sum over slice pairs (s, t) of A_s B_t, and level d = s + t carries
// the weight 2^-7(d+2).  Levels 0..S-1 are formed.  Every FP32 partial sum of
// a level is an exact integer (in units of the level) as long as the K range
// it spans is short enough (host-chosen chunk per level); the two lowest
// levels run over the whole K.
//
// A persistent grid (one CTA per SM) walks work items (tile, component
// pair, level group) over 128 x 128 quaternion tiles: an item computes two
// of the four output components (0-1 or 2-3) of its tile for one of two
// level groups of equal cost, each group summed into its own int64
// accumulator, so that 4 x tiles items balance over the SMs.  For each level
// of its item the MMA warps accumulate K-chunks into two FP32 TMEM buffers in
// turn (256 columns each: the pair's two components x 128 columns), so the
// tensor core fills one while the eight epilogue warps drain the other (one
// MMA-issuing warp per component of the pair, so that one thread's issue
// rate does not bound the tensor core): each epilogue warp converts its 32
// rows x 128 columns of one component exactly to int32 and adds them into
// the level's sums, held in its registers (128 per thread), then releases
// the buffer.  At the end of a level the int32 sums are shifted to the
// common 64-bit fixed point and added to the global int64 accumulator of the
// item's group (each thread its own row segment, 16-byte accesses; the
// group's first level stores, so the accumulators need no clearing).  Global
// traffic per product is one read-modify-write of an accumulator per level
// instead of one per chunk, and there is a single launch per product.
//
// Tile shape: every MMA of an item reads one 128 x 16 A tile and one 128 x 16
// B tile for a 128 x 128 x 16 product; with 64-column tiles and all four
// components per item (the earlier shape) each 128 x 64 x 16 MMA read a
// 128 x 16 A and a 64 x 16 B tile, and the tensor core's shared-memory operand
// reads held it at 58 % pipe activity.  A component pair reads all four A and
// B planes per K step (each component takes every plane once), so the TMA
// traffic per MMA work is a third higher than with four components.  Staging
// A in tensor memory with tcgen05.cp instead was measured slower (10.7
// against 9.2 ms for the 8-slice 2048^3 product, 64-column shape).
//
// int32 range: a level-d sum is bounded by 4K 2^12 (d + 3) (2^14 for d = 0)
// level units; launch_qgemm_emu refuses K beyond what keeps this below 2^31.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qp {
namespace {

constexpr int EBM = 128, EBN = 128, EBK = 32, ESWB = 64;
constexpr int ESTAGES = 3;
constexpr int EA_PLANE = EBM * EBK * 2;                    // 8 KB
constexpr int EB_PLANE = EBN * EBK * 2;                    // 8 KB
constexpr int ESTAGE = 4 * (EA_PLANE + EB_PLANE);          // 64 KB
constexpr int ESMEM = ESTAGES * ESTAGE + 1024;             // + alignment slack
constexpr int EEPI_WARPS = 8;                              // two per TMEM lane quarter
constexpr int EMMA_WARPS = 2;                              // MMA issuers: one per component of the item
constexpr int EEPI0 = 1 + EMMA_WARPS;                      // first epilogue warp
constexpr int ETHREADS = 32 * (EEPI0 + EEPI_WARPS);        // TMA warp, MMA warps, epilogue warps
constexpr int EGROUP_M = 16;
// A work item computes two of the four output components (a component
// pair) of a 128 x 128 tile.  TMEM columns: two FP32 chunk accumulators of
// 256 columns (the pair's first component at 0, the second at EBN): the
// MMAs of chunk w fill buffer w % 2 while the epilogue drains the other.
constexpr uint32_t ECHUNK_COLS = 2 * EBN;
static_assert(ESMEM <= 227 * 1024, "shared memory per CTA");
static_assert(2 * ECHUNK_COLS == 512, "TMEM columns");

constexpr uint32_t EIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(EBN >> 3) << 17) |
                            ((uint32_t)(EBM >> 4) << 24);

// The 4 signed MMAs of one K = 16 step that feed output component c (its
// accumulator at d_tmem): A plane r times B plane r xor c, the sign of block
// (r, c) of M(B) in the negate-A bit.
__device__ __forceinline__ void qmma_k16_comp(uint32_t d_tmem, int c, uint64_t ad0, uint64_t bd0, bool fresh) {
  constexpr uint32_t NEG_A = 1u << 13;
#pragma unroll
  for (int r = 0; r < 4; r++)
    mma_bf16(d_tmem, ad0 + ((r * EA_PLANE) >> 4), bd0 + (((r ^ c) * EB_PLANE) >> 4),
             qsign_neg(r, c) ? EIDESC | NEG_A : EIDESC, (fresh && r == 0) ? 0u : 1u);
}

struct EParams {
  int M, N, K, S;
  int Mt, Nt;
  int kc[8];  // K chunk of each level (elements; multiple of EBK, or >= K)
  // Work items (tile, component pair, group): the levels are split into
  // `ngroups` groups of about equal cost (level d costs d + 1 slice pairs),
  // each with its own int64 accumulator, so that CTAs share a tile without
  // atomics and the persistent grid balances (tiles x 2 x groups) items.
  int ngroups, items;
  int nlv[2], lv[2][8];  // levels of each group, largest first
  long long* C64g[2];
  long ld64, ps64;
  int shift;  // int64 fixed point: value * 2^shift
  int* err;
};

// Grouped rasterization of tile t: consecutive tiles walk EGROUP_M row tiles.
__device__ __forceinline__ void tile_origin(const EParams& P, int t, int& m0, int& n0) {
  const int per_group = EGROUP_M * P.Nt, group = t / per_group, local = t % per_group;
  const int gm = min(EGROUP_M, P.Mt - group * EGROUP_M);
  m0 = (group * EGROUP_M + local % gm) * EBM;
  n0 = (local / gm) * EBN;
}

// int64 += v, or = v for the group's first level (two columns when both
// exist and the address is 16-byte aligned).
__device__ __forceinline__ void add64_pair(long long* dst, long long v0, long long v1, bool two, bool first) {
  if (two && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
    longlong2 g = first ? make_longlong2(0, 0) : *reinterpret_cast<longlong2*>(dst);
    g.x += v0;
    g.y += v1;
    *reinterpret_cast<longlong2*>(dst) = g;
  } else {
    dst[0] = first ? v0 : dst[0] + v0;
    if (two) dst[1] = first ? v1 : dst[1] + v1;
  }
}

__global__ void __launch_bounds__(ETHREADS, 1)
    k_qgemm_emu(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, EParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[ESTAGES], bar_empty[ESTAGES], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < ESTAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), EMMA_WARPS);  // one commit per MMA issuer
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&bar_acc_full[b]), EMMA_WARPS);
      mbar_init(smem_u32(&bar_acc_empty[b]), EEPI_WARPS);  // one arrival per epilogue warp
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

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int u = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < P.items && ok; item += gridDim.x) {
       const int g = item % P.ngroups;
       int m0, n0;
       tile_origin(P, item / (2 * P.ngroups), m0, n0);
       for (int li = 0; li < P.nlv[g] && ok; li++) {
        const int d = P.lv[g][li];
        for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d]) {
          const int kb0 = k0 / EBK, kb1 = (min(P.K, k0 + P.kc[d]) + EBK - 1) / EBK;
          for (int kb = kb0; kb < kb1 && ok; kb++) {
            for (int s = 0; s <= d; s++, u++) {
              const int st = u % ESTAGES;
              if (u >= ESTAGES &&
                  !mbar_wait(smem_u32(&bar_empty[st]), ((u / ESTAGES) - 1) & 1, &abort_flag, P.err, 11)) {
                ok = false;
                break;
              }
              const uint32_t fb = smem_u32(&bar_full[st]);
              mbar_expect_tx(fb, ESTAGE);
              uint8_t* sp = smem + (size_t)st * ESTAGE;
              for (int c = 0; c < 4; c++)
                tma_load_3d(smem_u32(sp + c * EA_PLANE), &tmA, kb * EBK, m0, s * 4 + c, fb);
              for (int c = 0; c < 4; c++)
                tma_load_3d(smem_u32(sp + 4 * EA_PLANE + c * EB_PLANE), &tmB, kb * EBK, n0, (d - s) * 4 + c, fb);
              issued = u + 1;
            }
          }
        }
       }
      }
    }
  } else if (warp < EEPI0) {
    // ---------------- MMA issuers: warp 1 the pair's first component, warp 2 its second ----------------
    if (lane == 0) {
      const int half = warp - 1;
      int u = 0, w = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < P.items && ok; item += gridDim.x) {
       const int g = item % P.ngroups;
       const int c = 2 * ((item / P.ngroups) & 1) + half;  // output component of this issuer
       for (int li = 0; li < P.nlv[g] && ok; li++) {
        const int d = P.lv[g][li];
        for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d], w++) {
          // buffer w % 2 is free once the epilogue has read chunk w - 2
          const int b = w & 1;
          if (w >= 2 && !mbar_wait(smem_u32(&bar_acc_empty[b]), ((w >> 1) - 1) & 1, &abort_flag, P.err, 12)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t dacc = tmem + b * ECHUNK_COLS + half * EBN;
          const int kb0 = k0 / EBK, kb1 = (min(P.K, k0 + P.kc[d]) + EBK - 1) / EBK;
          bool first = true;
          for (int kb = kb0; kb < kb1 && ok; kb++) {
            for (int s = 0; s <= d; s++, u++) {
              const int st = u % ESTAGES;
              if (!mbar_wait(smem_u32(&bar_full[st]), (u / ESTAGES) & 1, &abort_flag, P.err, 13)) {
                ok = false;
                break;
              }
              fence_after();
              uint8_t* sp = smem + (size_t)st * ESTAGE;
              const uint64_t ad0 = smem_desc_sw<ESWB>(smem_u32(sp)),
                             bd0 = smem_desc_sw<ESWB>(smem_u32(sp + 4 * EA_PLANE));
#pragma unroll
              for (int kk = 0; kk < EBK / 16; kk++)
                qmma_k16_comp(dacc, c, ad0 + kk * 2, bd0 + kk * 2, first && kk == 0);
              first = false;
              mma_commit(smem_u32(&bar_empty[st]));
            }
          }
          if (ok) mma_commit(smem_u32(&bar_acc_full[b]));
        }
       }
      }
    }
  } else {
    // ---------------- epilogue: exact FP32 -> int32 per chunk (registers), int64 per level ----------------
    // Warp e = warp - EEPI0 reads TMEM lane quarter warp % 4 (its 32 rows) and
    // the column half e / 4 (one component of the item's pair, 128 columns):
    // 128 int32 level sums per thread.
    const int e = warp - EEPI0, quarter = warp & 3, half = e >> 2;
    const uint32_t tb0 = tmem + ((uint32_t)(quarter * 32) << 16) + half * EBN;
    int w = 0;
    bool ok = true;
    int acc[128];
    for (int item = blockIdx.x; item < P.items && ok; item += gridDim.x) {
     const int g = item % P.ngroups;
     const int c = 2 * ((item / P.ngroups) & 1) + half;  // this warp's output component
     int m0, n0;
     tile_origin(P, item / (2 * P.ngroups), m0, n0);
     const int row = m0 + quarter * 32 + lane;
     long long* const C64 = P.C64g[g];
     for (int li = 0; li < P.nlv[g] && ok; li++) {
      const int d = P.lv[g][li];
      const float scale = ldexpf(1.0f, 7 * (d + 2));  // level unit -> integer (a power of two: exact)
      const int sh = P.shift - 7 * (d + 2);
      for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d], w++) {
        const int b = w & 1;
        const uint32_t tb = tb0 + b * ECHUNK_COLS;
        int have = 1;
        if (lane == 0) have = mbar_wait(smem_u32(&bar_acc_full[b]), (w >> 1) & 1, &abort_flag, P.err, 14) ? 1 : 0;
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
        // every FP32 value of the chunk is in registers: release the buffer
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_acc_empty[b]));
        const bool last = k0 + P.kc[d] >= P.K;
        if (!last || row >= P.M) continue;
        // level done: int64 += int32 * 2^sh (rounded shift when sh < 0), this
        // thread's row of component c, 128 columns
#pragma unroll
        for (int p = 0; p < 4; p++) {
          const int j0 = n0 + p * 32;
          long long* dst = C64 + c * P.ps64 + (long)row * P.ld64 + j0;
#pragma unroll
          for (int t = 0; t < 32; t += 2) {
            if (j0 + t >= P.N) break;
            const long long x0 = (long long)acc[p * 32 + t], x1 = (long long)acc[p * 32 + t + 1];
            const long long y0 = sh >= 0 ? (x0 << sh) : ((x0 + (1LL << (-sh - 1))) >> (-sh));
            const long long y1 = sh >= 0 ? (x1 << sh) : ((x1 + (1LL << (-sh - 1))) >> (-sh));
            add64_pair(dst + t, y0, y1, j0 + t + 1 < P.N, li == 0);
          }
        }
      }
     }
    }
  }

  fence_before();
  __syncthreads();
  if (warp == 0 && lane == 0 && abort_flag) {
    for (int u = (issued > ESTAGES ? issued - ESTAGES : 0); u < issued; u++)
      (void)mbar_wait(smem_u32(&bar_full[u % ESTAGES]), (u / ESTAGES) & 1, &abort_flag, nullptr, 0);
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace

bool emu_fused_ok(int K, int S) {
  if (S < 1 || S > 8 || K < 1) return false;
  const double lvl0 = 4.0 * K * 16384.0, lvlhi = 4.0 * K * 4096.0 * (S + 2);
  return lvl0 < 2147483648.0 && lvlhi < 2147483648.0;
}

cudaError_t launch_qgemm_emu(const EmuGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  if (!a.A || !a.B || !a.A->a || !a.B->b || !a.C64 || !emu_fused_ok(a.K, a.S)) return cudaErrorInvalidValue;
  if (a.A->levels < a.S || a.B->levels < a.S) return cudaErrorInvalidValue;
  if ((a.A->lda % 8) || (a.A->psa % 8) || (a.B->ldb % 8) || (a.B->psb % 8)) return cudaErrorInvalidValue;
  EParams P;
  P.M = a.M;
  P.N = a.N;
  P.K = a.K;
  P.S = a.S;
  for (int d = 0; d < 8; d++) {
    const int kc = d < a.S ? a.kc[d] : a.K;
    if (kc < a.K && (kc <= 0 || kc % EBK)) return cudaErrorInvalidValue;
    P.kc[d] = kc < a.K ? kc : a.K;
  }
  // level groups: largest cost first, each to the lighter group
  P.ngroups = a.C64b ? 2 : 1;
  P.nlv[0] = P.nlv[1] = 0;
  int load[2] = {0, 0};
  for (int d = a.S - 1; d >= 0; d--) {
    const int g = (P.ngroups == 2 && load[1] < load[0]) ? 1 : 0;
    P.lv[g][P.nlv[g]++] = d;
    load[g] += d + 1;
  }
  P.C64g[0] = a.C64;
  P.C64g[1] = a.C64b ? a.C64b : a.C64;
  P.ld64 = a.ld64;
  P.ps64 = a.ps64;
  P.shift = a.shift;
  P.err = a.err;

  P.Mt = (a.M + EBM - 1) / EBM;
  P.Nt = (a.N + EBN - 1) / EBN;
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A->a, a.K, a.M, 4 * a.A->levels, a.A->lda, a.A->psa, EBM, EBK)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.B->b, a.K, a.N, 4 * a.B->levels, a.B->ldb, a.B->psb, EBN, EBK)) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k_qgemm_emu, ESMEM, attr_done)) return e;
  P.items = P.Mt * P.Nt * 2 * P.ngroups;
  static int nsm[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidValue;
  if (!nsm[dev] && cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  const int grid = std::min(P.items, nsm[dev]);  // persistent: one CTA per SM
  k_qgemm_emu<<<grid, ETHREADS, ESMEM, st>>>(mA, mB, P);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
