// qgemm_emu_pair.cu -- the FP64-accurate exact-slice quaternion GEMM of
// qgemm_emu.cu on pairs of SMs (tcgen05 cta_group::2).
//
// Same arithmetic as k_qgemm_emu (exact BF16 slices, level d = s + t summed
// in K chunks whose FP32 partial sums are exact, int32 level sums in the
// epilogue's registers, int64 fixed-point accumulators per level group), but
// a work item is a 256 x 64 quaternion tile computed by a cluster of two CTAs
// on two SMs with M = 256 MMAs: each CTA stages its own 128 rows of A and
// half of the tile's B (32 of the 64 columns), the first CTA of the pair
// issues the MMAs for both, and each CTA's TMEM receives its own 128 rows.
// Per SM and MMA the tensor core then reads 128 x 16 of A and 32 x 16 of B
// from its shared memory instead of 128 x 16 and 64 x 16: the single-SM
// kernel is bound by exactly those operand reads.
//
// Pair protocol (stage u, chunk w):
//   * both CTAs' TMA loads of a stage signal the first CTA's full[u % ST]
//     barrier (cta_group::2 copies), whose expected bytes cover both;
//   * the MMA commits arrive on both CTAs' empty / acc_full barriers
//     (multicast), so each producer and each epilogue waits on its own CTA;
//   * each epilogue warp of either CTA arrives on the first CTA's
//     acc_empty[w % 2] once it has drained the chunk (16 arrivals);
//   * cluster barriers after the barrier initialisation and before TMEM is
//     freed and the CTAs exit (the peer's shared memory is read by the
//     MMAs, and its epilogue arrives remotely).
// Every wait is bounded (2 s); on expiry a CTA records the error code, stops
// issuing work and still reaches the final cluster barrier.
#include <cuda.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace qp {
namespace {

constexpr int PBM = 128;        // rows per CTA (TMEM lanes); the pair tile is 2 * PBM
constexpr int PBN = 64;         // quaternion columns per pair tile
constexpr int PBN_HALF = 32;    // columns of B staged per CTA
constexpr int PBK = 32, PSWB = 64;
constexpr int PSTAGES = 5;
constexpr int PA_PLANE = PBM * PBK * 2;         // 8 KB
constexpr int PB_PLANE = PBN_HALF * PBK * 2;    // 2 KB
constexpr int PSTAGE = 4 * (PA_PLANE + PB_PLANE);  // 40 KB per CTA
// + alignment slack, + one B tile of tail so that no operand read of the
// last stage can leave the allocation
constexpr int PSMEM = PSTAGES * PSTAGE + 1024 + 4 * PBN * PBK * 2;
constexpr int PEPI_WARPS = 8;
constexpr int PMMA_WARPS = 2;
constexpr int PEPI0 = 1 + PMMA_WARPS;
constexpr int PTHREADS = 32 * (PEPI0 + PEPI_WARPS);
constexpr int PGROUP_M = 8;  // pair row tiles per rasterization group
constexpr uint32_t PCHUNK_COLS = 4 * PBN;
static_assert(PSMEM <= 227 * 1024, "shared memory per CTA");
static_assert(2 * PCHUNK_COLS == 512, "TMEM columns");

// kind::f16, D = F32, A = B = BF16, K-major, N = 64, M = 256 (the pair)
constexpr uint32_t PIDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(PBN >> 3) << 17) |
                            ((uint32_t)((2 * PBM) >> 4) << 24);

struct PParams {
  int M, N, K, S;
  int Mt, Nt;  // pair row tiles (256 rows), column tiles
  int kc[8];
  int ngroups, items;
  int nlv[2], lv[2][8];
  long long* C64g[2];
  long ld64, ps64;
  int shift;
  int* err;
};

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// The same shared-memory offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// mbarrier wait at cluster scope (arrivals come from the other CTA too), bounded.
__device__ __forceinline__ bool mbar_try_cl(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ bool mbar_wait_cl(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err, int code) {
  if (mbar_try_cl(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 1;; ++it) {
    if (mbar_try_cl(bar, parity)) return true;
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
// TMA tile load whose completion is signalled on a barrier of either CTA of the pair.
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Commit of this thread's MMAs to the barrier at `bar` in both CTAs of the pair.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          bar),
      "h"(mask)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}
// The 8 signed MMAs of one K = 16 step that feed components C0 and C0 + 1
// (the Hamilton-product signs of qsign_neg, as in qmma_k16_half).
template <int C0>
__device__ __forceinline__ void qmma_k16_pair(uint32_t d_tmem, uint64_t ad0, uint64_t bd0, bool fresh) {
  constexpr uint32_t NEG_A = 1u << 13;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const uint64_t ad = ad0 + ((r * PA_PLANE) >> 4);
    const uint32_t acc = (fresh && r == 0) ? 0u : 1u;
#pragma unroll
    for (int c = C0; c < C0 + 2; c++)
      mma_bf16_pair(d_tmem + c * PBN, ad, bd0 + (((r ^ c) * PB_PLANE) >> 4),
                    qsign_neg(r, c) ? PIDESC | NEG_A : PIDESC, acc);
  }
}

// Grouped rasterization of pair tile t.
__device__ __forceinline__ void pair_tile_origin(const PParams& P, int t, int& m0, int& n0) {
  const int per_group = PGROUP_M * P.Nt, group = t / per_group, local = t % per_group;
  const int gm = min(PGROUP_M, P.Mt - group * PGROUP_M);
  m0 = (group * PGROUP_M + local % gm) * (2 * PBM);
  n0 = (local / gm) * PBN;
}

__device__ __forceinline__ void add64_pair2(long long* dst, long long v0, long long v1, bool two, bool first) {
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

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PTHREADS, 1)
    k_qgemm_emu_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, PParams P) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t bar_full[PSTAGES], bar_empty[PSTAGES], bar_acc_full[2], bar_acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cta_rank();  // 0: issues the MMAs of the pair
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < PSTAGES; s++) {
      mbar_init(smem_u32(&bar_full[s]), 1);              // the first CTA's producer; bytes of both CTAs
      mbar_init(smem_u32(&bar_empty[s]), PMMA_WARPS);    // one commit per MMA issuer (multicast)
    }
    for (int b = 0; b < 2; b++) {
      mbar_init(smem_u32(&bar_acc_full[b]), PMMA_WARPS);
      mbar_init(smem_u32(&bar_acc_empty[b]), 2 * PEPI_WARPS);  // epilogue warps of both CTAs
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any remote arrival or copy
  fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;

  if (warp == 0) {
    // ---------------- TMA producer (each CTA: its A rows and its half of B) ----------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      int u = 0;
      bool ok = true;
      for (int item = pair; item < P.items && ok; item += npairs) {
        const int g = item % P.ngroups;
        int m0, n0;
        pair_tile_origin(P, item / P.ngroups, m0, n0);
        const int ma = m0 + (int)rank * PBM, nb = n0 + (int)rank * PBN_HALF;
        for (int li = 0; li < P.nlv[g] && ok; li++) {
          const int d = P.lv[g][li];
          for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d]) {
            const int kb0 = k0 / PBK, kb1 = (min(P.K, k0 + P.kc[d]) + PBK - 1) / PBK;
            for (int kb = kb0; kb < kb1 && ok; kb++) {
              for (int s = 0; s <= d; s++, u++) {
                const int st = u % PSTAGES;
                if (u >= PSTAGES &&
                    !mbar_wait_cl(smem_u32(&bar_empty[st]), ((u / PSTAGES) - 1) & 1, &abort_flag, P.err, 31)) {
                  ok = false;
                  break;
                }
                const uint32_t fb_local = smem_u32(&bar_full[st]);
                if (rank == 0) mbar_expect_tx(fb_local, 2 * PSTAGE);
                const uint32_t fb = map_rank(fb_local, 0);
                uint8_t* sp = smem + (size_t)st * PSTAGE;
                for (int c = 0; c < 4; c++)
                  tma_load_3d_pair(smem_u32(sp + c * PA_PLANE), &tmA, kb * PBK, ma, s * 4 + c, fb);
                for (int c = 0; c < 4; c++)
                  tma_load_3d_pair(smem_u32(sp + 4 * PA_PLANE + c * PB_PLANE), &tmB, kb * PBK, nb, (d - s) * 4 + c,
                                   fb);
                issued = u + 1;
              }
            }
          }
        }
      }
      // the MMA's last commits arrive on this CTA's empty barriers too: wait
      // (bounded) for them before the CTA can leave
      for (int v = (issued > PSTAGES ? issued - PSTAGES : 0); v < issued && ok; v++)
        ok = mbar_wait_cl(smem_u32(&bar_empty[v % PSTAGES]), (v / PSTAGES) & 1, &abort_flag, P.err, 35);
    }
  } else if (warp < PEPI0) {
    // ---------------- MMA issuers (first CTA only): warp 1 components 0, 1; warp 2 components 2, 3 ----------------
    if (lane == 0 && rank == 0) {
      const bool lo = warp == 1;
      int u = 0, w = 0;
      bool ok = true;
      for (int item = pair; item < P.items && ok; item += npairs) {
        const int g = item % P.ngroups;
        for (int li = 0; li < P.nlv[g] && ok; li++) {
          const int d = P.lv[g][li];
          for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d], w++) {
            const int b = w & 1;
            if (w >= 2 &&
                !mbar_wait_cl(smem_u32(&bar_acc_empty[b]), ((w >> 1) - 1) & 1, &abort_flag, P.err, 32)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t dacc = tmem + b * PCHUNK_COLS;
            const int kb0 = k0 / PBK, kb1 = (min(P.K, k0 + P.kc[d]) + PBK - 1) / PBK;
            bool first = true;
            for (int kb = kb0; kb < kb1 && ok; kb++) {
              for (int s = 0; s <= d; s++, u++) {
                const int st = u % PSTAGES;
                if (!mbar_wait_cl(smem_u32(&bar_full[st]), (u / PSTAGES) & 1, &abort_flag, P.err, 33)) {
                  ok = false;
                  break;
                }
                fence_after();
                uint8_t* sp = smem + (size_t)st * PSTAGE;
                const uint64_t ad0 = smem_desc_sw<PSWB>(smem_u32(sp)),
                               bd0 = smem_desc_sw<PSWB>(smem_u32(sp + 4 * PA_PLANE));
#pragma unroll
                for (int kk = 0; kk < PBK / 16; kk++) {
                  if (lo)
                    qmma_k16_pair<0>(dacc, ad0 + kk * 2, bd0 + kk * 2, first && kk == 0);
                  else
                    qmma_k16_pair<2>(dacc, ad0 + kk * 2, bd0 + kk * 2, first && kk == 0);
                }
                first = false;
                mma_commit_pair(smem_u32(&bar_empty[st]));
              }
            }
            if (ok) mma_commit_pair(smem_u32(&bar_acc_full[b]));
          }
        }
      }
    }
  } else {
    // ---------------- epilogue (both CTAs): FP32 chunk -> int32 sums -> int64 per level ----------------
    const int e = warp - PEPI0, quarter = warp & 3, half = e >> 2;
    const uint32_t tb0 = tmem + ((uint32_t)(quarter * 32) << 16) + half * 128;
    int w = 0;
    bool ok = true;
    int acc[128];
    for (int item = pair; item < P.items && ok; item += npairs) {
      const int g = item % P.ngroups;
      int m0, n0;
      pair_tile_origin(P, item / P.ngroups, m0, n0);
      const int row = m0 + (int)rank * PBM + quarter * 32 + lane;
      long long* const C64 = P.C64g[g];
      for (int li = 0; li < P.nlv[g] && ok; li++) {
        const int d = P.lv[g][li];
        const float scale = ldexpf(1.0f, 7 * (d + 2));  // level unit -> integer (a power of two: exact)
        const int sh = P.shift - 7 * (d + 2);
        for (int k0 = 0; k0 < P.K && ok; k0 += P.kc[d], w++) {
          const int b = w & 1;
          const uint32_t tb = tb0 + b * PCHUNK_COLS;
          int have = 1;
          if (lane == 0)
            have = mbar_wait_cl(smem_u32(&bar_acc_full[b]), (w >> 1) & 1, &abort_flag, P.err, 34) ? 1 : 0;
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
          // the chunk is in registers: release the buffer to the pair's MMA issuer
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_remote(map_rank(smem_u32(&bar_acc_empty[b]), 0));
          const bool last = k0 + P.kc[d] >= P.K;
          if (!last || row >= P.M) continue;
#pragma unroll
          for (int p = 0; p < 4; p++) {
            const int c = 2 * half + (p >> 1), j0 = n0 + (p & 1) * 32;
            long long* dst = C64 + c * P.ps64 + (long)row * P.ld64 + j0;
#pragma unroll
            for (int t = 0; t < 32; t += 2) {
              if (j0 + t >= P.N) break;
              const long long x0 = (long long)acc[p * 32 + t], x1 = (long long)acc[p * 32 + t + 1];
              const long long y0 = sh >= 0 ? (x0 << sh) : ((x0 + (1LL << (-sh - 1))) >> (-sh));
              const long long y1 = sh >= 0 ? (x1 << sh) : ((x1 + (1LL << (-sh - 1))) >> (-sh));
              add64_pair2(dst + t, y0, y1, j0 + t + 1 < P.N, li == 0);
            }
          }
        }
      }
    }
  }

  fence_before();
  __syncthreads();
  // after an abort, the first CTA waits (bounded) for the stages still in
  // flight: its full barriers count the copies of both CTAs
  if (warp == 0 && lane == 0 && rank == 0 && abort_flag) {
    for (int u = (issued > PSTAGES ? issued - PSTAGES : 0); u < issued; u++)
      (void)mbar_wait_cl(smem_u32(&bar_full[u % PSTAGES]), (u / PSTAGES) & 1, &abort_flag, nullptr, 0);
  }
  __syncthreads();
  cluster_sync();  // no MMA reads the other CTA's shared memory and no remote arrival is pending
  if (warp == 1) {
    __syncwarp();
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace

cudaError_t launch_qgemm_emu_pair(const EmuGemmArgs& a, cudaStream_t st) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0) return cudaSuccess;
  if (!a.A || !a.B || !a.A->a || !a.B->b || !a.C64 || !emu_fused_ok(a.K, a.S)) return cudaErrorInvalidValue;
  if (a.A->levels < a.S || a.B->levels < a.S) return cudaErrorInvalidValue;
  if ((a.A->lda % 8) || (a.A->psa % 8) || (a.B->ldb % 8) || (a.B->psb % 8)) return cudaErrorInvalidValue;
  PParams P;
  P.M = a.M;
  P.N = a.N;
  P.K = a.K;
  P.S = a.S;
  for (int d = 0; d < 8; d++) {
    const int kc = d < a.S ? a.kc[d] : a.K;
    if (kc < a.K && (kc <= 0 || kc % PBK)) return cudaErrorInvalidValue;
    P.kc[d] = kc < a.K ? kc : a.K;
  }
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
  P.Mt = (a.M + 2 * PBM - 1) / (2 * PBM);
  P.Nt = (a.N + PBN - 1) / PBN;
  CUtensorMap mA, mB;
  if (!make_map(&mA, a.A->a, a.K, a.M, 4 * a.A->levels, a.A->lda, a.A->psa, PBM, PBK)) return cudaErrorInvalidValue;
  if (!make_map(&mB, a.B->b, a.K, a.N, 4 * a.B->levels, a.B->ldb, a.B->psb, PBN_HALF, PBK))
    return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_done{0};
  if (cudaError_t e = ensure_smem_attr(k_qgemm_emu_pair, PSMEM, attr_done)) return e;
  P.items = P.Mt * P.Nt * P.ngroups;
  static int nsm[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidValue;
  if (!nsm[dev] && cudaDeviceGetAttribute(&nsm[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaErrorInvalidValue;
  // persistent: as many pairs as can be resident at once (clusters stay
  // within a GPC, so this may be below half the SM count)
  static int nclusters[64] = {0};
  if (!nclusters[dev]) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nsm[dev], 1, 1);
    cfg.blockDim = dim3(PTHREADS, 1, 1);
    cfg.dynamicSmemBytes = PSMEM;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_qgemm_emu_pair, &cfg) != cudaSuccess || n < 1) n = nsm[dev] / 2;
    nclusters[dev] = std::min(n, nsm[dev] / 2);
  }
  const int pairs = std::min(P.items, nclusters[dev]);
  k_qgemm_emu_pair<<<2 * pairs, PTHREADS, PSMEM, st>>>(mA, mB, P);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace qp
