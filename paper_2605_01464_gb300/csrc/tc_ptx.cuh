// tc_ptx.cuh -- inline-PTX building blocks of the sm_103a tensor-core kernels:
// mbarriers with bounded waits, TMA tile loads, tcgen05 MMA / commit / TMEM
// loads and stores, shared-memory matrix descriptors, and the host-side TMA
// tensor-map encoder (driver entry point, no libcuda link).
#pragma once
#include <cuda.h>

#include <atomic>

#include "common.cuh"

namespace qp {
namespace {

constexpr unsigned long long WAIT_NS = 2000000000ull;  // bound of every spin wait (2 s of globaltimer)

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
// Shared-memory matrix descriptor: K-major, rows of `swb` swizzled bytes
// (64 or 128), 8-row groups 8 * swb bytes apart.
template <int SWB>
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr) {
  constexpr unsigned long long layout = SWB == 128 ? 2ull : 4ull;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * SWB) >> 4) << 32) |
         ((uint64_t)1 << 46) | (layout << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Sign pattern of the real form of the Hamilton product: block (r, c) of
// M(B) is -B_{r xor c} for these (r, c), +B_{r xor c} otherwise.
__host__ __device__ constexpr bool qsign_neg(int r, int c) {
  return (r == 1 && (c == 0 || c == 2)) || (r == 2 && (c == 0 || c == 3)) || (r == 3 && (c == 0 || c == 1));
}
// The 8 of those MMAs that feed components C0 and C0 + 1 (two issuing
// threads then share a K step).
template <uint32_t A_PLANE, uint32_t B_PLANE, int C0>
__device__ __forceinline__ void qmma_k16_half(uint32_t d_tmem, uint32_t ncols, uint64_t ad0, uint64_t bd0,
                                              uint32_t idesc, bool fresh) {
  constexpr uint32_t NEG_A = 1u << 13;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const uint64_t ad = ad0 + ((r * A_PLANE) >> 4);
    const uint32_t acc = (fresh && r == 0) ? 0u : 1u;
#pragma unroll
    for (int c = C0; c < C0 + 2; c++)
      mma_bf16(d_tmem + c * ncols, ad, bd0 + (((r ^ c) * B_PLANE) >> 4), qsign_neg(r, c) ? idesc | NEG_A : idesc,
               acc);
  }
}
// The 16 signed (r, c) MMAs of one K = 16 step: A plane r times B plane
// r xor c into component c's accumulator (d_tmem + c * ncols), the sign from
// the instruction descriptor's negate-A bit (bit 13).  ad0 / bd0 are the
// descriptors of the step's first A and B planes; a plane's descriptor is
// ad0 plus its byte offset / 16 (the address field is the low 14 bits and
// every operand lies below 256 KB, so the add never carries out of it).
// The issuing thread feeds the tensor core one MMA per few dozen cycles, so
// the loop is kept to one add per descriptor.
template <uint32_t A_PLANE, uint32_t B_PLANE>
__device__ __forceinline__ void qmma_k16(uint32_t d_tmem, uint32_t ncols, uint64_t ad0, uint64_t bd0, uint32_t idesc,
                                         bool fresh) {
  constexpr uint32_t NEG_A = 1u << 13;
#pragma unroll
  for (int r = 0; r < 4; r++) {
    const uint64_t ad = ad0 + ((r * A_PLANE) >> 4);
    const uint32_t acc = (fresh && r == 0) ? 0u : 1u;
#pragma unroll
    for (int c = 0; c < 4; c++)
      mma_bf16(d_tmem + c * ncols, ad, bd0 + (((r ^ c) * B_PLANE) >> 4), qsign_neg(r, c) ? idesc | NEG_A : idesc,
               acc);
  }
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

__device__ __forceinline__ void tmem_ld32u(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32u(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
      "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
// 32 lanes x 16 consecutive columns (one row of 16 values per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 16; t++) v[t] = __uint_as_float(r[t]);
}
__device__ __forceinline__ void tmem_ld16u(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// Epilogue row writers: lane j handles column j of up to 32 consecutive rows
// (stride ld) of a transposed 32 x 33 shared-memory block `st` (already offset
// by the lane).  All loads are issued before any store so that the 32 row
// accesses of a lane are in flight together.
__device__ __forceinline__ void rmw_rows64(long long* __restrict__ dst, long ld, int nrow,
                                           const long long* __restrict__ st) {
#pragma unroll 1
  for (int h = 0; h < 32; h += 16) {  // 16 rows in flight: bounded register use
    long long g[16];
#pragma unroll
    for (int r = 0; r < 16; r++)
      if (h + r < nrow) g[r] = dst[(long)(h + r) * ld];
#pragma unroll
    for (int r = 0; r < 16; r++)
      if (h + r < nrow) dst[(long)(h + r) * ld] = g[r] + st[(h + r) * 33];
  }
}
__device__ __forceinline__ void store_rows32(float* __restrict__ dst, long ld, int nrow,
                                             const float* __restrict__ st) {
  float g[32];
#pragma unroll
  for (int r = 0; r < 32; r++) g[r] = st[r * 33];
#pragma unroll
  for (int r = 0; r < 32; r++)
    if (r < nrow) dst[(long)r * ld] = g[r];
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per device (bit d of `done`; a repeated call from a racing
// thread is harmless).  The attribute is per device: a flag shared by all
// devices would skip the call on the second one.
template <typename Kern>
cudaError_t ensure_smem_attr(Kern kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
  return e;
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

}  // namespace
}  // namespace qp
