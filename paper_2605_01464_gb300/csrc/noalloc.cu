// noalloc.cu -- an allocation-free variant of the tensor-core quaternion GEMM.
//
// Some callers cannot allocate device memory at the point where they need a
// product: code running inside a memory pool or arena that forbids further
// cudaMalloc calls, real-time or embedded-style loops that must not touch the
// allocator after start-up, and callers that hold no library context (a
// context allocates its workspace on first use).  qpinv_qgemm_noalloc serves
// them: it computes the same product as qpinv_qgemm with QPINV_PREC_TC, but
// its scratch -- the BF16 operand splits, the FP32 accumulator and the
// kernel's error word -- lives in one file-scope __device__ array of fixed,
// modest size (about 4 MiB, held by every GPU that loads the library until
// the process exits).  Nothing here calls cudaMalloc, cudaFree or an
// allocating library routine.
//
// Set-up: the host cannot use the array's name as a device address (in host
// code it is only a stand-in).  The first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it.
//
// Each call is synchronous: it reads the kernel's error word back into host
// memory and waits for its stream before it returns.
//
// Sharing: every call uses the same array and leaves its contents behind.
// The error word is cleared at the start of each call; everything else that
// is read is written first in the same call.  Calls whose work overlaps on
// the GPU (different streams, or host threads without ordering) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "../../include/qpinv.h"
#include "common.cuh"

namespace qp {
namespace {

constexpr int NA_MAX = QPINV_NOALLOC_MAX_DIM;  // m, k, n <= NA_MAX
constexpr int NA_LEVELS = 3;
constexpr size_t NA_SPLIT_BYTES = (size_t)NA_LEVELS * 4 * NA_MAX * NA_MAX * sizeof(bf16);
constexpr size_t NA_ACC_BYTES = (size_t)4 * NA_MAX * NA_MAX * sizeof(float);
constexpr size_t NA_OFF_A = 0;
constexpr size_t NA_OFF_B = NA_OFF_A + NA_SPLIT_BYTES;
constexpr size_t NA_OFF_C = NA_OFF_B + NA_SPLIT_BYTES;
constexpr size_t NA_OFF_ERR = NA_OFF_C + NA_ACC_BYTES;
constexpr size_t NA_TOTAL = NA_OFF_ERR + 256;

static_assert(NA_OFF_B % 1024 == 0 && NA_OFF_C % 1024 == 0 && NA_OFF_ERR % 1024 == 0, "aligned sections");

// The scratch array shared by every call of qpinv_qgemm_noalloc.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_TOTAL];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

struct Ptr4 {
  const double* p[4];
};
struct OutPtr4 {
  double* p[4];
};

__device__ __forceinline__ void split3(bf16* base, long idx, long lstride, int levels, float v) {
  float r = v;
  for (int l = 0; l < levels; l++) {
    const bf16 t = __float2bfloat16_rn(r);
    base[l * lstride + idx] = t;
    r -= __bfloat162float(t);
  }
}

// A (rows x cols, four separate planes) -> A-form splits [level][comp][rows][ld16].
__global__ void k_na_split_a(Ptr4 A, long lda, int rows, int cols, int levels, bf16* dst, long ld16) {
  const long total = (long)rows * cols;
  const long ps = (long)rows * ld16;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long i = t / cols, j = t % cols;
    for (int c = 0; c < 4; c++) split3(dst, c * ps + i * ld16 + j, 4 * ps, levels, (float)A.p[c][i * lda + j]);
  }
}

// B (rows = K x cols = N, four planes) -> B-form splits [level][comp][cols][ld16] (transposed).
__global__ void k_na_split_b(Ptr4 B, long ldb, int rows, int cols, int levels, bf16* dst, long ld16) {
  const long total = (long)rows * cols;
  const long ps = (long)cols * ld16;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long j = t / rows, i = t % rows;  // consecutive threads walk K: coalesced writes
    for (int c = 0; c < 4; c++) split3(dst, c * ps + j * ld16 + i, 4 * ps, levels, (float)B.p[c][i * ldb + j]);
  }
}

__global__ void k_na_store(const float* acc, long ldacc, long psacc, int rows, int cols, OutPtr4 C, long ldc) {
  const long total = (long)rows * cols;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long i = t / cols, j = t % cols;
    for (int c = 0; c < 4; c++) C.p[c][i * ldc + j] = (double)acc[c * psacc + i * ldacc + j];
  }
}

int blocks_for(long total) {
  long b = (total + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

// True if every pointer is device (or managed) memory of device `dev`: the
// kernels run on the current device, and memory of another GPU would be read
// through a peer mapping that may not exist.
bool all_device(const void* const* p, int n, int dev) {
  for (int t = 0; t < n; t++) {
    cudaPointerAttributes at;
    if (!p[t] || cudaPointerGetAttributes(&at, p[t]) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
    if (at.device != dev) return false;
  }
  return true;
}

}  // namespace
}  // namespace qp

using namespace qp;

extern "C" int qpinv_qgemm_noalloc(void* stream, int m, int k, int n, const double* const A[4], long lda,
                                   const double* const B[4], long ldb, double* const C[4], long ldc,
                                   int split_level) {
  if (m <= 0 || n <= 0 || k <= 0 || lda < k || ldb < n || ldc < n || split_level < 1 || split_level > NA_LEVELS ||
      !A || !B || !C)
    return QPINV_E_INVALID;
  if (m > NA_MAX || n > NA_MAX || k > NA_MAX) return QPINV_E_NOALLOC_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return QPINV_E_CUDA;
  if (!all_device((const void* const*)A, 4, dev) || !all_device((const void* const*)B, 4, dev) ||
      !all_device((const void* const*)C, 4, dev))
    return QPINV_E_INVALID;
  if (!tc_supported()) return QPINV_E_UNSUPPORTED;
  unsigned char* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return QPINV_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  const long ldk = (k + 7) / 8 * 8, ldn = (n + 7) / 8 * 8;
  Split16 sa, sb;
  sa.levels = sb.levels = split_level;
  sa.a = reinterpret_cast<bf16*>(base + NA_OFF_A);
  sa.lda = ldk;
  sa.psa = (long)m * ldk;
  sb.b = reinterpret_cast<bf16*>(base + NA_OFF_B);
  sb.ldb = ldk;
  sb.psb = (long)n * ldk;
  Planes<float> acc;
  acc.p = reinterpret_cast<float*>(base + NA_OFF_C);
  acc.ld = ldn;
  acc.ps = (long)m * ldn;
  int* err = reinterpret_cast<int*>(base + NA_OFF_ERR);

  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return QPINV_E_CUDA;
  Ptr4 pa, pb;
  OutPtr4 pc;
  for (int c = 0; c < 4; c++) {
    pa.p[c] = A[c];
    pb.p[c] = B[c];
    pc.p[c] = C[c];
  }
  k_na_split_a<<<blocks_for((long)m * k), 256, 0, st>>>(pa, lda, m, k, split_level, sa.a, ldk);
  k_na_split_b<<<blocks_for((long)k * n), 256, 0, st>>>(pb, ldb, k, n, split_level, sb.b, ldk);
  if (cudaGetLastError() != cudaSuccess) return QPINV_E_CUDA;

  TcGemmArgs g;
  g.M = m;
  g.N = n;
  g.K = k;
  g.k0 = 0;
  g.k1 = k;
  g.A = &sa;
  g.B = &sb;
  static const int pi3[6] = {2, 1, 0, 1, 0, 0}, pj3[6] = {0, 1, 2, 0, 1, 0};
  static const int pi2[3] = {1, 0, 0}, pj2[3] = {0, 1, 0};
  g.npairs = split_level == 3 ? 6 : (split_level == 2 ? 3 : 1);
  for (int t = 0; t < g.npairs; t++) {
    g.pair_i[t] = split_level == 3 ? pi3[t] : (split_level == 2 ? pi2[t] : 0);
    g.pair_j[t] = split_level == 3 ? pj3[t] : (split_level == 2 ? pj2[t] : 0);
  }
  g.C = acc;
  g.err = err;
  if (launch_qgemm_tc(g, st) != cudaSuccess) return QPINV_E_CUDA;
  k_na_store<<<blocks_for((long)m * n), 256, 0, st>>>(acc.p, acc.ld, acc.ps, m, n, pc, ldc);
  if (cudaGetLastError() != cudaSuccess) return QPINV_E_CUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return QPINV_E_CUDA;
  return h_err ? QPINV_E_TIMEOUT : QPINV_OK;
}
