// elementwise.cu -- HBM-bound kernels of the solve: the fused combine pass
// that follows every quaternion product (residual R = I - AX, polynomial
// blocks, X update with the stop-test norms), BF16 operand splitting and
// exact slicing with transposed copies, initialisation X_0 = alpha A^H, and
// the norm and Penrose-residual reductions.
//
// GB300's FP64 pipe is a small fraction of its FP32 rate, so the
// tensor-core phase runs these passes on FP32 masters; only the FP64 phase
// (polish, Penrose) uses double arithmetic, and exact slicing and exponent
// extraction use integer operations on the bit patterns.  Reductions are
// deterministic: each block writes partial sums and one block adds them in a
// fixed order.
#include <algorithm>

#include "common.cuh"

namespace qp {

thread_local long long g_kernel_launches = 0;

namespace {

constexpr int TILE = 32;
constexpr int TROWS = 8;  // block = 32 x 8 threads, each thread 4 rows of the tile

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
  return r;  // valid in thread 0 only
}

// Inf / NaN from the exponent bits (integer instructions: GB300's FP64 pipe
// is the scarce resource in these passes).
__device__ __forceinline__ int nonfinite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) == 0x7FF ? 1 : 0;
}
__device__ __forceinline__ int nonfinite_bits(float x) { return ((__float_as_int(x) >> 23) & 0xFF) == 0xFF ? 1 : 0; }

// Round-to-nearest BF16 split of the FP32 value: 3 terms cover all 24 bits.
__device__ __forceinline__ void split_store(bf16* base, long idx, long lstride, int levels, float v) {
  float r = v;
  for (int l = 0; l < levels; l++) {
    const bf16 t = __float2bfloat16_rn(r);
    base[l * lstride + idx] = t;
    r -= __bfloat162float(t);
  }
}

// round(v * 2^sh) as an integer, from the bits of v (integer arithmetic only).
// Requires |v * 2^sh| < 2^62; subnormal inputs count as zero.
__device__ __forceinline__ long long to_fixed(double v, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int k = ex - 1075 + sh;  // v * 2^sh = mant * 2^k
  long long F;
  if (k >= 0) F = mant << k;
  else if (k <= -55) F = 0;
  else F = (mant + (1ll << (-k - 1))) >> (-k);
  return (b >> 63) ? -F : F;
}
__device__ __forceinline__ long long to_fixed(float v, int sh) {
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

// Binary exponent e with |v| < 2^e (0 for zero / subnormal), from the bits.
__device__ __forceinline__ int exp_of(double v) {
  const int ex = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FF);
  return ex == 0 ? -100000 : ex - 1022;
}
__device__ __forceinline__ int exp_of(float v) {
  const int ex = (int)((__float_as_uint(v) >> 23) & 0xFF);
  return ex == 0 ? -100000 : ex - 126;
}

// Exact slices of v * 2^-e (|v| < 2^e): F = round(v * 2^(7S - e)) written in
// balanced base 128, least significant digit first; slice s = digit_s * 2^-(7(s+1)).
template <typename T>
__device__ __forceinline__ void slice_store(bf16* base, long idx, long lstride, int S, T v, int e) {
  long long F = to_fixed(v, 7 * S - e);
  for (int l = S - 1; l >= 1; l--) {
    int d = (int)(F & 127);
    if (d >= 64) d -= 128;
    F = (F - d) >> 7;
    base[l * lstride + idx] = __float2bfloat16_rn(ldexpf((float)d, -7 * (l + 1)));
  }
  base[idx] = __float2bfloat16_rn(ldexpf((float)F, -7));
}

// q 2^e as a double, rounded to nearest (ties to even) from the integer bits:
// the same value as ldexp((double)q, e), without FP64 arithmetic (GB300's
// FP64 rate is a small fraction of its integer rate).  Results below the
// normal range or above the finite range take ldexp.
__device__ __forceinline__ double i64_scaled(long long q, int e) {
  if (q == 0) return 0.0;
  const unsigned long long sgn = q < 0 ? (1ull << 63) : 0ull;
  unsigned long long mag = q < 0 ? 0ull - (unsigned long long)q : (unsigned long long)q;
  const int lz = __clzll((long long)mag);
  mag <<= lz;  // leading one at bit 63
  unsigned long long m = mag >> 11;  // 53 significant bits
  const unsigned long long rem = mag & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) m++;
  int ex = 63 - lz + e;  // value = m 2^(ex - 52)
  if (m >> 53) {
    m >>= 1;
    ex++;
  }
  const int biased = ex + 1023;
  if (biased <= 0 || biased >= 2047) return ldexp((double)q, e);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)biased << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

template <typename T>
__device__ __forceinline__ T acc_value(const CombineArgs& a, int c, int i, int j) {
  const long off = c * a.ps_acc + (long)i * a.ld_acc + j;
  if (a.acc_kind == ACC_F64) return (T)((const double*)a.acc)[off];
  if (a.acc_kind == ACC_I64) {
    const long long q = ((const long long*)a.acc)[off] + (a.acc2 ? a.acc2[off] : 0LL);
    const int e = a.acc_erow[i] + a.acc_ecol[j] - a.acc_shift;
    if (sizeof(T) == 4) return (T)ldexpf((float)q, e);
    return (T)i64_scaled(q, e);
  }
  return (T)((const float*)a.acc)[off];
}

// cacc x for cacc = +-1 without arithmetic (a sign flip), else the product.
template <typename T>
__device__ __forceinline__ T times_coef(T x, T cacc) {
  if (cacc == (T)1) return x;
  if (cacc == (T)-1) return -x;
  return cacc * x;
}

// One 32x32 tile per block; threads (tx, ty), tid = ty * 32 + tx.
template <typename T>
__global__ void __launch_bounds__(256) k_combine(CombineArgs a) {
  __shared__ T stage[4][TILE][TILE + 1];
  __shared__ double red[8];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;
  T s_dx = 0, s_x = 0;
  int s_bad = 0;

  for (int o = 0; o < a.nout; o++) {
    const OutSpec& O = a.out[o];
    const T cacc = (T)O.cacc, diag = (T)O.diag;
    for (int q = 0; q < TILE / TROWS; q++) {
      const int i = r0 + ty + q * TROWS, j = c0 + tx;
      T v[4] = {0, 0, 0, 0};
      if (i < a.rows && j < a.cols) {
        if (a.acc && O.cacc != 0.0)
          for (int c = 0; c < 4; c++) v[c] = times_coef<T>(acc_value<T>(a, c, i, j), cacc);
        for (int t = 0; t < 4; t++) {
          if (!a.aux[t] || O.caux[t] == 0.0) continue;
          const T* ap = (const T*)a.aux[t];
          const T ct = (T)O.caux[t];
          for (int c = 0; c < 4; c++) v[c] += ct * ap[c * a.ps_aux[t] + (long)i * a.ld_aux[t] + j];
        }
        if (i == j) v[0] += diag;
        if (o == 0 && a.partials) {
          const T* x0p = (const T*)a.aux[0];
          for (int c = 0; c < 4; c++) {
            s_x += v[c] * v[c];
            if (x0p) {
              const T dx = v[c] - x0p[c * a.ps_aux[0] + (long)i * a.ld_aux[0] + j];
              s_dx += dx * dx;
            }
            s_bad += nonfinite_bits(v[c]);
          }
        }
        if (O.mp)
          for (int c = 0; c < 4; c++) ((T*)O.mp)[c * O.mps + (long)i * O.mld + j] = v[c];
        if (O.s16.a) {
          for (int c = 0; c < 4; c++) {
            const long idx = c * O.s16.psa + (long)i * O.s16.lda + j;
            if (O.exp_a) slice_store<T>(O.s16.a, idx, 4 * O.s16.psa, O.s16.levels, v[c], O.exp_a[i]);
            else split_store(O.s16.a, idx, 4 * O.s16.psa, O.s16.levels, (float)v[c]);
          }
        }
      }
      if (O.s16.b)
        for (int c = 0; c < 4; c++) stage[c][ty + q * TROWS][tx] = v[c];
    }
    if (O.s16.b) {
      __syncthreads();
      for (int q = 0; q < TILE / TROWS; q++) {
        const int jj = c0 + ty + q * TROWS, ii = r0 + tx;  // B-form element (jj, ii) = out(ii, jj)
        if (ii < a.rows && jj < a.cols) {
          for (int c = 0; c < 4; c++) {
            const long idx = c * O.s16.psb + (long)jj * O.s16.ldb + ii;
            const T val = stage[c][tx][ty + q * TROWS];
            if (O.exp_b) slice_store<T>(O.s16.b, idx, 4 * O.s16.psb, O.s16.levels, val, O.exp_b[jj]);
            else split_store(O.s16.b, idx, 4 * O.s16.psb, O.s16.levels, (float)val);
          }
        }
      }
      __syncthreads();
    }
  }
  if (a.partials) {
    if (!a.aux[0]) s_dx = s_x;  // ||v - 0||^2
    const long b = (long)blockIdx.y * gridDim.x + blockIdx.x;
    const double t0 = block_sum((double)s_dx, red);
    const double t1 = block_sum((double)s_x, red);
    const double t2 = block_sum((double)s_bad, red);
    if (threadIdx.x == 0) {
      a.partials[3 * b + 0] = t0;
      a.partials[3 * b + 1] = t1;
      a.partials[3 * b + 2] = t2;
    }
  }
}

// FP32 passes over column pairs: 32 rows x 64 columns per block, each thread
// two adjacent columns (8-byte loads and stores, packed BF16 pairs), which
// halves the index arithmetic and store instructions per element.  Needs even
// leading dimensions and plane strides for every FP32 / FP64 / int64 plane it
// touches (combine_pairs_ok); the BF16 forms have ld, ps multiples of 8.
__device__ __forceinline__ void split_store2(bf16* base, long idx, long lstride, int levels, float x, float y) {
  float rx = x, ry = y;
  for (int l = 0; l < levels; l++) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(rx, ry);
    *reinterpret_cast<__nv_bfloat162*>(base + l * lstride + idx) = t;
    rx -= __low2float(t);
    ry -= __high2float(t);
  }
}

__device__ __forceinline__ void acc_pair(const CombineArgs& a, int c, int i, int j, bool two, float& x, float& y) {
  const long off = c * a.ps_acc + (long)i * a.ld_acc + j;
  if (a.acc_kind == ACC_F32) {
    if (two) {
      const float2 t = *reinterpret_cast<const float2*>((const float*)a.acc + off);
      x = t.x;
      y = t.y;
    } else {
      x = ((const float*)a.acc)[off];
    }
  } else if (a.acc_kind == ACC_F64) {
    const double* p = (const double*)a.acc + off;
    x = (float)p[0];
    if (two) y = (float)p[1];
  } else {
    const long long* p = (const long long*)a.acc + off;
    long long q0 = p[0], q1 = two ? p[1] : 0;
    if (a.acc2) {
      q0 += a.acc2[off];
      if (two) q1 += a.acc2[off + 1];
    }
    const int er = a.acc_erow[i] - a.acc_shift;
    x = ldexpf((float)q0, er + a.acc_ecol[j]);
    if (two) y = ldexpf((float)q1, er + a.acc_ecol[j + 1]);
  }
}

__global__ void __launch_bounds__(256) k_combine_f2(CombineArgs a) {
  __shared__ float stage[4][2 * TILE][TILE + 1];  // [plane][column][row]
  __shared__ double red[8];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * 2 * TILE;
  const int j = c0 + 2 * tx;
  float s_dx = 0.f, s_x = 0.f;
  int s_bad = 0;

  for (int o = 0; o < a.nout; o++) {
    const OutSpec& O = a.out[o];
    const float cacc = (float)O.cacc, diag = (float)O.diag;
    for (int q = 0; q < TILE / TROWS; q++) {
      const int i = r0 + ty + q * TROWS;
      float v[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      const bool in0 = i < a.rows && j < a.cols, two = in0 && j + 1 < a.cols;
      if (in0) {
        if (a.acc && O.cacc != 0.0)
          for (int c = 0; c < 4; c++) {
            float x = 0.f, y = 0.f;
            acc_pair(a, c, i, j, two, x, y);
            v[c][0] = cacc * x;
            v[c][1] = cacc * y;
          }
        for (int t = 0; t < 4; t++) {
          if (!a.aux[t] || O.caux[t] == 0.0) continue;
          const float* ap = (const float*)a.aux[t];
          const float ct = (float)O.caux[t];
          for (int c = 0; c < 4; c++) {
            const long off = c * a.ps_aux[t] + (long)i * a.ld_aux[t] + j;
            if (two) {
              const float2 u = *reinterpret_cast<const float2*>(ap + off);
              v[c][0] += ct * u.x;
              v[c][1] += ct * u.y;
            } else {
              v[c][0] += ct * ap[off];
            }
          }
        }
        if (i == j) v[0][0] += diag;
        if (two && i == j + 1) v[0][1] += diag;
        if (o == 0 && a.partials) {
          const float* x0p = (const float*)a.aux[0];
          for (int c = 0; c < 4; c++)
            for (int h = 0; h < (two ? 2 : 1); h++) {
              const float x0 = x0p ? x0p[c * a.ps_aux[0] + (long)i * a.ld_aux[0] + j + h] : 0.f;
              s_dx += (v[c][h] - x0) * (v[c][h] - x0);
              s_x += v[c][h] * v[c][h];
              s_bad += isfinite(v[c][h]) ? 0 : 1;
            }
        }
        if (O.mp)
          for (int c = 0; c < 4; c++) {
            float* dst = (float*)O.mp + c * O.mps + (long)i * O.mld + j;
            if (two) *reinterpret_cast<float2*>(dst) = make_float2(v[c][0], v[c][1]);
            else dst[0] = v[c][0];
          }
        if (O.s16.a)
          for (int c = 0; c < 4; c++) {
            const long idx = c * O.s16.psa + (long)i * O.s16.lda + j;
            if (O.exp_a) {
              slice_store<float>(O.s16.a, idx, 4 * O.s16.psa, O.s16.levels, v[c][0], O.exp_a[i]);
              if (two) slice_store<float>(O.s16.a, idx + 1, 4 * O.s16.psa, O.s16.levels, v[c][1], O.exp_a[i]);
            } else if (two) {
              split_store2(O.s16.a, idx, 4 * O.s16.psa, O.s16.levels, v[c][0], v[c][1]);
            } else {
              split_store(O.s16.a, idx, 4 * O.s16.psa, O.s16.levels, v[c][0]);
            }
          }
      }
      if (O.s16.b)
        for (int c = 0; c < 4; c++) {
          stage[c][2 * tx][ty + q * TROWS] = v[c][0];
          stage[c][2 * tx + 1][ty + q * TROWS] = v[c][1];
        }
    }
    if (O.s16.b) {
      __syncthreads();
      // B-form row jj (an output column) holds the block's 32 rows ii: thread
      // t writes the pair ii = 2 (t % 16), +1 of columns t / 16 + 16 k.
      const int p = threadIdx.x & 15;
      for (int k = 0; k < 4; k++) {
        const int jl = (threadIdx.x >> 4) + 16 * k, jj = c0 + jl, ii = r0 + 2 * p;
        if (jj < a.cols && ii < a.rows) {
          const bool pair = ii + 1 < a.rows;
          for (int c = 0; c < 4; c++) {
            const long idx = c * O.s16.psb + (long)jj * O.s16.ldb + ii;
            const float x = stage[c][jl][2 * p], y = stage[c][jl][2 * p + 1];
            if (O.exp_b) {
              slice_store<float>(O.s16.b, idx, 4 * O.s16.psb, O.s16.levels, x, O.exp_b[jj]);
              if (pair) slice_store<float>(O.s16.b, idx + 1, 4 * O.s16.psb, O.s16.levels, y, O.exp_b[jj]);
            } else if (pair) {
              split_store2(O.s16.b, idx, 4 * O.s16.psb, O.s16.levels, x, y);
            } else {
              split_store(O.s16.b, idx, 4 * O.s16.psb, O.s16.levels, x);
            }
          }
        }
      }
      __syncthreads();
    }
  }
  if (a.partials) {
    const long b = (long)blockIdx.y * gridDim.x + blockIdx.x;
    const double t0 = block_sum((double)s_dx, red);
    const double t1 = block_sum((double)s_x, red);
    const double t2 = block_sum((double)s_bad, red);
    if (threadIdx.x == 0) {
      a.partials[3 * b + 0] = t0;
      a.partials[3 * b + 1] = t1;
      a.partials[3 * b + 2] = t2;
    }
  }
}

// The pair kernel applies to FP32 passes whose FP32 / FP64 / int64 planes all
// have even leading dimensions, plane strides and 16-byte aligned bases.
static bool combine_pairs_ok(const CombineArgs& a) {
  if (a.f64) return false;
  auto even = [](long x) { return (x & 1) == 0; };
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (a.acc && (!even(a.ld_acc) || !even(a.ps_acc) || !al(a.acc) || (a.acc2 && !al(a.acc2)))) return false;
  for (int t = 0; t < 4; t++)
    if (a.aux[t] && (!even(a.ld_aux[t]) || !even(a.ps_aux[t]) || !al(a.aux[t]))) return false;
  for (int o = 0; o < a.nout; o++) {
    const OutSpec& O = a.out[o];
    if (O.mp && (!even(O.mld) || !even(O.mps) || !al(O.mp))) return false;
    if (O.s16.a && (!al(O.s16.a) || (O.s16.lda & 1) || (O.s16.psa & 1))) return false;
    if (O.s16.b && (!al(O.s16.b) || (O.s16.ldb & 1) || (O.s16.psb & 1))) return false;
  }
  return true;
}

// ---------------------------------------------------------------- exact slicing
// S exact slices (slice_store's digits) of 8 consecutive entries that share
// one exponent, written as one 16-byte store per slice plane.
template <typename T>
__device__ __forceinline__ void slice8_store(bf16* base, long lstride, int S, const T* v, int e) {
  long long F[8];
#pragma unroll
  for (int q = 0; q < 8; q++) F[q] = to_fixed(v[q], 7 * S - e);
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

// A-form slices of a row-major plane set (row exponents e[i]): one thread per
// (plane, row, 8 columns), columns past `cols` up to the padded pitch as 0.
template <typename T>
__global__ void __launch_bounds__(256) k_slice_rows(Planes<const T> A, int rows, int cols, const int* __restrict__ e,
                                                    int S, bf16* dst, long ld, long ps) {
  const int g8 = (cols + 7) / 8;
  const long total = 4L * rows * g8;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int g = (int)(t % g8);
    const long ci = t / g8;
    const int i = (int)(ci % rows), c = (int)(ci / rows);
    const T* src = A.p + c * A.ps + (long)i * A.ld + 8 * g;
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = 8 * g + q < cols ? src[q] : (T)0;
    slice8_store<T>(dst + c * ps + (long)i * ld + 8 * g, 4 * ps, S, v, e[i]);
  }
}

// B-form slices (the plane-wise transpose; column exponents e[j]): a block
// takes 32 rows x 64 columns of one plane through shared memory, then each
// thread writes 8 consecutive rows of one column, rows past `rows` up to the
// padded pitch as 0.
template <typename T>
__global__ void __launch_bounds__(256) k_slice_cols(Planes<const T> A, int rows, int cols, const int* __restrict__ e,
                                                    int S, bf16* dst, long ld, long ps) {
  __shared__ T tile[64][33];
  const int c = blockIdx.z, i0 = blockIdx.y * 32, j0 = blockIdx.x * 64;
  {
    const int il = threadIdx.x >> 3, j8 = (threadIdx.x & 7) * 8;  // 32 rows x 8 groups of 8 columns
    const T* src = A.p + c * A.ps + (long)(i0 + il) * A.ld + j0 + j8;
#pragma unroll
    for (int q = 0; q < 8; q++)
      tile[j8 + q][il] = (i0 + il < rows && j0 + j8 + q < cols) ? src[q] : (T)0;
  }
  __syncthreads();
  const int jl = threadIdx.x >> 2, ig = (threadIdx.x & 3) * 8;  // 64 columns x 4 groups of 8 rows
  const int j = j0 + jl;
  if (j < cols && i0 + ig < ((rows + 7) / 8) * 8) {
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; q++) v[q] = tile[jl][ig + q];
    slice8_store<T>(dst + c * ps + (long)j * ld + i0 + ig, 4 * ps, S, v, e[j]);
  }
}

__global__ void k_reduce_partials(const double* p, int nblocks, int nvals, double* out) {
  __shared__ double sh[8];
  for (int v = 0; v < nvals; v++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += p[(long)b * nvals + v];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) out[v] = t;
  }
}

__global__ void k_row_abs_sums(Planes<const double> A, int m, int n, double* rowsum) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= m) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) {
    double q = 0.0;
    for (int c = 0; c < 4; c++) {
      const double x = A.p[c * A.ps + (long)warp * A.ld + j];
      q += x * x;
    }
    s += sqrt(q);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) rowsum[warp] = s;
}

// Column reductions: blocks of 32 columns x one row chunk (a warp reads 32
// consecutive entries of a row) write one partial per (chunk, column); the
// finishing kernel combines the partials in chunk order, so the result does
// not depend on scheduling.
constexpr int CR_COLS = 32, CR_ROWS = 8, CR_MAX_CHUNKS = 64;

__global__ void k_col_abs_part(Planes<const double> A, int m, int n, int chunk_rows, double* part) {
  __shared__ double sh[CR_ROWS][CR_COLS];
  const int j = blockIdx.x * CR_COLS + threadIdx.x;
  const int r0 = blockIdx.y * chunk_rows, r1 = min(m, r0 + chunk_rows);
  double s = 0.0;
  if (j < n)
    for (int i = r0 + threadIdx.y; i < r1; i += CR_ROWS) {
      double q = 0.0;
      for (int c = 0; c < 4; c++) {
        const double x = A.p[c * A.ps + (long)i * A.ld + j];
        q += x * x;
      }
      s += sqrt(q);
    }
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    for (int t = 1; t < CR_ROWS; t++) s += sh[t][threadIdx.x];
    part[(long)blockIdx.y * n + j] = s;
  }
}

__global__ void k_col_abs_finish(const double* part, int chunks, int n, double* colsum) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int ch = 0; ch < chunks; ch++) s += part[(long)ch * n + j];
  colsum[j] = s;
}

__global__ void k_max(const double* v, int n, double* out) {
  __shared__ double sh[256];
  double mx = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) mx = fmax(mx, v[t]);
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

// partials per block: sum |A - B|^2 (or |A|^2 if B is null), non-finite count of A.
// ||scale A + diag I - B||_F^2 (B optional; diag on plane s) and the
// non-finite count of A.  Work is split into tasks of one row and FRO_COLS
// consecutive columns; a block takes tasks blockIdx.x + k gridDim.x, FRO_U of
// them at a time with all their loads of A issued before the first use.  Per
// element four FP64 FMAs (and the scaling and the subtraction of B where
// asked).
constexpr int FRO_COLS = 256, FRO_U = 2;
__global__ void __launch_bounds__(FRO_COLS) k_fro2(Planes<const double> A, Planes<const double> B, int hasB, int m,
                                                   int n, double scale, double diag, double* partials) {
  __shared__ double sh[8];
  const long chunks = (n + FRO_COLS - 1) / FRO_COLS, tasks = (long)m * chunks;
  double s = 0.0;
  int bad = 0;
  for (long t0 = blockIdx.x; t0 < tasks; t0 += (long)FRO_U * gridDim.x) {
    double x[FRO_U][4];
    long ii[FRO_U];
    int jj[FRO_U];
    bool ok[FRO_U];
#pragma unroll
    for (int u = 0; u < FRO_U; u++) {
      const long t = t0 + (long)u * gridDim.x;
      ii[u] = t / chunks;
      jj[u] = (int)(t - ii[u] * chunks) * FRO_COLS + threadIdx.x;
      ok[u] = t < tasks && jj[u] < n;
#pragma unroll
      for (int c = 0; c < 4; c++) x[u][c] = ok[u] ? A.p[c * A.ps + ii[u] * A.ld + jj[u]] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < FRO_U; u++) {
      if (!ok[u]) continue;
#pragma unroll
      for (int c = 0; c < 4; c++) {
        double v = x[u][c];
        bad += nonfinite_bits(v);
        if (scale != 1.0) v *= scale;
        if (c == 0 && ii[u] == jj[u] && diag != 0.0) v += diag;
        if (hasB) v -= B.p[c * B.ps + ii[u] * B.ld + jj[u]];
        s = fma(v, v, s);
      }
    }
  }
  const double t0 = block_sum(s, sh);
  const double t1 = block_sum((double)bad, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = t0;
    partials[2 * blockIdx.x + 1] = t1;
  }
}

// sum over (i, j) of |conj(M_ji) - M_ij|^2 for square M: ||M^H - M||_F^2.
__global__ void __launch_bounds__(256) k_antiherm(Planes<const double> M, int n, double* partials) {
  __shared__ double t[4][TILE][TILE + 1];
  __shared__ double sh[8];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;
  // load the mirrored tile M[c0.., r0..] transposed into shared memory
  for (int q = 0; q < TILE / TROWS; q++) {
    const int i = c0 + ty + q * TROWS, j = r0 + tx;
    for (int c = 0; c < 4; c++)
      t[c][tx][ty + q * TROWS] = (i < n && j < n) ? M.p[c * M.ps + (long)i * M.ld + j] : 0.0;
  }
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < TILE / TROWS; q++) {
    const int i = r0 + ty + q * TROWS, j = c0 + tx;
    if (i < n && j < n) {
      for (int c = 0; c < 4; c++) {
        const double mij = M.p[c * M.ps + (long)i * M.ld + j];
        const double mji = t[c][ty + q * TROWS][tx];  // M[j][i]
        const double d = (c == 0 ? mji : -mji) - mij;
        s += d * d;
      }
    }
  }
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) partials[(long)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// X (n x m) = alpha * A^H, A m x n: X[j][i] = alpha * conj(A[i][j]).
__global__ void __launch_bounds__(256) k_init_x0(Planes<const double> A, int m, int n, double al,
                                                 Planes<double> X) {
  __shared__ double t[4][TILE][TILE + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int r0 = blockIdx.y * TILE, c0 = blockIdx.x * TILE;  // tile of A: rows r0.., cols c0..
  for (int q = 0; q < TILE / TROWS; q++) {
    const int i = r0 + ty + q * TROWS, j = c0 + tx;
    for (int c = 0; c < 4; c++)
      t[c][ty + q * TROWS][tx] = (i < m && j < n) ? A.p[c * A.ps + (long)i * A.ld + j] : 0.0;
  }
  __syncthreads();
  for (int q = 0; q < TILE / TROWS; q++) {
    const int j = c0 + ty + q * TROWS, i = r0 + tx;  // X element (j, i)
    if (i < m && j < n)
      for (int c = 0; c < 4; c++) {
        const double v = t[c][tx][ty + q * TROWS];
        X.p[c * X.ps + (long)j * X.ld + i] = al * (c == 0 ? v : -v);
      }
  }
}

// Exponent e with |v| < 2^e for every v of a row (A-operand scaling) or a
// column (B-operand scaling), over all four planes; integer ops on the bits.
template <typename T>
__global__ void k_row_maxexp(Planes<const T> A, int rows, int cols, int* e) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  int mx = -100000;
  for (int j = lane; j < cols; j += 32)
    for (int c = 0; c < 4; c++) mx = max(mx, exp_of(A.p[c * A.ps + (long)warp * A.ld + j]));
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) e[warp] = mx == -100000 ? 0 : mx;
}

template <typename T>
__global__ void k_col_maxexp_part(Planes<const T> A, int rows, int cols, int chunk_rows, int* part) {
  __shared__ int sh[CR_ROWS][CR_COLS];
  const int j = blockIdx.x * CR_COLS + threadIdx.x;
  const int r0 = blockIdx.y * chunk_rows, r1 = min(rows, r0 + chunk_rows);
  int mx = -100000;
  if (j < cols)
    for (int i = r0 + threadIdx.y; i < r1; i += CR_ROWS)
      for (int c = 0; c < 4; c++) mx = max(mx, exp_of(A.p[c * A.ps + (long)i * A.ld + j]));
  sh[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && j < cols) {
    for (int t = 1; t < CR_ROWS; t++) mx = max(mx, sh[t][threadIdx.x]);
    part[(long)blockIdx.y * cols + j] = mx;
  }
}

__global__ void k_col_maxexp_finish(const int* part, int chunks, int cols, int* e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  int mx = -100000;
  for (int ch = 0; ch < chunks; ch++) mx = max(mx, part[(long)ch * cols + j]);
  e[j] = mx == -100000 ? 0 : mx;
}

// Row chunks of a column reduction: about four blocks per SM of a 152-SM
// part in total, at least 64 rows per chunk.
static int col_chunks(int rows, int cols) {
  const int colblocks = (cols + CR_COLS - 1) / CR_COLS;
  int ch = (608 + colblocks - 1) / colblocks;
  ch = std::min(ch, (rows + 63) / 64);
  return std::max(1, std::min(ch, CR_MAX_CHUNKS));
}

__global__ void k_f32_to_f64(Planes<const float> S, int rows, int cols, Planes<double> D) {
  const long total = (long)rows * cols;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long i = t / cols, j = t % cols;
    for (int c = 0; c < 4; c++) D.p[c * D.ps + i * D.ld + j] = (double)S.p[c * S.ps + i * S.ld + j];
  }
}

__global__ void k_f64_to_f32(Planes<const double> S, int rows, int cols, Planes<float> D) {
  const long total = (long)rows * cols;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long i = t / cols, j = t % cols;
    for (int c = 0; c < 4; c++) D.p[c * D.ps + i * D.ld + j] = (float)S.p[c * S.ps + i * S.ld + j];
  }
}

int grid_for(long total) {
  long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

}  // namespace

int combine_blocks(const CombineArgs& a) {
  const int cw = combine_pairs_ok(a) ? 2 * TILE : TILE;
  return ((a.cols + cw - 1) / cw) * ((a.rows + TILE - 1) / TILE);
}

cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st, int* blocks_out) {
  const bool pairs = combine_pairs_ok(a);
  const int cw = pairs ? 2 * TILE : TILE;
  dim3 grid((a.cols + cw - 1) / cw, (a.rows + TILE - 1) / TILE);
  if (blocks_out) *blocks_out = grid.x * grid.y;
  if (a.rows <= 0 || a.cols <= 0) return cudaSuccess;
  if (pairs) {
    k_combine_f2<<<grid, TILE * TROWS, 0, st>>>(a);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  if (a.f64)
    k_combine<double><<<grid, TILE * TROWS, 0, st>>>(a);
  else
    k_combine<float><<<grid, TILE * TROWS, 0, st>>>(a);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double* partials, int nblocks, int nvals, double* out,
                                   cudaStream_t st) {
  k_reduce_partials<<<1, 256, 0, st>>>(partials, nblocks, nvals, out);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_abs_sums(const Planes<const double>& A, int m, int n, double* rowsum, double* colsum,
                            double* scratch, cudaStream_t st) {
  k_row_abs_sums<<<(m + 7) / 8, 256, 0, st>>>(A, m, n, rowsum);
  ++g_kernel_launches;
  const int ch = col_chunks(m, n), chunk_rows = (m + ch - 1) / ch;
  k_col_abs_part<<<dim3((n + CR_COLS - 1) / CR_COLS, ch), dim3(CR_COLS, CR_ROWS), 0, st>>>(A, m, n, chunk_rows,
                                                                                         scratch);
  ++g_kernel_launches;
  k_col_abs_finish<<<(n + 255) / 256, 256, 0, st>>>(scratch, ch, n, colsum);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_max(const double* v, int n, double* out, cudaStream_t st) {
  k_max<<<1, 256, 0, st>>>(v, n, out);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_fro2_partials(const Planes<const double>& A, const Planes<const double>* B, int m, int n,
                                 double* partials, cudaStream_t st, int* blocks_out, double scale, double diag) {
  const long tasks = (long)m * ((n + FRO_COLS - 1) / FRO_COLS);
  int blocks = (int)(tasks < 1024 ? tasks : 1024);
  if (blocks < 1) blocks = 1;
  *blocks_out = blocks;
  Planes<const double> Bz = B ? *B : Planes<const double>();
  k_fro2<<<blocks, FRO_COLS, 0, st>>>(A, Bz, B ? 1 : 0, m, n, scale, diag, partials);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_antiherm_partials(const Planes<const double>& M, int n, double* partials, cudaStream_t st,
                                     int* blocks_out) {
  dim3 grid((n + TILE - 1) / TILE, (n + TILE - 1) / TILE);
  *blocks_out = grid.x * grid.y;
  k_antiherm<<<grid, TILE * TROWS, 0, st>>>(M, n, partials);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_init_x0(const Planes<const double>& A, int m, int n, double alpha, const Planes<double>& X,
                           cudaStream_t st) {
  dim3 grid((n + TILE - 1) / TILE, (m + TILE - 1) / TILE);
  k_init_x0<<<grid, TILE * TROWS, 0, st>>>(A, m, n, alpha, X);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_maxexp(const Planes<const double>& A, int rows, int cols, int by_col, int* e, int* scratch,
                          cudaStream_t st) {
  if (by_col) {
    const int ch = col_chunks(rows, cols), chunk_rows = (rows + ch - 1) / ch;
    k_col_maxexp_part<double><<<dim3((cols + CR_COLS - 1) / CR_COLS, ch), dim3(CR_COLS, CR_ROWS), 0, st>>>(
        A, rows, cols, chunk_rows, scratch);
    k_col_maxexp_finish<<<(cols + 255) / 256, 256, 0, st>>>(scratch, ch, cols, e);
    g_kernel_launches += 2;
  } else {
    k_row_maxexp<double><<<(rows + 7) / 8, 256, 0, st>>>(A, rows, cols, e);
    ++g_kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_maxexp_f32(const Planes<const float>& A, int rows, int cols, int by_col, int* e, int* scratch,
                              cudaStream_t st) {
  if (by_col) {
    const int ch = col_chunks(rows, cols), chunk_rows = (rows + ch - 1) / ch;
    k_col_maxexp_part<float><<<dim3((cols + CR_COLS - 1) / CR_COLS, ch), dim3(CR_COLS, CR_ROWS), 0, st>>>(
        A, rows, cols, chunk_rows, scratch);
    k_col_maxexp_finish<<<(cols + 255) / 256, 256, 0, st>>>(scratch, ch, cols, e);
    g_kernel_launches += 2;
  } else {
    k_row_maxexp<float><<<(rows + 7) / 8, 256, 0, st>>>(A, rows, cols, e);
    ++g_kernel_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const Planes<const float>& src, int rows, int cols, const Planes<double>& dst,
                              cudaStream_t st) {
  k_f32_to_f64<<<grid_for((long)rows * cols), 256, 0, st>>>(src, rows, cols, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_f64_to_f32(const Planes<const double>& src, int rows, int cols, const Planes<float>& dst,
                              cudaStream_t st) {
  k_f64_to_f32<<<grid_for((long)rows * cols), 256, 0, st>>>(src, rows, cols, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}


template <typename T>
static cudaError_t slice_rows_t(const Planes<const T>& A, int rows, int cols, const int* e, int S, bf16* dst,
                                long ld, long ps, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if ((ld & 7) || (ps & 7) || (reinterpret_cast<uintptr_t>(dst) & 15) || ld < ((cols + 7) / 8) * 8)
    return cudaErrorInvalidValue;
  const long total = 4L * rows * ((cols + 7) / 8);
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_slice_rows<T><<<blocks, 256, 0, st>>>(A, rows, cols, e, S, dst, ld, ps);
  ++g_kernel_launches;
  return cudaGetLastError();
}
template <typename T>
static cudaError_t slice_cols_t(const Planes<const T>& A, int rows, int cols, const int* e, int S, bf16* dst,
                                long ld, long ps, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if ((ld & 7) || (ps & 7) || (reinterpret_cast<uintptr_t>(dst) & 15) || ld < ((rows + 7) / 8) * 8)
    return cudaErrorInvalidValue;
  dim3 grid((cols + 63) / 64, (rows + 31) / 32, 4);
  k_slice_cols<T><<<grid, 256, 0, st>>>(A, rows, cols, e, S, dst, ld, ps);
  ++g_kernel_launches;
  return cudaGetLastError();
}
cudaError_t launch_slice_rows(const Planes<const double>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st) {
  return slice_rows_t<double>(A, rows, cols, e, S, dst, ld, ps, st);
}
cudaError_t launch_slice_rows(const Planes<const float>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st) {
  return slice_rows_t<float>(A, rows, cols, e, S, dst, ld, ps, st);
}
cudaError_t launch_slice_cols(const Planes<const double>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st) {
  return slice_cols_t<double>(A, rows, cols, e, S, dst, ld, ps, st);
}
cudaError_t launch_slice_cols(const Planes<const float>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st) {
  return slice_cols_t<float>(A, rows, cols, e, S, dst, ld, ps, st);
}

}  // namespace qp
