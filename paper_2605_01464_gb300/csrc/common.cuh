// common.cuh -- internal types shared by the CUDA sources of libqpinv.
//
// A quaternion matrix lives in HBM as four real planes (s, x, y, z), the
// layout of the C ABI.  Besides the FP64 "master" planes, a matrix that
// feeds the tensor cores also carries BF16 split copies:
//   A-form: row-major rows x cols (K-major when the matrix is the left
//           operand, K = cols);
//   B-form: the plane-wise transpose, cols x rows (K-major when the matrix
//           is the right operand, K = rows).
// Split level L stores L BF16 terms v = t0 + t1 + ... (each the BF16
// rounding of the remainder), level-major then component-major.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qp {

// kernels launched by this thread through the launch_* functions below
extern thread_local long long g_kernel_launches;

typedef __nv_bfloat16 bf16;

// Row-major plane set: element (c, i, j) at p[c * ps + i * ld + j].
template <typename T>
struct Planes {
  T* p = nullptr;
  long ld = 0;  // elements between rows
  long ps = 0;  // elements between component planes
};

// BF16 split forms of one matrix (either pointer may be null).
struct Split16 {
  bf16* a = nullptr;  // A-form [level][comp][rows][lda]
  long lda = 0, psa = 0;
  bf16* b = nullptr;  // B-form [level][comp][cols][ldb]
  long ldb = 0, psb = 0;
  int levels = 0;
};

// Output specification of the fused combine kernel:
//   out = cacc * acc + sum_t caux[t] * aux_t + diag * I   (diag on plane s)
// The master output (and every aux input) has the master type of the pass:
// float (tensor-core phase) or double (FP64 phase).  BF16 outputs are either
// round-to-nearest splits of the FP32 value (t0 = bf16(v), t1 = bf16(v - t0),
// ...) or, when exp_a / exp_b are given, exact 7-bit slices of v * 2^-e
// (e = exponent of the row (A-form) or column (B-form) maximum): slice s is
// an integer in [-64, 64] ([-128, 128] for s = 0) times 2^(-7(s+1)), which
// BF16 holds exactly.  Slicing is done in integer arithmetic.
struct OutSpec {
  void* mp = nullptr;  // master output planes (type of the pass), may be null
  long mld = 0, mps = 0;
  Split16 s16;         // BF16 outputs (a and/or b may be null)
  const int* exp_a = nullptr;  // per-row exponents: exact slicing of the A-form
  const int* exp_b = nullptr;  // per-column exponents: exact slicing of the B-form
  double cacc = 0.0;
  double caux[4] = {0, 0, 0, 0};
  double diag = 0.0;
};

enum { ACC_F32 = 0, ACC_F64 = 1, ACC_I64 = 2 };

constexpr int kMaxOut = 3;

struct CombineArgs {
  int rows = 0, cols = 0;
  int f64 = 0;                // master type of aux inputs and outputs: 0 float, 1 double
  const void* acc = nullptr;  // accumulator planes, may be null
  const long long* acc2 = nullptr;  // ACC_I64: a second accumulator of the same layout, summed
  int acc_kind = ACC_F32;     // ACC_I64: fixed point, value = acc * 2^(erow[i] + ecol[j] - shift)
  long ld_acc = 0, ps_acc = 0;
  const int* acc_erow = nullptr;
  const int* acc_ecol = nullptr;
  int acc_shift = 0;
  const void* aux[4] = {nullptr, nullptr, nullptr, nullptr};
  long ld_aux[4] = {0, 0, 0, 0}, ps_aux[4] = {0, 0, 0, 0};
  OutSpec out[kMaxOut];
  int nout = 0;
  double* partials = nullptr;  // per block: ||out0 - aux0||^2, ||out0||^2, non-finite count
};

}  // namespace qp

// Host-side launch helpers implemented in elementwise.cu / qgemm_*.cu.
namespace qp {

// blocks (and partials) launch_combine will use for these arguments
int combine_blocks(const CombineArgs& a);
cudaError_t launch_combine(const CombineArgs& a, cudaStream_t st, int* blocks_out);
cudaError_t launch_reduce_partials(const double* partials, int nblocks, int nvals, double* out,
                                   cudaStream_t st);
// colsum needs `scratch` of COL_SCRATCH(n) doubles
cudaError_t launch_abs_sums(const Planes<const double>& A, int m, int n, double* rowsum,
                            double* colsum, double* scratch, cudaStream_t st);
cudaError_t launch_max(const double* v, int n, double* out, cudaStream_t st);
// scratch entries of a column reduction over `cols` columns
inline long COL_SCRATCH(long cols) { return 64 * cols; }
// Partials (sum of squares, non-finite count of A) of ||scale A + diag I - B||_F^2
// (B optional; diag on plane s only): 2 doubles per block, *blocks_out blocks.
cudaError_t launch_fro2_partials(const Planes<const double>& A, const Planes<const double>* B, int m,
                                 int n, double* partials, cudaStream_t st, int* blocks_out, double scale = 1.0,
                                 double diag = 0.0);
cudaError_t launch_antiherm_partials(const Planes<const double>& M, int n, double* partials,
                                     cudaStream_t st, int* blocks_out);
cudaError_t launch_init_x0(const Planes<const double>& A, int m, int n, double alpha, const Planes<double>& X,
                           cudaStream_t st);
// by_col needs `scratch` of COL_SCRATCH(cols) ints
cudaError_t launch_maxexp_f32(const Planes<const float>& A, int rows, int cols, int by_col, int* e, int* scratch,
                              cudaStream_t st);
cudaError_t launch_f64_to_f32(const Planes<const double>& src, int rows, int cols, const Planes<float>& dst,
                              cudaStream_t st);
cudaError_t launch_maxexp(const Planes<const double>& A, int rows, int cols, int by_col, int* e, int* scratch,
                          cudaStream_t st);
cudaError_t launch_f32_to_f64(const Planes<const float>& src, int rows, int cols,
                              const Planes<double>& dst, cudaStream_t st);

// Exact slices (S balanced 7-bit digits of v * 2^-e) of a row-major plane
// set: A-form rows (row exponents e[i]; dst [S][4][rows][ld]) or the
// transposed B-form (column exponents e[j]; dst [S][4][cols][ld]); padding
// up to the next multiple of 8 along the slice rows is written as 0.
cudaError_t launch_slice_rows(const Planes<const double>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st);
cudaError_t launch_slice_rows(const Planes<const float>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st);
cudaError_t launch_slice_cols(const Planes<const double>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st);
cudaError_t launch_slice_cols(const Planes<const float>& A, int rows, int cols, const int* e, int S, bf16* dst,
                              long ld, long ps, cudaStream_t st);

cudaError_t launch_qgemm_f64(int M, int K, int N, const Planes<const double>& A,
                             const Planes<const double>& B, const Planes<double>& C,
                             cudaStream_t st);

// Combine pass fused into the epilogue of the tensor-core GEMM: the product
// never goes to HBM; each output o is
//   out_o = cacc * (A B) + sum_t caux[t] * aux_t + diag * I   (diag on plane s)
// evaluated in the master type (FP32, or FP64 with f64 = 1) and written as a
// master and/or round-to-nearest BF16 splits of its FP32 rounding (A-form
// row-major, B-form transposed); in the FP32 case optionally with the
// stop-test partials of output 0 (||out0 - aux0||^2, ||out0||^2, non-finite
// count) per (CTA, epilogue warp).
// Outputs must not alias the product's operand forms (other CTAs are still
// reading them); an output may alias an aux plane (same element, same thread).
struct EpiOut {
  void* mp = nullptr;  // master planes, float (double when EpiArgs::f64); may be null
  long mld = 0, mps = 0;
  bf16* a = nullptr;  // A-form splits [level][comp][rows][lda] (may be null)
  long lda = 0, psa = 0;
  bf16* b = nullptr;  // B-form splits [level][comp][cols][ldb] (may be null)
  long ldb = 0, psb = 0;
  int levels = 0;
  double cacc = 0.0, caux[4] = {0, 0, 0, 0}, diag = 0.0;  // rounded to the master type at use
};
struct EpiArgs {
  int nout = 0;  // 0: plain FP32 store of the product into TcGemmArgs::C
  EpiOut out[kMaxOut];
  const void* aux[4] = {nullptr, nullptr, nullptr, nullptr};  // planes of the master type
  long ld_aux[4] = {0, 0, 0, 0}, ps_aux[4] = {0, 0, 0, 0};
  double* partials = nullptr;  // 3 values per (CTA, epilogue warp): tc_partial_blocks(M, N) blocks (f64 == 0 only)
  int f64 = 0;  // 1: aux inputs and output masters are double planes (FP64 arithmetic in the epilogue)
};
int tc_partial_blocks(int M, int N, int broad);

// Tensor-core quaternion GEMM on BF16 split operands.  acc (FP32) = sum over
// the listed (i, j) term pairs of A_i * B_j, restricted to k in [k0, k1).
struct TcGemmArgs {
  int M = 0, N = 0, K = 0;
  // Output: FP32 store into C, or (C64 != null) int64 fixed-point
  // accumulation C64 += rint(acc * 2^shift).
  long long* C64 = nullptr;
  long ld64 = 0, ps64 = 0;
  int shift = 0;
  int k0 = 0, k1 = 0;
  const Split16* A = nullptr;  // uses the A-form
  const Split16* B = nullptr;  // uses the B-form
  int npairs = 0;
  int pair_i[16] = {0}, pair_j[16] = {0};
  int pair_acc[16] = {0};  // TMEM accumulator of each pair (1 only with C64: the two are summed)
  Planes<float> C;  // FP32 output
  EpiArgs epi;      // epi.nout > 0: fused combine instead of the plain store (FP32 output only)
  int broad = -1;   // one-accumulator products with N >= 128 on 128-column tiles (one CTA per SM):
                    // 1 always, 0 never, -1 when the epilogue is not fused
  int* err = nullptr;  // device error word (bounded-wait expiry)
};
cudaError_t launch_qgemm_tc(const TcGemmArgs& a, cudaStream_t st);

// FP64-accurate product from S exact slices per operand in one launch
// (qgemm_emu.cu): C64 (+ C64b) = sum over levels d < S of the level-d slice
// products, in 64-bit fixed point (value * 2^shift); the accumulators are
// written, not added to (no clearing needed).  kc[d] = K chunk of level d
// (multiple of 32, or >= K), short enough that every FP32 partial sum of the
// level is exact.  emu_fused_ok(K, S) says whether K is small enough for the
// kernel's int32 per-level sums.
struct EmuGemmArgs {
  int M = 0, N = 0, K = 0;
  const Split16* A = nullptr;  // A-form slices (levels >= S)
  const Split16* B = nullptr;  // B-form slices (levels >= S)
  int S = 0;
  int kc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long* C64 = nullptr;
  long long* C64b = nullptr;  // non-null: a second accumulator (same layout) for half of the levels
  long ld64 = 0, ps64 = 0;
  int shift = 0;
  int* err = nullptr;
};
bool emu_fused_ok(int K, int S);
cudaError_t launch_qgemm_emu(const EmuGemmArgs& a, cudaStream_t st);
// The same product on pairs of SMs (qgemm_emu_pair.cu: 256 x 64 tiles,
// tcgen05 cta_group::2); same arguments and result.
cudaError_t launch_qgemm_emu_pair(const EmuGemmArgs& a, cudaStream_t st);
bool tc_supported();

// Batched solver (batched_impl.cuh: host side in batched.cu, kernels in batched_tile<t>.cu).
struct BatchResultHost {
  int status, iters, side, gemms;
  double alpha, delta, delta_rel;
  double E[4], E_rel[4];
};
}  // namespace qp
#include <vector>
namespace qp {
// CTA GEMM engines of the batched kernel: CUDA-core double-FP32 tiles
// (quaternion entries) 0: 16x16, 1: 32x32, 2: 64x32, 3: 32x64, 4: 64x64, and
// 5: the tensor-core exact-slice engine (batched_tc.cu).
constexpr int BATCH_TILES = 6;
constexpr int BATCH_TILE_TC = 5;
const char* batched_tile_name(int tile);
// Device and pinned host buffers of one batched call (owned by the context).
struct BatchRun {
  int tile = 1, slots = 0;
  void* ws = nullptr;  // slots * batched_slot_bytes()
  void* tc_ws = nullptr;    // tensor-core engine: slots * batched_tc_slot_bytes()
  void* tc_maps = nullptr;  // ... its TMA maps on the device (2 per slot)
  void* host_maps = nullptr;  // pinned staging of the maps
  int* err = nullptr;       // device error word
  void *dev_items = nullptr, *dev_order = nullptr, *dev_results = nullptr;
  int* dev_counter = nullptr;
  void *host_items = nullptr, *host_order = nullptr, *host_results = nullptr;  // pinned
};
// A captured CUDA graph of the call (upload, counter reset, the persistent
// kernel, result download), replayed while the launch shape is unchanged.
struct BatchGraph {
  cudaStream_t stream = nullptr;  // capture / replay stream (non-blocking)
  cudaGraphExec_t exec = nullptr;
  unsigned long long key = 0;
  int replays = 0;
};
cudaError_t run_batched(int batch, const int* m, const int* n, const double* const* A, const long* lda,
                        double* const* X, const long* ldx, int method, double tol, int max_iter, int mparam,
                        int stop_rule, int alpha_mode, double alpha_user, const double* hpi19_k, const BatchRun& r,
                        BatchGraph* graph, std::vector<BatchResultHost>& out, cudaStream_t st);
size_t batched_slot_bytes();
size_t batched_tc_slot_bytes();  // slice scratch of one tensor-core engine slot
// Learned alpha (alpha.cu).
int alpha_nweights();
int alpha_ntrain();
int alpha_feature_scratch_floats(int m, int n);
int power_radius_doubles(int s, int steps);  // dscratch entries of power_radius
cudaError_t power_radius(const Planes<const float>& M, int s, int steps, float* scratch, double* dscratch,
                         double* pin, cudaStream_t st, double* rho);
cudaError_t alpha_features(const Planes<const float>& A, int m, int n, double fro2, double norm1, double norminf,
                           float* scratch, double* dscratch, double* pin, cudaStream_t st, float* feat,
                           double* theta1_out);
void alpha_init_weights(float* W, unsigned long long seed);
size_t alpha_scratch_floats(int B);
cudaError_t alpha_forward(const float* dW, const float* dX, int B, float* scratch, float* dy_out, cudaStream_t st);
cudaError_t alpha_gradient(const float* dW, const float* dX, const float* dT, int B, float* scratch, float* dG,
                           double* dloss, cudaStream_t st);
cudaError_t alpha_adam(float* dW, const float* dG, float* dM1, float* dM2, int t, float lr, cudaStream_t st);
size_t batched_item_bytes();
size_t batched_result_bytes();
int batched_max_dim();
int batched_slots_per_sm(int tile);

// CUR image completion (cur.cu): the data-consistency fill, the gather of the
// CUR factors and the Gaussian filter, on contiguous planes (ps = m * n).
struct CurFill {
  const double* M[4] = {nullptr, nullptr, nullptr, nullptr};  // observed planes, row stride ldm
  long ldm = 0;
  const unsigned char* mask = nullptr;  // nonzero = observed, row stride ldk
  long ldk = 0;
  const double* X = nullptr;  // estimate for the unobserved pixels (null: 0); may alias C
  double* C = nullptr;
  int m = 0, n = 0;
};
constexpr int kMaxGaussRadius = 16;
struct GaussTaps {
  int radius = 0;
  double w[2 * kMaxGaussRadius + 1];
};
cudaError_t launch_cur_fill(const CurFill& f, cudaStream_t st);
cudaError_t launch_cur_gather(const double* C, int m, int n, int r, const int* I, const int* J, double* CJ,
                              double* RI, double* W, cudaStream_t st);
cudaError_t launch_cur_gauss(const double* in, double* out, int m, int n, const GaussTaps& g, cudaStream_t st);
// Signal filtering (toeplitz.cu): X(i, j) = x(t0 + i - j), (p+1) x (p+1),
// from planes of samples with plane stride xps; X contiguous.
cudaError_t launch_toeplitz(const double* x, long xps, int p, int t0, double* X, cudaStream_t st);
// Global Krylov solvers (krylov.cu): blocks of L doubles, basis stride L.
cudaError_t launch_block_dot(const double* V, int c, const double* W, long L, double* h, cudaStream_t st);
cudaError_t launch_block_sub(double* W, const double* V, const double* h, int c, long L, double* hcol,
                             cudaStream_t st);
cudaError_t launch_norm_scale(const double* W, long L, double* nrm, double* out, cudaStream_t st);
cudaError_t launch_basis_add(double* X, const double* V, const double* y, int k, long L, cudaStream_t st);
cudaError_t launch_sub(double* out, const double* a, const double* b, long L, cudaStream_t st);
cudaError_t launch_givens(double* col, double* cs, double* sn, double* g, int j, int fom, double* res,
                          cudaStream_t st);
// C = A B (FP64) for B with 1..16 columns: one block per row of C.
bool skinny_ok(int m);
cudaError_t launch_qgemm_skinny(int M, int K, int m, const Planes<const double>& A, const Planes<const double>& B,
                                const Planes<double>& C, cudaStream_t st);

}  // namespace qp
