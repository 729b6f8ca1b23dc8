/*
 * qpinv.h -- C ABI of the GB300 (sm_103a) quaternion pseudoinverse library.
 *
 * The library computes X ~ A^dagger, the Moore-Penrose pseudoinverse of an
 * m x n quaternion matrix A (Definition 2.1: AXA = A, XAX = X, (AX)^H = AX,
 * (XA)^H = XA), with the hyperpower iterations of the paper: QRAPID
 * (Algorithm 1), QSAI (Algorithm 2), QHPI19 (Algorithm 3, factorized
 * order-19 form of Sec. 3.3) and the Newton-Schulz baseline
 * X_{j+1} = X_j (2I - A X_j) (Sec. 1).  Every iteration starts from
 * X_0 = alpha A^H (Theorem 1) and is dominated by quaternion matrix-matrix
 * products, which run in the library's own CUDA kernels.
 *
 * Data layout (every entry point): a quaternion matrix is passed as four
 * real component planes s, x, y, z (q = s + x i + y j + z k, Sec. 2), each a
 * row-major array of doubles with a leading dimension (elements between
 * consecutive rows).  A is m x n with leading dimension lda >= n; X is n x m
 * with leading dimension ldx >= m.  Plane pointers may be device pointers
 * (cudaMalloc / torch CUDA tensors) or host pointers (pageable or pinned);
 * the library detects which with cudaPointerGetAttributes and, for host
 * pointers, copies through device buffers it owns, inside the call.
 *
 * Ownership: the caller owns A and X and every array passed in.  The
 * context owns all scratch memory (residual powers, polynomial blocks,
 * tensor-core operand splits, reduction partials), grown on demand and
 * released by qpinv_free.  The library never frees caller memory.
 *
 * Errors: every int-returning entry point returns QPINV_OK (0) or a
 * negative QPINV_E_* code; qpinv_last_error(ctx) gives a message.  Solver
 * outcomes (converged, plateau, not converged, diverged) are not errors:
 * they are reported in qpinv_result.status, and X is always written.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Calls are synchronous with respect to the host: they
 * return after the result has been read back (the stop test needs two
 * scalars per iteration).
 */
#ifndef QPINV_H
#define QPINV_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define QPINV_OK 0
#define QPINV_E_INVALID (-1)      /* bad size, leading dimension, pointer or option */
#define QPINV_E_CUDA (-2)         /* a CUDA runtime/driver call failed */
#define QPINV_E_NOMEM (-3)        /* device workspace could not be allocated */
#define QPINV_E_NONFINITE (-4)    /* A contains NaN or Inf */
#define QPINV_E_TIMEOUT (-5)      /* a device-side bounded wait expired (kernel aborted cleanly) */
#define QPINV_E_UNSUPPORTED (-6)  /* option combination not available on this device */
#define QPINV_E_NOALLOC_LIMIT (-7) /* qpinv_qgemm_noalloc: a dimension exceeds QPINV_NOALLOC_MAX_DIM */

/* Largest m, k and n accepted by qpinv_qgemm_noalloc. */
#define QPINV_NOALLOC_MAX_DIM 256

/* ---- solver outcome (qpinv_result.status) ----------------------------- */
#define QPINV_CONVERGED 0     /* stop rule met; X is X_{j+1}.  In MIXED's polish phase also when the
                                 residual R of the returned X bounds the next step below tol:
                                 ||R||_F <= tol (relative rule) or ||X||_F r / (1 - r) < tol,
                                 r = ||R||_F (absolute rule) */
#define QPINV_PLATEAU 1       /* rounding floor reached: the relative step stopped decreasing after
                                 falling below 1e-3 (X is the iterate before that step), or, in
                                 MIXED's polish phase, the step (or the residual of X, which bounds
                                 the next step) is below 2^-53 sqrt(||A||_1 ||A||_inf) ||X||_F */
#define QPINV_NOT_CONVERGED 2 /* max_iter updates (or MIXED's polish iterations) done without the
                                 above; X is the last iterate */
#define QPINV_DIVERGED 3      /* a non-finite iterate appeared; X is the last finite iterate */
#define QPINV_NONFINITE_INPUT 4 /* qpinv_solve_batched: this A holds NaN/Inf; its X is left untouched */

/* ---- methods ----------------------------------------------------------- */
typedef enum {
  QPINV_NS = 0,     /* Newton-Schulz, order 2, 2 products per iteration (Sec. 1) */
  QPINV_QSAI = 1,   /* Algorithm 2, order 10, 6 products per iteration */
  QPINV_QRAPID = 2, /* Algorithm 1 with step parameter N, 8+2N products per iteration */
  QPINV_QHPI19 = 3, /* Algorithm 3, order 19, 7 products per iteration */
  QPINV_QHPIM = 4   /* unfactorized hyperpower iteration of order k = hyper_order (Definition 1;
                       QHONSchultz(k) of Example 3): X_{j+1} = X_j (I + R + ... + R^{k-1}),
                       the sum by Horner's rule, k products per iteration */
} qpinv_method;

/* ---- options --------------------------------------------------------- */
enum {
  QPINV_PREC_FP64 = 0,  /* every product in FP64 on the CUDA cores */
  QPINV_PREC_MIXED = 1, /* tensor-core BF16-split products with FP32 accumulation, then
                           polish iterations whose residual R = I - A X and update X t are
                           FP64-accurate (QPINV_PREC_EMU products) */
  QPINV_PREC_TC = 2,    /* tensor-core products only (FP32-level output) */
  QPINV_PREC_EMU = 3,   /* every product FP64-accurate on the tensor cores: exact 7-bit slices
                           per operand (power-of-two row and column scaling; 8 slices in a
                           solve, `split_level` = 2..8 in qpinv_qgemm), K-chunked so every FP32
                           partial sum is exact, accumulated in 64-bit fixed point.  Use it for
                           rank-deficient A, whose null-space rounding noise the iteration
                           multiplies by its order each step */
  QPINV_PREC_DF32 = 4   /* reported only (qpinv_result.precision of batched solves): double-FP32
                           arithmetic on the CUDA cores */
};
enum { QPINV_ALPHA_SAFE = 0,     /* 1 / (||A||_1 ||A||_inf), entry moduli; always < 2/sigma_1^2 */
       QPINV_ALPHA_SPECTRAL = 1, /* 1 / sigma_1^2 (Algorithms 1-3), sigma_1 by power iteration */
       QPINV_ALPHA_FRO = 2,      /* 1 / ||A||_F^2 (Sec. 4 text) */
       QPINV_ALPHA_USER = 3,     /* alpha_user (Example 3 uses a fixed alpha) */
       QPINV_ALPHA_LEARNED = 4   /* MLP on sketched features; falls back to SAFE on a failed check */ };
enum { QPINV_SIDE_AUTO = 0,  /* residual on the smaller side */
       QPINV_SIDE_RIGHT = 1, /* paper's form: R = I_m - A X, X_{j+1} = X p(R) */
       QPINV_SIDE_LEFT = 2   /* R = I_n - X A, X_{j+1} = p(R) X (same iterates in exact arithmetic) */ };
enum { QPINV_STOP_PAPER_ABS = 0,  /* ||X_{j+1} - X_j||_F < tol (Algorithms 1-3) */
       QPINV_STOP_REL_PLATEAU = 1 /* ||X_{j+1}-X_j||_F / ||X_{j+1}||_F <= tol, with plateau detection */ };

typedef struct {
  int precision;     /* QPINV_PREC_FP64, _MIXED, _TC or _EMU; default MIXED */
  int split_level;   /* BF16 terms of the tensor-core R-products (polynomials in R): 1 = bf16,
                        2 = bf16x3, 3 = bf16x6; 0 = automatic (1 term while the relative step
                        exceeds 0.5, then 2).  X-products use 2 terms (square MIXED) or 3, then
                        exact slices once ||A|| ||X|| > 1e3 (4 for the residual; 3 for the update
                        X t of square MIXED solves) */
  int polish_iters;  /* MIXED: iterations with an FP64 residual at the end (default 2); the
                        tensor-core phase ends when the step stalls, when the residual predicted
                        after the polish iterations is negligible (||R_j||_F, or the spectral
                        radius of R_j when the relative step suggests it), or when drel < 1e-6.
                        Rectangular A is projected onto the pseudoinverse's row / column space
                        after the first polish iteration */
  int alpha_mode;    /* QPINV_ALPHA_*, default SAFE */
  double alpha_user; /* used with QPINV_ALPHA_USER */
  int qrapid_N;      /* QRAPID step parameter N >= 0 (default 5) */
  int side;          /* QPINV_SIDE_*, default AUTO; a residual forced onto the larger side runs
                        MIXED / TC solves as QPINV_PREC_EMU (its complement behaves like a
                        rank-deficient residual) */
  int stop_rule;     /* QPINV_STOP_*, default REL_PLATEAU */
  int penrose;       /* 1: compute E1..E4 in FP64 after the solve (default 1) */
  int profile;       /* 1: time every kernel launch with CUDA events (qpinv_get_stats) */
  int batched_tile;  /* qpinv_solve_batched CTA GEMM engine: -1 = autotune (default; each batch
                        signature is timed once per context on a sample of its matrices),
                        CUDA-core double-FP32 tiles 0 = 16x16, 1 = 32x32, 2 = 64x32, 3 = 32x64,
                        4 = 64x64, or 5 = tensor cores (exact 7-bit BF16 slices of the
                        double-FP32 operands, tcgen05, int64 accumulation) */
  int hyper_order;   /* QPINV_QHPIM order k, 2..64 (default 19; k = 2 is Newton-Schulz, and
                        k = 1, X_{j+1} = X_j, makes no progress and is rejected) */
  int fuse_epilogue; /* 1 (default): the combine pass after a BF16 tensor-core product (residual
                        R = I - A X, the polynomial blocks in R, the X update with its stop norms)
                        runs in the GEMM's epilogue, on FP32 masters and, in the FP64 polish
                        steps, on FP64 masters (passes that carry FP64 stop norms excepted);
                        0: separate combine kernel (same arithmetic) */
  int emu_pair;      /* 1: FP64-accurate exact-slice products with more than 128 rows on pairs of SMs
                        (256 x 64 tiles, one MMA for both CTAs, half of the B operand staged per SM);
                        0 or -1 (default): one SM per 128 x 128 tile and component pair, which was
                        measured faster at every size (5.3 against 7.3 ms at 2048^3, 44.9 against
                        58.3 ms at 4096^3, 8 slices).  Same arithmetic, bit-identical results */
  int tc_broad;      /* BF16-split products with M, N >= 128 and one accumulator on 128-column tiles
                        (one CTA per SM, a 512-column TMEM accumulator) or 64-column tiles (two CTAs
                        per SM): -1 (default) 128 columns for products without a fused combine
                        epilogue (measured 10-19 % faster; with the epilogue the one CTA per SM
                        cancels the gain), 1 always, 0 never.  Same arithmetic, bit-identical
                        results */
} qpinv_options;

typedef struct {
  int status;        /* QPINV_CONVERGED / _PLATEAU / _NOT_CONVERGED / _DIVERGED */
  int iters;         /* X-updates contained in the returned X */
  int tc_iters;      /* ... of which with tensor-core residuals */
  int polish_iters;  /* ... of which with an FP64 residual */
  double alpha;      /* scaling used in X_0 = alpha A^H */
  int alpha_source;  /* QPINV_ALPHA_* actually used */
  int side;          /* QPINV_SIDE_RIGHT or QPINV_SIDE_LEFT actually used */
  int precision;     /* precision that produced X: a MIXED solve with penrose = 1 that diverges or
                        whose E_rel[0] exceeds 1e-9 (typically rank-deficient A) is repeated in
                        QPINV_PREC_EMU and reports EMU here, gemms then counting both attempts;
                        batched solves report QPINV_PREC_DF32 */
  double delta;      /* ||X_{j+1} - X_j||_F of the last computed step */
  double delta_rel;  /* delta / ||X_{j+1}||_F */
  double E[4];       /* Sec. 4: ||AXA-A||_F, ||XAX-X||_F, ||(AX)^H-AX||_F, ||(XA)^H-XA||_F */
  double E_rel[4];   /* E divided by ||A||_F, ||X||_F, ||AX||_F, ||XA||_F */
  long long gemms;   /* quaternion matrix products issued */
  double time_ms;    /* wall time of the call */
  int alpha_fallback; /* 1: QPINV_ALPHA_LEARNED was asked for and the safe alpha used instead --
                         the prediction failed Thm. 1's condition before the solve, or the solve
                         started from it did not contract (a residual norm that grew, a diverged
                         or unconverged iteration) and was restarted from the safe alpha */
} qpinv_result;

typedef struct {
  long long kernel_launches;  /* every kernel of this library launched since the last reset */
  long long tc_gemm_launches; /* tcgen05 quaternion GEMM launches (BF16 splits; chunked
                                 exact-slice launches for K beyond the fused kernel's range) */
  double tc_gemm_ms;          /* their summed duration (CUDA events on the launch stream; profile=1) */
  double tc_gemm_flops;       /* algorithmic real flops: 32 per quaternion multiply-add */
  double tc_gemm_flops_issued;/* tensor-core flops issued (split products count each pass) */
  long long f64_gemm_launches;
  double f64_gemm_ms;
  double f64_gemm_flops;
  long long ew_launches;      /* fused elementwise / reduction kernels */
  double ew_ms;
  double ew_bytes;            /* algorithmic HBM bytes of those kernels */
  long long emu_gemm_launches;/* fused exact-slice (FP64-accurate) tensor-core GEMM launches */
  double emu_gemm_ms;
  double emu_gemm_flops;      /* algorithmic: 32 per quaternion multiply-add */
  double emu_gemm_flops_issued;/* tensor-core flops issued: S(S+1)/2 slice-pair passes */
  long long batched_tile;     /* CTA GEMM tile of the last batched call (see batched_tile) */
  double batched_tune_ms;     /* time spent autotuning batched tiles */
  long long batched_graph_replays; /* batched calls served by replaying a captured CUDA graph */
  long long fused_epilogues;       /* tensor-core products whose combine pass ran in the GEMM epilogue */
  long long penrose_reused;        /* Penrose passes that reused the residual I - AX (or I - XA) the last
                                      iteration had formed for the returned X with FP64 masters and
                                      FP64-accurate products (one product fewer) */
} qpinv_stats;

typedef struct qpinv_ctx qpinv_ctx;

/* Fills *opt with the defaults listed above. */
void qpinv_default_options(qpinv_options* opt);

/* Creates a context bound to CUDA device `device` (the caller's current
 * device is restored on return from every call).  opt may be NULL (defaults).
 * *ctx receives the context; release it with qpinv_free. */
int qpinv_init(qpinv_ctx** ctx, int device, const qpinv_options* opt);

/* Replaces the options of an existing context. */
int qpinv_set_options(qpinv_ctx* ctx, const qpinv_options* opt);

/* Single solve (Algorithms 1-3, Newton-Schulz and the unfactorized iteration of
 * Definition 1; stop rules of Sec. 4 and
 * the plateau rule).  A: four planes of an m x n matrix (lda >= n); X: four
 * planes of the n x m output (ldx >= m), caller-owned.  tol: stop tolerance
 * of the chosen rule; max_iter >= 1 bounds the X-updates.  out (host,
 * may be NULL) receives the outcome.  Returns QPINV_E_NONFINITE if A holds
 * NaN or Inf (X is then left untouched). */
int qpinv_solve(qpinv_ctx* ctx, void* stream, int m, int n, const double* const A[4], long lda,
                qpinv_method method, double tol, int max_iter, double* const X[4], long ldx,
                qpinv_result* out);

/* Batched solve of `batch` independent matrices of uneven shapes (CUR
 * intersection blocks and the like; the paper solves them one by one).
 * m[b], n[b] (host arrays): shape of matrix b, each in [1, 256]; A[4*b + c]
 * and X[4*b + c] (host arrays of DEVICE pointers): plane c of matrix b, with
 * leading dimensions lda[b] >= n[b] and ldx[b] >= m[b].  All matrices are
 * solved in ONE persistent kernel launch: every CTA takes matrices from a
 * work counter (largest first) and runs alpha, X_0 = alpha A^H, the method
 * (residual on the smaller side), the stop rule of the context's options and
 * E1..E4 for each, with double-FP32 masters (an unevaluated sum of two
 * floats, ~2^-46: small blocks are often rank deficient, and null-space
 * noise grows by ~kappa^2 over a solve); the products run on the CUDA
 * cores in double-FP32 or on the tensor cores as exact-slice products of
 * the same accuracy (batched_tile).  Options used: stop_rule, qrapid_N,
 * hyper_order, batched_tile, alpha_mode (SAFE, FRO or USER; SPECTRAL and
 * LEARNED run as SAFE).
 * out[b] (host array, may be NULL) receives each outcome; tc_iters and
 * polish_iters are 0; time_ms is the whole call.  Matrices are independent:
 * a non-finite A gives QPINV_NONFINITE_INPUT for that matrix only. */
int qpinv_solve_batched(qpinv_ctx* ctx, void* stream, int batch, const int* m, const int* n,
                        const double* const* A, const long* lda, qpinv_method method, double tol,
                        int max_iter, double* const* X, const long* ldx, qpinv_result* out);

/* Releases the context and all device memory it owns.  NULL is ignored. */
void qpinv_free(qpinv_ctx* ctx);

/* Message for the last error on this context (never NULL). */
const char* qpinv_last_error(qpinv_ctx* ctx);

/* ---- learned initial scaling alpha for X_0 = alpha A^H (Thm. 1) ----
 * A 32 -> 64 -> 64 -> 1 tanh network maps 32 cheap sketched features of A to
 * y = log(alpha * theta_1), where theta_1 <= sigma_1^2 is the top Ritz value
 * of a 16-step Lanczos run on A^H A; labels are the optimum of Thm. 1's
 * contraction factor max|1 - alpha sigma_i^2|, alpha* = 2/(sigma_1^2 +
 * sigma_r^2).  With QPINV_ALPHA_LEARNED, qpinv_solve uses the prediction only
 * if alpha * theta_1 * 1.05 < 2 (Thm. 1's condition alpha < 2/sigma_1^2 with a
 * margin for theta_1); otherwise, or while the network is untrained, it uses
 * QPINV_ALPHA_SAFE (reported in qpinv_result.alpha_source). */
#define QPINV_ALPHA_NFEAT 32
#define QPINV_ALPHA_NWEIGHTS 6401 /* W1 64x32, b1, W2 64x64, b2, w3 64, b3, input mean 32, input sd 32 */
#define QPINV_ALPHA_NTRAIN 6337   /* trainable parameters: the block up to and including b3 */

/* Features of A (planes as in qpinv_solve): feat (host, 32 floats); theta1
 * (host, may be NULL) receives the Lanczos estimate of sigma_1^2. */
int qpinv_alpha_features(qpinv_ctx* ctx, void* stream, int m, int n, const double* const A[4], long lda,
                         float* feat, double* theta1);

/* Trains the context's network from scratch on the GPU (own forward,
 * backward and Adam kernels): `count` samples, feat (host, count x 32 floats,
 * row-major), label (host, count floats of y = log(alpha * theta_1)),
 * minibatches of `batch`, `epochs` passes in a seeded shuffled order, learning
 * rate lr.  loss (host, may be NULL) receives the final mean squared error. */
int qpinv_alpha_train(qpinv_ctx* ctx, void* stream, int count, const float* feat, const float* label, int epochs,
                      int batch, float lr, unsigned long long seed, double* loss);

/* Network output y for one feature vector (host, 32 floats). */
int qpinv_alpha_predict(qpinv_ctx* ctx, void* stream, const float* feat, double* y);

/* Gradient of the mean squared error over `count` samples with respect to
 * the QPINV_ALPHA_NTRAIN trainable parameters (host out), and the loss. */
int qpinv_alpha_gradient(qpinv_ctx* ctx, void* stream, int count, const float* feat, const float* label,
                         float* grad, double* loss);

/* Reads (set = 0) or loads (set = 1) the QPINV_ALPHA_NWEIGHTS weight block (host). */
int qpinv_alpha_weights(qpinv_ctx* ctx, float* w, int count, int set);

/* ---- application: CUR image completion (Sec. 5.1) ----------------------
 * Impute-reconstruct loop (eq. (update)): C^(0) = Omega . M (unobserved
 * pixels 0); for t = 0 .. iters-1:
 *   C_J = C^(t)(:, J_t), R_I = C^(t)(I_t, :);
 *   U = C_J^dagger C^(t) R_I^dagger   (form 0: eq. (Uopt), A read as the
 *                                      current filled matrix), or
 *   U = W^dagger, W = C^(t)(I_t, J_t) (form 1: the cross form, eq. (Ucross));
 *   X^(t) = (C_J U) R_I, then, if sigma > 0, the 2-D Gaussian filter of
 *   standard deviation sigma on every plane (sampled on |x| <= ceil(2 sigma),
 *   normalised, replicated borders);
 *   C^(t+1) = Omega . M + (1 - Omega) . X^(t).
 * Each pseudoinverse is a qpinv_solve with the context's options (method,
 * tol, max_iter as given); the products are FP64-accurate (exact-slice
 * tensor-core GEMMs; CUDA-core FP64 when the context's precision is FP64).
 *   - M: four planes of the m x n image (colour images: zero real plane,
 *     R, G, B in x, y, z), ldm >= n; values at unobserved pixels are ignored.
 *     mask: m x n bytes, nonzero = observed, row stride ldmask >= n.  Device
 *     or host pointers.
 *   - r in [1, min(m, n)]; I, J: HOST arrays of iters x r row / column
 *     indices (0-based; row t holds the sets of iteration t).
 *   - C: four planes (device or host, ldc >= n) receive C^(iters).
 *   - out (host, may be NULL): summary of the pseudoinverse solves.
 *   - Errors: QPINV_E_INVALID for bad sizes, strides, indices, form, method,
 *     or sigma outside [0, 8]; errors of the inner solves are returned as is
 *     (their message prefixed "pseudoinverse:"). */
typedef struct {
  int pinv_solves;        /* pseudoinverse solves run (2 per iteration, 1 with the cross form) */
  int pinv_iters;         /* their iterations, summed */
  int pinv_worst_status;  /* largest qpinv_result.status among them */
  double pinv_max_E1_rel; /* largest E1/||.||_F among them */
  double time_ms;         /* wall time of the call */
} qpinv_cur_result;

int qpinv_cur_complete(qpinv_ctx* ctx, void* stream, int m, int n, const double* const M[4], long ldm,
                       const unsigned char* mask, long ldmask, int r, int iters, const int* I, const int* J,
                       int form, qpinv_method method, double tol, int max_iter, double sigma,
                       double* const C[4], long ldc, qpinv_cur_result* out);

/* ---- application: quaternion signal filtering (Sec. 5.2) ---------------
 * Filter s(t) ~ sum_{m=0}^{p} x(t - m) h_m (eq. (conv)) as X h = s with the
 * (p+1) x (p+1) data matrix X(i, j) = x(t0 + i - j) and s(i) = s(t0 + i),
 * i, j = 0..p: h = X^dagger s by qpinv_solve (the context's options, method,
 * tol and max_iter as given), s_hat = X h (FP64-accurate products) and
 * err = ||s_hat - s|| / ||s||.
 *   - x, s: four planes of N samples each (device or host; plane c of a
 *     quaternion signal in x[c]); p >= 0 and p <= t0 <= N - 1 - p.
 *   - h, s_hat: four planes of p + 1 values each (device or host), written.
 *   - pinv_out (host, may be NULL) receives the outcome of the solve for
 *     X^dagger; err (host, may be NULL) the relative error.
 *   - Errors: QPINV_E_INVALID for bad sizes, pointers or method; errors of
 *     the solve are returned as is (message prefixed "pseudoinverse:"). */
int qpinv_toeplitz_filter(qpinv_ctx* ctx, void* stream, int N, const double* const x[4], const double* const s[4],
                          int p, int t0, qpinv_method method, double tol, int max_iter, double* const h[4],
                          double* const s_hat[4], qpinv_result* pinv_out, double* err);

/* ---- application: preconditioned global Krylov solvers (Sec. 3.5) -------
 * Solves A X = B (A n x n, B n x m quaternion) by Gl-QGMRES (kind 0) or
 * Gl-QFOM (kind 1): global Arnoldi with the real inner product
 * <V, W> = Re tr(V^H W) (classical Gram-Schmidt applied twice), Givens
 * rotations for the residual estimate, restarts every `restart` steps
 * (0 = none), X_0 = 0.  With precond_iters = k > 0 the system is left
 * preconditioned, M A X = M B, M = X_k of k QSAI iterations on A (Alg. 2,
 * safe alpha, FP64 products).  Stop: ||B' - A' X_j||_F / ||B'||_F <= tol for
 * the system solved, or max_iter Arnoldi steps.  Products are FP64 (CUDA
 * cores); the small Hessenberg least-squares updates run on the host.
 *   - A (lda >= n), B (ldb >= m), X (ldx >= m, written): four planes each,
 *     device or host.
 *   - out (host, may be NULL): iterations, convergence, the relative residual
 *     of the system solved and the true one ||B - A X|| / ||B||.
 *   - Errors: QPINV_E_INVALID for bad sizes, kind, restart < 0,
 *     precond_iters outside [0, 100], max_iter outside [1, 100000], or a
 *     cycle (restart, or max_iter without restarts) above 10000 steps: one
 *     cycle keeps (cycle + 1) basis blocks and a (cycle + 1) x cycle
 *     Hessenberg matrix; QPINV_E_NOMEM when they do not fit. */
typedef struct {
  int iters;           /* Arnoldi steps, over all restarts */
  int converged;       /* 1 if the stop tolerance was met */
  double rel_res;      /* ||B' - A' X||_F / ||B'||_F of the system solved (explicit) */
  double true_rel_res; /* ||B - A X||_F / ||B||_F */
  double time_ms;      /* wall time of the call */
} qpinv_krylov_result;

int qpinv_global_krylov(qpinv_ctx* ctx, void* stream, int n, int m, const double* const A[4], long lda,
                        const double* const B[4], long ldb, int kind, int restart, int precond_iters, double tol,
                        int max_iter, double* const X[4], long ldx, qpinv_krylov_result* out);

/* ---- building blocks, exposed for tests and measurement ---------------- */

/* C = A B for quaternion matrices (Hamilton product, Sec. 2): A is m x k
 * (lda >= k), B is k x n (ldb >= n), C is m x n (ldc >= n), all four-plane
 * FP64 arrays (device or host).  precision: QPINV_PREC_FP64 (CUDA-core FP64
 * kernel), QPINV_PREC_TC (tcgen05 kernel on BF16 splits of A and B with
 * `split_level` = 1..3 terms, FP32 accumulation) or QPINV_PREC_EMU (tcgen05,
 * `split_level` = 2..8 exact slices, FP64-accurate for 8).  C must not alias A or B. */
int qpinv_qgemm(qpinv_ctx* ctx, void* stream, int m, int k, int n, const double* const A[4],
                long lda, const double* const B[4], long ldb, double* const C[4], long ldc,
                int precision, int split_level);

/* Penrose residuals of Sec. 4 for a given pair (A, X), computed in FP64:
 * E[0..3] = ||AXA-A||_F, ||XAX-X||_F, ||(AX)^H-AX||_F, ||(XA)^H-XA||_F and
 * E_rel = E / (||A||_F, ||X||_F, ||AX||_F, ||XA||_F).  E, E_rel: host arrays of 4. */
int qpinv_penrose(qpinv_ctx* ctx, void* stream, int m, int n, const double* const A[4], long lda,
                  const double* const X[4], long ldx, double* E, double* E_rel);

/* Allocation-free quaternion GEMM (the paper has no counterpart: this is a
 * deployment convenience).  Computes C = A B like qpinv_qgemm with
 * QPINV_PREC_TC and `split_level` = 1..3 BF16 terms, for callers that may not
 * allocate device memory when they need the product -- code inside a memory
 * pool or arena that forbids new cudaMalloc calls, loops that must not touch
 * the allocator after start-up, or callers without a qpinv context (a
 * context allocates its workspace on first use).  All its scratch lives in a
 * fixed array of about 4 MiB that every GPU loading the library holds until
 * the process exits; it calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   - A (m x k), B (k x n), C (m x n): four FP64 planes each, DEVICE pointers
 *     only, row-major with leading dimensions lda >= k, ldb >= n, ldc >= n;
 *     1 <= m, k, n <= QPINV_NOALLOC_MAX_DIM, else QPINV_E_NOALLOC_LIMIT;
 *     host pointers, and device pointers of a GPU other than the current
 *     one, give QPINV_E_INVALID.  C must not alias A or B.
 *   - Runs on the caller's current device and on `stream`; synchronous: it
 *     reads the kernel's error word into host memory and waits for `stream`
 *     before it returns.
 *   - The first call on each device looks up the array's device address.
 *   - Every call shares the one array: calls whose work may overlap on the GPU
 *     (other streams, unsynchronised host threads) race and must be
 *     serialised by the caller. */
int qpinv_qgemm_noalloc(void* stream, int m, int k, int n, const double* const A[4], long lda,
                        const double* const B[4], long ldb, double* const C[4], long ldc, int split_level);

/* Kernel counters and (with profile = 1) CUDA-event timings since the last reset. */
int qpinv_get_stats(qpinv_ctx* ctx, qpinv_stats* stats);
int qpinv_reset_stats(qpinv_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* QPINV_H */
