/*
 * qoracle.c -- plain, slow, FP64 CPU oracle for the quaternion hyperpower
 * pseudoinverse iterations (QRAPID, QSAI, QHPI19, Newton-Schulz, and the
 * unfactorized hyperpower iteration QHPIM of order k).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Representation: a quaternion matrix is an array of `quat` structs
 * (s, x, y, z interleaved), row-major.  Every product is the Hamilton product
 * written out per scalar (Sec. 2); every matrix product is the naive sum over
 * k in increasing order.  The loops of each algorithm follow the paper's
 * Algorithms 1-3 step by step, in the paper's notation.
 *
 * Readings of the paper (each stated where it is used):
 *  - X0 = alpha * A^H (Algs. 1-3); Sec. 4 writes A^T, which for quaternions
 *    must be the adjoint.
 *  - Alg. 3 lists R^8 and R^16 but never uses them; they are not formed
 *    (the paper's own count of seven products per iteration excludes them).
 *  - The stop rule of Algs. 1-3 is absolute (||X_{j+1}-X_j||_F < tol); a
 *    relative rule with plateau detection is offered as an option because the
 *    absolute rule is scale dependent and, for rank-deficient input, rounding
 *    noise in the null-space part of X grows by p(1) per extra iteration:
 *    PLATEAU = the relative step stopped decreasing after it had fallen below
 *    1e-3, i.e. the rounding floor was reached; X_j is returned.
 *  - Side: the paper's residual is R = I_m - A X (right form).  The left form
 *    R' = I_n - X A with X_{j+1} = p(R') X gives the same iterates in exact
 *    arithmetic (X (AX)^k = (XA)^k X); it is offered for tall inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double s, x, y, z; } quat;

/* -------- mutation hook (tests plant a mistake here to prove the pins bite) */
static int g_mutation = 0;
void qo_set_mutation(int m) { g_mutation = m; }

/* -------- quaternion scalars (Sec. 2) ------------------------------------ */

/* Hamilton product: i^2 = j^2 = k^2 = ijk = -1 (Sec. 2). */
static quat q_mul(quat p, quat q) {
  quat r;
  r.s = p.s * q.s - p.x * q.x - p.y * q.y - p.z * q.z;
  r.x = p.s * q.x + p.x * q.s + p.y * q.z - p.z * q.y;
  r.y = p.s * q.y - p.x * q.z + p.y * q.s + p.z * q.x;
  r.z = p.s * q.z + p.x * q.y - p.y * q.x + p.z * q.s;
  if (g_mutation == 1) r.z = p.s * q.z + p.x * q.y + p.y * q.x + p.z * q.s;
  return r;
}
static quat q_conj(quat q) {
  quat r = {q.s, -q.x, -q.y, -q.z};
  if (g_mutation == 2) r.y = q.y;
  return r;
}
static quat q_add(quat a, quat b) { quat r = {a.s + b.s, a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static quat q_sub(quat a, quat b) { quat r = {a.s - b.s, a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static quat q_scale(double c, quat a) { quat r = {c * a.s, c * a.x, c * a.y, c * a.z}; return r; }
static double q_abs2(quat a) { return a.s * a.s + a.x * a.x + a.y * a.y + a.z * a.z; }
static double q_abs(quat a) { return sqrt(q_abs2(a)); }

/* -------- quaternion matrices ------------------------------------------- */

typedef struct { int r, c; quat *d; } qmat;

static qmat qm_new(int r, int c) {
  qmat M; M.r = r; M.c = c;
  M.d = (quat *)calloc((size_t)(r > 0 ? r : 1) * (size_t)(c > 0 ? c : 1), sizeof(quat));
  return M;
}
static void qm_free(qmat *M) { free(M->d); M->d = NULL; }
static quat *qm_at(const qmat *M, int i, int j) { return &M->d[(size_t)i * M->c + j]; }
static qmat qm_copy(const qmat *A) {
  qmat B = qm_new(A->r, A->c);
  memcpy(B.d, A->d, sizeof(quat) * (size_t)A->r * A->c);
  return B;
}
/* a*P + b*Q + c*I  (P, Q square of the same size; Q may be NULL). */
static qmat qm_comb(double a, const qmat *P, double b, const qmat *Q, double c) {
  qmat C = qm_new(P->r, P->c);
  for (int i = 0; i < P->r; i++)
    for (int j = 0; j < P->c; j++) {
      quat v = q_scale(a, *qm_at(P, i, j));
      if (Q) v = q_add(v, q_scale(b, *qm_at(Q, i, j)));
      if (i == j) v.s += c;
      *qm_at(&C, i, j) = v;
    }
  return C;
}
static qmat qm_add(const qmat *P, const qmat *Q) { return qm_comb(1.0, P, 1.0, Q, 0.0); }

/* Adjoint A^H = conj(A)^T (Sec. 2). */
static qmat qm_adjoint(const qmat *A) {
  qmat H = qm_new(A->c, A->r);
  for (int i = 0; i < A->r; i++)
    for (int j = 0; j < A->c; j++) *qm_at(&H, j, i) = q_conj(*qm_at(A, i, j));
  return H;
}

static long long g_gemm_count = 0;

/* C = A B, C_ij = sum_k A_ik B_kj, k summed in increasing order. */
static qmat qm_mul(const qmat *A, const qmat *B) {
  qmat C = qm_new(A->r, B->c);
  const int M = A->r, K = A->c, N = B->c;
  g_gemm_count++;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < M; i++) {
    quat *crow = &C.d[(size_t)i * N];
    for (int k = 0; k < K; k++) {
      const quat a = A->d[(size_t)i * K + k];
      const quat *brow = &B->d[(size_t)k * N];
      for (int j = 0; j < N; j++) crow[j] = q_add(crow[j], q_mul(a, brow[j]));
    }
  }
  return C;
}

static double qm_fro2(const qmat *A) {
  double s = 0.0;
  for (size_t t = 0; t < (size_t)A->r * A->c; t++) s += q_abs2(A->d[t]);
  return s;
}
static double qm_fro(const qmat *A) { return sqrt(qm_fro2(A)); }
static double qm_diff_fro(const qmat *A, const qmat *B) {
  double s = 0.0;
  for (size_t t = 0; t < (size_t)A->r * A->c; t++) s += q_abs2(q_sub(A->d[t], B->d[t]));
  return sqrt(s);
}
/* ||A||_1: largest column sum of entry moduli. */
static double qm_norm1(const qmat *A) {
  double best = 0.0;
  for (int j = 0; j < A->c; j++) {
    double s = 0.0;
    for (int i = 0; i < A->r; i++) s += q_abs(*qm_at(A, i, j));
    if (s > best) best = s;
  }
  return best;
}
/* ||A||_inf: largest row sum of entry moduli. */
static double qm_norminf(const qmat *A) {
  double best = 0.0;
  for (int i = 0; i < A->r; i++) {
    double s = 0.0;
    for (int j = 0; j < A->c; j++) s += q_abs(*qm_at(A, i, j));
    if (s > best) best = s;
  }
  return best;
}

static qmat qm_from(int r, int c, const double *p) {
  qmat M = qm_new(r, c);
  memcpy(M.d, p, sizeof(quat) * (size_t)r * c);
  return M;
}
static void qm_to(const qmat *M, double *p) { memcpy(p, M->d, sizeof(quat) * (size_t)M->r * M->c); }

/* -------- constants of the residual polynomials ------------------------- */

/* QSAI (Sec. 3.2): beta1 + beta2 = 1, beta1 beta2 = -1. */
static double beta1(void) { return (1.0 + sqrt(5.0)) / 2.0; }
static double beta2(void) { return (1.0 - sqrt(5.0)) / 2.0; }
/* QHPI19 (Sec. 3.3): coefficients of the factorized order-19 polynomial. */
typedef struct { double a1, a2, a3, b1, b2, c1, c2, d1, d2, d3, e1, e2; } hpi19_coef;
static hpi19_coef hpi19_coefficients(void) {
  const double s93 = sqrt(93.0);
  hpi19_coef k;
  k.a1 = 5.0 / 496.0 * (31.0 + s93);
  k.a2 = (3.0 + s93) / 8.0;
  k.a3 = 0.5;
  k.b1 = -5.0 / 496.0 * (s93 - 31.0);
  k.b2 = (3.0 - s93) / 8.0;
  k.c1 = 3.0 / 8.0;
  k.c2 = 321.0 / 1984.0;
  k.d1 = 0.25 * (sqrt(27.0 - 2.0 * s93) + 1.0);
  k.d2 = 0.25 * (1.0 - sqrt(27.0 - 2.0 * s93));
  k.d3 = (5.0 * s93 - 93.0) / 496.0;
  k.e1 = (-93.0 - 5.0 * s93) / 496.0;
  k.e2 = -s93 / 4.0;
  if (g_mutation == 3) k.c2 = 321.0 / 1985.0;
  return k;
}

/* -------- one iteration of each method ---------------------------------- */

enum { M_NS = 0, M_QSAI = 1, M_QRAPID = 2, M_QHPI19 = 3, M_QHPIM = 4 };

/* Newton-Schulz (Sec. 1): X_{j+1} = X_j (2I - A X_j); left form (2I - X A) X. */
static qmat step_ns(const qmat *A, const qmat *X, int left) {
  if (!left) {
    qmat P = qm_mul(A, X);
    qmat T = qm_comb(-1.0, &P, 0.0, NULL, 2.0);
    qmat Xn = qm_mul(X, &T);
    qm_free(&P); qm_free(&T);
    return Xn;
  }
  qmat P = qm_mul(X, A);
  qmat T = qm_comb(-1.0, &P, 0.0, NULL, 2.0);
  qmat Xn = qm_mul(&T, X);
  qm_free(&P); qm_free(&T);
  return Xn;
}

/* QSAI (Alg. 2): R = I - AX; Q = (I + b1 R^2 + R^4)(I + b2 R^2 + R^4);
 * X_{j+1} = X (I + R) Q.  Left form: R = I - XA, X_{j+1} = Q (I + R) X. */
static qmat step_qsai(const qmat *A, const qmat *X, int left) {
  qmat P = left ? qm_mul(X, A) : qm_mul(A, X);
  qmat R = qm_comb(-1.0, &P, 0.0, NULL, 1.0);
  qmat R2 = qm_mul(&R, &R);
  qmat R4 = qm_mul(&R2, &R2);
  qmat F1 = qm_comb(beta1(), &R2, 1.0, &R4, 1.0);
  qmat F2 = qm_comb(beta2(), &R2, 1.0, &R4, 1.0);
  qmat Q = qm_mul(&F1, &F2);
  qmat IpR = qm_comb(1.0, &R, 0.0, NULL, 1.0);
  qmat T, Xn;
  if (!left) { T = qm_mul(X, &IpR); Xn = qm_mul(&T, &Q); }
  else { T = qm_mul(&IpR, X); Xn = qm_mul(&Q, &T); }
  qm_free(&P); qm_free(&R); qm_free(&R2); qm_free(&R4); qm_free(&F1); qm_free(&F2);
  qm_free(&Q); qm_free(&IpR); qm_free(&T);
  return Xn;
}

/* QHPI19 (Alg. 3): R, R^2, R^4; U = (I + d1 R^2 + R^4)(I + d2 R^2 + R^4);
 * V = U + d3 R^2; W = U + e1 R^2 + e2 R^4; Gamma = V W + c1 R^2 + c2 R^4;
 * X_{j+1} = X (I + (R + R^2) Gamma).  Left form: R = I - XA and the
 * polynomial multiplies X from the left. */
static qmat step_qhpi19(const qmat *A, const qmat *X, int left) {
  const hpi19_coef k = hpi19_coefficients();
  qmat P = left ? qm_mul(X, A) : qm_mul(A, X);
  qmat R = qm_comb(-1.0, &P, 0.0, NULL, 1.0);
  qmat R2 = qm_mul(&R, &R);
  qmat R4 = qm_mul(&R2, &R2);
  qmat F1 = qm_comb(k.d1, &R2, 1.0, &R4, 1.0);
  qmat F2 = qm_comb(k.d2, &R2, 1.0, &R4, 1.0);
  qmat U = qm_mul(&F1, &F2);
  qmat d3R2 = qm_comb(k.d3, &R2, 0.0, NULL, 0.0);
  qmat V = qm_add(&U, &d3R2);
  qmat eR = qm_comb(k.e1, &R2, k.e2, &R4, 0.0);
  qmat W = qm_add(&U, &eR);
  qmat VW = qm_mul(&V, &W);
  qmat cR = qm_comb(k.c1, &R2, k.c2, &R4, 0.0);
  qmat G = qm_add(&VW, &cR);
  qmat S = qm_add(&R, &R2);
  qmat SG = qm_mul(&S, &G);
  qmat T = qm_comb(1.0, &SG, 0.0, NULL, 1.0);
  qmat Xn = left ? qm_mul(&T, X) : qm_mul(X, &T);
  qm_free(&P); qm_free(&R); qm_free(&R2); qm_free(&R4); qm_free(&F1); qm_free(&F2);
  qm_free(&U); qm_free(&d3R2); qm_free(&V); qm_free(&eR); qm_free(&W); qm_free(&VW);
  qm_free(&cR); qm_free(&G); qm_free(&S); qm_free(&SG); qm_free(&T);
  return Xn;
}

/* The correction step of Alg. 1:  W + Y (I - A W)  in the right form;
 * the left form is  W + (I - W A) Y. */
static qmat rapid_correct(const qmat *A, const qmat *Wm, const qmat *Ym, int left) {
  if (!left) {
    qmat AW = qm_mul(A, Wm);
    qmat E = qm_comb(-1.0, &AW, 0.0, NULL, 1.0);
    qmat YE = qm_mul(Ym, &E);
    qmat Z = qm_add(Wm, &YE);
    qm_free(&AW); qm_free(&E); qm_free(&YE);
    return Z;
  }
  qmat WA = qm_mul(Wm, A);
  qmat E = qm_comb(-1.0, &WA, 0.0, NULL, 1.0);
  qmat EY = qm_mul(&E, Ym);
  qmat Z = qm_add(Wm, &EY);
  qm_free(&WA); qm_free(&E); qm_free(&EY);
  return Z;
}

/* QRAPID (Alg. 1) with step parameter N:
 *   P = A X;  U = 1/4 X (13I - P(15I - P(7I - P)));  V = U + X (I - A U);
 *   Y0 = U, W0 = V;  for l = 1..N: Z_l = W_{l-1} + Y_{l-1}(I - A W_{l-1}),
 *   Y_l = W_{l-1}, W_l = Z_l;  (N = 0: Z = V)
 *   X_{j+1} = Z_N + X (I - A Z_N). */
static qmat step_qrapid(const qmat *A, const qmat *X, int N, int left) {
  qmat P = left ? qm_mul(X, A) : qm_mul(A, X);
  qmat T = qm_comb(-1.0, &P, 0.0, NULL, 7.0);
  qmat PT = qm_mul(&P, &T);
  qmat T2 = qm_comb(-1.0, &PT, 0.0, NULL, 15.0);
  qmat PT2 = qm_mul(&P, &T2);
  qmat T3 = qm_comb(-1.0, &PT2, 0.0, NULL, 13.0);
  qmat XT3 = left ? qm_mul(&T3, X) : qm_mul(X, &T3);
  qmat U = qm_comb(0.25, &XT3, 0.0, NULL, 0.0);
  qmat V = rapid_correct(A, &U, X, left);
  qmat Z;
  if (N == 0) {
    Z = qm_copy(&V);
  } else {
    qmat Y = qm_copy(&U), Wm = qm_copy(&V);
    for (int l = 1; l <= N; l++) {
      qmat Zl = rapid_correct(A, &Wm, &Y, left);
      qm_free(&Y);
      Y = Wm;
      Wm = Zl;
    }
    Z = Wm;
    qm_free(&Y);
  }
  qmat Xn = rapid_correct(A, &Z, X, left);
  qm_free(&P); qm_free(&T); qm_free(&PT); qm_free(&T2); qm_free(&PT2); qm_free(&T3);
  qm_free(&XT3); qm_free(&U); qm_free(&V); qm_free(&Z);
  return Xn;
}

/* Unfactorized hyperpower iteration of order k (Definition 1; the
 * QHONSchultz(k) solvers of Example 3):  R = I - A X,
 *   X_{j+1} = X (I + R + R^2 + ... + R^{k-1}).
 * The powers are formed one after another (R^i = R^{i-1} R) and added in
 * increasing order: k - 2 products for the powers, so k per iteration with
 * the residual and the update.  Left form: R = I - X A and the sum
 * multiplies X from the left.  k = 1 (the empty sum I) leaves X unchanged. */
static qmat step_qhpim(const qmat *A, const qmat *X, int k, int left) {
  if (g_mutation == 4) k -= 1; /* planted mistake: the highest power is dropped */
  qmat P = left ? qm_mul(X, A) : qm_mul(A, X);
  qmat R = qm_comb(-1.0, &P, 0.0, NULL, 1.0);
  qmat Sum = qm_comb(0.0, &R, 0.0, NULL, 1.0); /* R^0 = I */
  qmat Pw = qm_comb(0.0, &R, 0.0, NULL, 1.0);
  for (int i = 1; i < k; i++) {
    qmat next = i == 1 ? qm_copy(&R) : qm_mul(&Pw, &R);
    qm_free(&Pw);
    Pw = next;
    qmat acc = qm_add(&Sum, &Pw);
    qm_free(&Sum);
    Sum = acc;
  }
  qmat Xn = left ? qm_mul(&Sum, X) : qm_mul(X, &Sum);
  qm_free(&P); qm_free(&R); qm_free(&Sum); qm_free(&Pw);
  return Xn;
}

/* N: QRAPID's step parameter, or the order k of QHPIM. */
static qmat method_step(const qmat *A, const qmat *X, int method, int N, int left) {
  switch (method) {
    case M_NS: return step_ns(A, X, left);
    case M_QSAI: return step_qsai(A, X, left);
    case M_QRAPID: return step_qrapid(A, X, N, left);
    case M_QHPIM: return step_qhpim(A, X, N, left);
    default: return step_qhpi19(A, X, left);
  }
}

/* -------- initialisation: alpha rules (Thm. 1, Algs. 1-3, Sec. 4) -------- */

enum { ALPHA_SAFE = 0, ALPHA_SPECTRAL = 1, ALPHA_FRO = 2, ALPHA_USER = 3 };

/* sigma_max(A)^2 by power iteration on A^H A (a Hermitian positive
 * semidefinite quaternion matrix, whose eigenvalues are real).  The start
 * vector is a fixed pseudo-random quaternion vector. */
static double sigma_max2(const qmat *A) {
  const int n = A->c;
  qmat v = qm_new(n, 1);
  uint64_t st = 0x2545F4914F6CDD1DULL;
  for (int i = 0; i < n; i++) {
    double c[4];
    for (int t = 0; t < 4; t++) {
      st ^= st << 13; st ^= st >> 7; st ^= st << 17;
      c[t] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    quat q = {c[0], c[1], c[2], c[3]};
    *qm_at(&v, i, 0) = q;
  }
  qmat AH = qm_adjoint(A);
  double lam = 0.0;
  for (int it = 0; it < 5000; it++) {
    double nv = qm_fro(&v);
    for (int i = 0; i < n; i++) *qm_at(&v, i, 0) = q_scale(1.0 / nv, *qm_at(&v, i, 0));
    qmat Av = qm_mul(A, &v);
    qmat w = qm_mul(&AH, &Av);
    g_gemm_count -= 2; /* matrix-vector products are not counted as GEMMs */
    double lam_new = qm_fro(&w); /* ||A^H A v|| with ||v|| = 1 */
    qm_free(&Av);
    qm_free(&v);
    v = w;
    if (it > 10 && fabs(lam_new - lam) <= 1e-14 * lam_new) { lam = lam_new; break; }
    lam = lam_new;
  }
  qm_free(&v); qm_free(&AH);
  return lam;
}

static double choose_alpha(const qmat *A, int mode, double user) {
  switch (mode) {
    case ALPHA_SAFE: return 1.0 / (qm_norm1(A) * qm_norminf(A));
    case ALPHA_SPECTRAL: return 1.0 / sigma_max2(A);
    case ALPHA_FRO: return 1.0 / qm_fro2(A);
    default: return user;
  }
}

/* -------- Penrose residuals E1..E4 (Sec. 4, eq. for E1-E4) --------------- */

static void penrose(const qmat *A, const qmat *X, double E[4], double Erel[4]) {
  qmat AX = qm_mul(A, X);
  qmat XA = qm_mul(X, A);
  qmat AXA = qm_mul(&AX, A);
  qmat XAX = qm_mul(&XA, X);
  qmat AXH = qm_adjoint(&AX);
  qmat XAH = qm_adjoint(&XA);
  E[0] = qm_diff_fro(&AXA, A);
  E[1] = qm_diff_fro(&XAX, X);
  E[2] = qm_diff_fro(&AXH, &AX);
  E[3] = qm_diff_fro(&XAH, &XA);
  const double nrm[4] = {qm_fro(A), qm_fro(X), qm_fro(&AX), qm_fro(&XA)};
  for (int t = 0; t < 4; t++) Erel[t] = nrm[t] > 0 ? E[t] / nrm[t] : E[t];
  qm_free(&AX); qm_free(&XA); qm_free(&AXA); qm_free(&XAX); qm_free(&AXH); qm_free(&XAH);
}

/* ======================= exported C ABI (tests only) ===================== */

typedef struct {
  int status;      /* 0 converged, 1 plateau, 2 not converged, 3 diverged */
  int iters;       /* X-updates kept in the returned X */
  double alpha;
  double delta;    /* last ||X_{j+1} - X_j||_F */
  double delta_rel;
  double E[4];
  double E_rel[4];
  long long gemms; /* quaternion GEMMs spent inside the iteration loop */
} qo_result;

enum { STOP_PAPER_ABS = 0, STOP_REL_PLATEAU = 1 };

void qo_qmul(const double *p, const double *q, double *r) {
  quat a = {p[0], p[1], p[2], p[3]}, b = {q[0], q[1], q[2], q[3]};
  quat c = q_mul(a, b);
  r[0] = c.s; r[1] = c.x; r[2] = c.y; r[3] = c.z;
}

void qo_matmul(int m, int k, int n, const double *A, const double *B, double *C) {
  qmat a = qm_from(m, k, A), b = qm_from(k, n, B);
  qmat c = qm_mul(&a, &b);
  qm_to(&c, C);
  qm_free(&a); qm_free(&b); qm_free(&c);
}

void qo_adjoint(int m, int n, const double *A, double *AH) {
  qmat a = qm_from(m, n, A);
  qmat h = qm_adjoint(&a);
  qm_to(&h, AH);
  qm_free(&a); qm_free(&h);
}

void qo_norms(int m, int n, const double *A, double *out3) {
  qmat a = qm_from(m, n, A);
  out3[0] = qm_norm1(&a); out3[1] = qm_norminf(&a); out3[2] = qm_fro(&a);
  qm_free(&a);
}

double qo_sigma_max(int m, int n, const double *A) {
  qmat a = qm_from(m, n, A);
  double s = sqrt(sigma_max2(&a));
  qm_free(&a);
  return s;
}

double qo_alpha(int m, int n, const double *A, int mode, double user) {
  qmat a = qm_from(m, n, A);
  double al = choose_alpha(&a, mode, user);
  qm_free(&a);
  return al;
}

void qo_init_x0(int m, int n, const double *A, double alpha, double *X0) {
  qmat a = qm_from(m, n, A);
  qmat h = qm_adjoint(&a);
  for (size_t t = 0; t < (size_t)m * n; t++) h.d[t] = q_scale(alpha, h.d[t]);
  qm_to(&h, X0);
  qm_free(&a); qm_free(&h);
}

void qo_step(int m, int n, const double *A, const double *X, int method, int N, int left, double *Xn) {
  qmat a = qm_from(m, n, A), x = qm_from(n, m, X);
  qmat y = method_step(&a, &x, method, N, left);
  qm_to(&y, Xn);
  qm_free(&a); qm_free(&x); qm_free(&y);
}

void qo_penrose(int m, int n, const double *A, const double *X, double *E4, double *Erel4) {
  qmat a = qm_from(m, n, A), x = qm_from(n, m, X);
  penrose(&a, &x, E4, Erel4);
  qm_free(&a); qm_free(&x);
}

/* Full solve.  X (n x m) receives the returned iterate.  If x0 != NULL it is
 * the starting iterate (warm start) and alpha is not used.  delta_trace, if
 * not NULL, receives ||X_{j+1}-X_j||_F for every computed step (max_iter). */
void qo_solve(int m, int n, const double *A, int method, int N, int alpha_mode,
              double alpha_user, int stop_rule, double tol, int max_iter, int left,
              const double *x0, double *X, double *delta_trace, qo_result *res) {
  qmat a = qm_from(m, n, A);
  memset(res, 0, sizeof(*res));
  qmat x;
  if (x0) {
    x = qm_from(n, m, x0);
    res->alpha = 0.0;
  } else {
    res->alpha = choose_alpha(&a, alpha_mode, alpha_user);
    x = qm_adjoint(&a);
    for (size_t t = 0; t < (size_t)m * n; t++) x.d[t] = q_scale(res->alpha, x.d[t]);
  }
  long long g0 = g_gemm_count;
  double prev_rel = INFINITY;
  res->status = 2;
  res->iters = max_iter;
  for (int j = 0; j < max_iter; j++) {
    qmat xn = method_step(&a, &x, method, N, left);
    const double d = qm_diff_fro(&xn, &x);
    const double nx = qm_fro(&xn);
    if (delta_trace) delta_trace[j] = d;
    if (!isfinite(d) || !isfinite(nx)) {
      res->status = 3; res->iters = j;
      qm_free(&xn);
      break;
    }
    const double drel = nx > 0 ? d / nx : d;
    res->delta = d; res->delta_rel = drel;
    if (stop_rule == STOP_PAPER_ABS) {
      qm_free(&x); x = xn;
      if (d < tol) { res->status = 0; res->iters = j + 1; break; }
    } else {
      if (drel <= tol) { qm_free(&x); x = xn; res->status = 0; res->iters = j + 1; break; }
      if (j > 0 && prev_rel < 1e-3 && drel >= prev_rel) {
        /* no progress: keep X_j, the iterate before the non-decreasing step */
        res->status = 1; res->iters = j;
        qm_free(&xn);
        break;
      }
      qm_free(&x); x = xn;
      prev_rel = drel;
    }
  }
  res->gemms = g_gemm_count - g0;
  penrose(&a, &x, res->E, res->E_rel);
  qm_to(&x, X);
  qm_free(&a); qm_free(&x);
}

/* A^dagger = V Sigma^dagger U^H from a singular value decomposition
 * A = U diag(sigma) V^H (Sec. 2, QSVD-based pseudoinverse); U is m x r,
 * V is n x r, sigma has r entries (zeros are not inverted). */
void qo_pinv_from_svd(int m, int n, int r, const double *U, const double *sigma,
                      const double *V, double *X) {
  qmat u = qm_from(m, r, U), v = qm_from(n, r, V);
  qmat uh = qm_adjoint(&u);
  qmat vs = qm_copy(&v);
  for (int i = 0; i < n; i++)
    for (int l = 0; l < r; l++)
      *qm_at(&vs, i, l) = q_scale(sigma[l] != 0.0 ? 1.0 / sigma[l] : 0.0, *qm_at(&v, i, l));
  qmat x = qm_mul(&vs, &uh);
  qm_to(&x, X);
  qm_free(&u); qm_free(&v); qm_free(&uh); qm_free(&vs); qm_free(&x);
}

void qo_constants(double *out14) {
  const hpi19_coef k = hpi19_coefficients();
  const double v[14] = {beta1(), beta2(), k.a1, k.a2, k.a3, k.b1, k.b2,
                        k.c1, k.c2, k.d1, k.d2, k.d3, k.e1, k.e2};
  memcpy(out14, v, sizeof(v));
}

long long qo_gemm_count(void) { return g_gemm_count; }
