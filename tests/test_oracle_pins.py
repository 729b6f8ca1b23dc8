"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code: the Hamilton identities,
the complex representation (a *-homomorphism, Sec. 2), the worked Example 1
(Section 4, Table 1), the residual recurrences of Theorems 2, 4 and 6, the
coefficient identities of the factorized polynomials (Sec. 3.2-3.3), closed
forms of the pseudoinverse (Def. 2.1, Sec. 2), LAPACK's pseudoinverse of the
complex representation, Proposition 1's invariants and the per-iteration
product counts of Sec. 3.4.  A final test plants known mistakes in the
oracle and checks that these pins catch each of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_01464_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example1.txt")
def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def load_example1():
    A = np.zeros((4, 3, 3))
    P = np.zeros((4, 3, 3))
    vals = {}
    for line in open(GOLDEN):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] in ("A", "P"):
            i, j = int(t[1]) - 1, int(t[2]) - 1
            (A if t[0] == "A" else P)[:, i, j] = [float(v) for v in t[3:7]]
        elif t[0] == "iters":
            vals[("iters", t[1])] = int(t[2])
        else:
            vals[t[0]] = float(t[1])
    return A, P, vals


# ------------------------------------------------------------ pin checks

def check_hamilton():
    one, i, j, k = np.eye(4)
    for u in (i, j, k):
        assert np.allclose(oracle.qmul(u, u), -one)
    assert np.allclose(oracle.qmul(oracle.qmul(i, j), k), -one)
    assert np.allclose(oracle.qmul(i, j), k) and np.allclose(oracle.qmul(j, i), -k)
    assert np.allclose(oracle.qmul(j, k), i) and np.allclose(oracle.qmul(k, j), -i)
    assert np.allclose(oracle.qmul(k, i), j) and np.allclose(oracle.qmul(i, k), -j)
    rng = np.random.default_rng(7)
    for _ in range(20):
        p, q = rng.standard_normal(4), rng.standard_normal(4)
        pq = oracle.qmul(p, q)
        assert math.isclose(np.linalg.norm(pq), np.linalg.norm(p) * np.linalg.norm(q), rel_tol=1e-14)


def check_matmul_chi():
    for (m, k, n, seed) in [(5, 3, 4, 1), (7, 7, 7, 2), (1, 9, 2, 3), (16, 11, 13, 4)]:
        A = I.gaussian_quaternion(m, k, seed)
        B = I.gaussian_quaternion(k, n, seed + 100)
        C = oracle.matmul(A, B)
        assert np.allclose(I.chi(C), I.chi(A) @ I.chi(B), rtol=1e-13, atol=1e-12)


def check_adjoint_chi():
    A = I.gaussian_quaternion(6, 4, 9)
    H = oracle.adjoint(A)
    assert np.array_equal(I.chi(H), I.chi(A).conj().T)


def check_example1(method="qsai", N=1):
    A, P, vals = load_example1()
    alpha = oracle.alpha(A, "spectral")
    assert abs(alpha - vals["alpha"]) <= 0.5e-9, alpha
    X, info = oracle.solve(A, method, tol=1e-10, alpha_mode="spectral", stop="paper_abs",
                           N=N, max_iter=100)
    assert info["status"] == "converged"
    assert np.max(np.abs(X - P)) <= 0.5e-4 + 1e-12, np.max(np.abs(X - P))
    assert max(info["E"]) <= vals["Emax"], info["E"]
    assert info["iters"] == vals[("iters", method)], info["iters"]
    return X


def check_coefficients():
    c = oracle.constants()
    P = np.polynomial.polynomial
    # QSAI: (1 + x)(1 + b1 x^2 + x^4)(1 + b2 x^2 + x^4) = sum_{k<=9} x^k
    qsai = P.polymul(P.polymul([1, 1], [1, 0, c["beta1"], 0, 1]), [1, 0, c["beta2"], 0, 1])
    assert np.allclose(qsai, np.ones(10), atol=1e-14)
    # QHPI19, in y = x^2: G1 = (1 + d1 y + y^2)(1 + d2 y + y^2) + d3 y,
    # G2 = same + e1 y + e2 y^2, G1 = 1 + a1 y + a2 y^2 + a3 y^3 + y^4,
    # G2 = 1 + b1 y + b2 y^2 + a3 y^3 + y^4, G1 G2 + c1 y + c2 y^2 = sum_{k<=8} y^k.
    quad = P.polymul([1, c["d1"], 1], [1, c["d2"], 1])
    g1 = P.polyadd(quad, [0, c["d3"]])
    g2 = P.polyadd(quad, [0, c["e1"], c["e2"]])
    assert np.allclose(g1, [1, c["a1"], c["a2"], c["a3"], 1], atol=1e-14)
    assert np.allclose(g2, [1, c["b1"], c["b2"], c["a3"], 1], atol=1e-14)
    gam = P.polyadd(P.polymul(g1, g2), [0, c["c1"], c["c2"]])
    assert np.allclose(gam, np.ones(9), atol=1e-13)
    # X_{j+1} = X (I + (R + R^2) Gamma(R^2)) is X times sum_{k<=18} R^k
    full = P.polyadd([1], P.polymul([0, 1, 1], np.ravel(np.column_stack([gam, np.zeros(9)]))[:17]))
    assert np.allclose(full, np.ones(19), atol=1e-12)


def fib(k):
    """a_k = (phi^k - (1-phi)^k)/sqrt(5), extended to negative k."""
    if k < 0:  # a_{-k} = (-1)^(k+1) a_k
        return fib(-k) if (-k) % 2 == 1 else -fib(-k)
    a, b = 0, 1
    for _ in range(k):
        a, b = b, a + b
    return a


def residual_map(method, r, N=5):
    """Scalar residual recurrence r_{j+1} = f(r_j) stated by the paper:
    Thm. 6 (QHPI19: r^19), Thm. 4 (QSAI: r^10), Sec. 3 (NS, k = 2: r^2),
    Thm. 2 for QRAPID: N = 0: 3/4 r^5 + 1/4 r^6; N = 1: (9 r^8 + 6 r^9 + r^10)/16;
    N >= 3: 4^(-a_{N+2}) (3 + r)^a_{N+2} r^nu_N with nu_N = 11 a_{N-1} + 7 a_{N-2} + 1.
    N = 2 (order 12 in the paper, no closed form printed) uses the N >= 3
    formula, which at N = 2 gives order 12.  QHPIM of order k (Definition 1,
    N = k): I - (I - R)(I + R + ... + R^(k-1)) = R^k."""
    if method == "qhpim":
        return r ** N
    if method == "qhpi19":
        return r ** 19
    if method == "qsai":
        return r ** 10
    if method == "ns":
        return r ** 2
    if N == 0:
        return Fraction(3, 4) * r ** 5 + Fraction(1, 4) * r ** 6
    if N == 1:
        return (9 * r ** 8 + 6 * r ** 9 + r ** 10) / 16
    a = fib(N + 2)
    nu = 11 * fib(N - 1) + 7 * fib(N - 2) + 1
    return (3 + r) ** a * r ** nu / Fraction(4) ** a


def check_diagonal_recurrence(method, N=5, side="right", tall=0):
    d = np.array([1.0, 0.5, 0.3, 0.1, 2.0, 0.05])
    n = d.size
    A = np.zeros((4, n + tall, n))
    A[0, np.arange(n), np.arange(n)] = d
    alpha = 0.2
    X = oracle.init_x0(A, alpha)
    for _ in range(3):
        r0 = [Fraction(1) - Fraction(float(d[i])) * Fraction(float(X[0, i, i])) for i in range(n)]
        X = oracle.step(A, X, method, N=N, side=side, order=N)
        # off-diagonal entries and imaginary planes stay exactly zero
        off = X.copy()
        off[0, np.arange(n), np.arange(n)] = 0
        assert np.max(np.abs(off)) == 0.0
        for i in range(n):
            r1 = 1.0 - d[i] * X[0, i, i]
            want = float(residual_map(method, r0[i], N))
            assert abs(r1 - want) <= 2e-15 + 1e-14 * abs(want), (method, N, i, r1, want)


def chi_pow(C, k):
    return np.linalg.matrix_power(C, k)


def check_matrix_recurrence(method, N=5, side="right", seed=11, shape=(9, 6)):
    m, n = shape
    A = I.gaussian_quaternion(m, n, seed)
    X0 = oracle.init_x0(A, oracle.alpha(A, "safe"))
    X1 = oracle.step(A, X0, method, N=N, side=side, order=N)
    cA, c0, c1 = I.chi(A), I.chi(X0), I.chi(X1)
    if side == "right":
        R0 = np.eye(2 * m) - cA @ c0
        R1 = np.eye(2 * m) - cA @ c1
    else:
        R0 = np.eye(2 * n) - c0 @ cA
        R1 = np.eye(2 * n) - c1 @ cA
    Id = np.eye(R0.shape[0])
    if method == "qhpim":  # Definition 1: R_{j+1} = R_j^k
        want = chi_pow(R0, N)
    elif method in ("qhpi19", "qsai", "ns"):
        want = chi_pow(R0, {"qhpi19": 19, "qsai": 10, "ns": 2}[method])
    else:
        a = fib(N + 2)
        nu = 11 * fib(N - 1) + 7 * fib(N - 2) + 1
        want = chi_pow(3 * Id + R0, a) @ chi_pow(R0, nu) / 4.0 ** a
    assert np.linalg.norm(R1 - want) <= 1e-12 * max(1.0, np.linalg.norm(R0)), \
        (method, N, side, np.linalg.norm(R1 - want))


# ------------------------------------------------------------------ tests

def test_hamilton_identities():
    check_hamilton()


def test_conjugation_is_anti_automorphism():
    rng = np.random.default_rng(3)
    for _ in range(10):
        p, q = rng.standard_normal((2, 4, 1, 1))
        lhs = oracle.adjoint(oracle.matmul(p, q))
        rhs = oracle.matmul(oracle.adjoint(q), oracle.adjoint(p))
        assert np.allclose(lhs, rhs, atol=1e-15)


def test_matmul_equals_complex_representation_product():
    check_matmul_chi()


def test_adjoint_equals_complex_conjugate_transpose():
    check_adjoint_chi()


def test_norms_and_sigma_max():
    A = I.gaussian_quaternion(13, 8, 5)
    n1, ninf, nf = oracle.norms(A)
    C = I.chi(A)
    # ||A^C||_F^2 = 2 ||A||_F^2; sigma(A) = sigma(A^C) (each doubled)
    assert math.isclose(np.linalg.norm(C) ** 2, 2 * nf ** 2, rel_tol=1e-13)
    smax = np.linalg.svd(C, compute_uv=False)[0]
    assert math.isclose(oracle.sigma_max(A), smax, rel_tol=1e-10)
    # Schur test with entry moduli: sigma_max^2 <= ||A||_1 ||A||_inf, so the
    # safe scaling lies inside the convergence region of Thm. 1.
    assert smax ** 2 <= n1 * ninf
    assert oracle.alpha(A, "safe") < 2.0 / smax ** 2
    mod = np.sqrt((A ** 2).sum(axis=0))
    assert math.isclose(n1, mod.sum(axis=0).max(), rel_tol=1e-14)
    assert math.isclose(ninf, mod.sum(axis=1).max(), rel_tol=1e-14)


@pytest.mark.parametrize("method,N", [("qsai", 5), ("qhpi19", 5), ("qrapid", 1), ("qrapid", 2)])
def test_example1_worked_example(method, N):
    X = check_example1(method, N)
    # row 3 of A is twice row 2, so A^dagger(:,3) = 2 A^dagger(:,2)
    assert np.allclose(X[:, :, 2], 2 * X[:, :, 1], atol=1e-13)


def test_coefficient_identities():
    check_coefficients()


@pytest.mark.parametrize("method,N", [("ns", 0), ("qsai", 0), ("qhpi19", 0)]
                         + [("qrapid", N) for N in range(6)]
                         + [("qhpim", k) for k in (1, 2, 3, 5, 10, 19)])
@pytest.mark.parametrize("side,tall", [("right", 0), ("left", 0), ("right", 3)])
def test_diagonal_closed_form_recurrence(method, N, side, tall):
    check_diagonal_recurrence(method, N, side, tall)


@pytest.mark.parametrize("method,N", [("ns", 0), ("qsai", 0), ("qhpi19", 0)]
                         + [("qrapid", N) for N in (0, 1, 3, 5)]
                         + [("qhpim", k) for k in (2, 3, 7, 10, 19)])
@pytest.mark.parametrize("side", ["right", "left"])
def test_matrix_residual_recurrence(method, N, side):
    check_matrix_recurrence(method, N, side)


@pytest.mark.parametrize("k,factorized", [(2, "ns"), (10, "qsai"), (19, "qhpi19")])
@pytest.mark.parametrize("side", ["right", "left"])
def test_unfactorized_equals_factorized_polynomial(k, factorized, side):
    # The factorized methods evaluate the same polynomial sum_{i<k} R^i in
    # fewer products (Sec. 3.2, 3.3, Example 3): Newton-Schulz is k = 2,
    # QSAI k = 10, QHPI19 k = 19.  Separate code paths, equal iterates.
    A = I.gaussian_quaternion(10, 7, 41)
    X = Y = oracle.init_x0(A, oracle.alpha(A, "safe"))
    for _ in range(3):
        X = oracle.step(A, X, "qhpim", side=side, order=k)
        Y = oracle.step(A, Y, factorized, side=side)
        assert rel(X, Y) <= 1e-13, (k, factorized, rel(X, Y))


def test_unfactorized_order_one_is_identity_step():
    # k = 1: the sum is I, so X_{j+1} = X_j; the stop rule sees a zero step
    A = I.gaussian_quaternion(6, 5, 42)
    X0 = oracle.init_x0(A, oracle.alpha(A, "safe"))
    assert np.array_equal(oracle.step(A, X0, "qhpim", order=1), X0)
    X, info = oracle.solve(A, "qhpim", order=1, tol=1e-12, max_iter=5)
    assert info["status"] == "converged" and info["iters"] == 1 and info["delta"] == 0.0
    assert np.array_equal(X, X0)


@pytest.mark.parametrize("method", ["ns", "qsai", "qrapid", "qhpi19", "qhpim"])
def test_left_and_right_forms_agree(method):
    A = I.gaussian_quaternion(10, 7, 21)
    X = oracle.init_x0(A, oracle.alpha(A, "safe"))
    Y = X.copy()
    for _ in range(3):
        X = oracle.step(A, X, method, N=2, side="right", order=6)
        Y = oracle.step(A, Y, method, N=2, side="left", order=6)
        assert rel(X, Y) <= 1e-12


@pytest.mark.parametrize("method", ["ns", "qsai", "qrapid", "qhpi19", "qhpim"])
def test_gemm_counts_per_iteration(method):
    A = I.gaussian_quaternion(6, 5, 2)
    X = oracle.init_x0(A, oracle.alpha(A, "safe"))
    Ns = {"qrapid": [0, 1, 5], "qhpim": [2, 3, 10, 19]}.get(method, [0])
    for N in Ns:
        g0 = oracle.gemm_count()
        oracle.step(A, X, method, N=N, order=N)
        # QHPIM(k): residual, k - 2 powers, update (Example 3: O(k n^3) per step)
        want = {"ns": 2, "qsai": 6, "qhpi19": 7, "qhpim": N}.get(method, 8 + 2 * N)
        assert oracle.gemm_count() - g0 == want


@pytest.mark.parametrize("method", ["ns", "qsai", "qrapid", "qhpi19", "qhpim"])
@pytest.mark.parametrize("shape", [(12, 7), (7, 12)])
def test_full_rank_closed_forms(method, shape):
    m, n = shape
    A = I.gaussian_quaternion(m, n, 31)
    X, info = oracle.solve(A, method, tol=1e-14, max_iter=200, order=5)
    assert info["status"] in ("converged", "plateau")
    C = I.chi(A)
    if m > n:  # full column rank: (A^H A)^{-1} A^H
        want = np.linalg.solve(C.conj().T @ C, C.conj().T)
    else:      # full row rank: A^H (A A^H)^{-1}
        want = C.conj().T @ np.linalg.inv(C @ C.conj().T)
    assert rel(I.chi(X), want) <= 1e-12
    assert max(info["E_rel"]) <= 1e-13


def test_unitary_gives_adjoint():
    U = I.orthonormal_columns(10, 10, 4)
    X, info = oracle.solve(U, "qhpi19", tol=1e-14, alpha_mode="user", alpha_user=1.0)
    assert rel(X, oracle.adjoint(U)) <= 1e-14
    X1 = oracle.step(U, oracle.adjoint(U), "qhpi19")  # R0 = I - U U^H = 0
    assert rel(X1, oracle.adjoint(U)) <= 1e-14


def test_quaternion_diagonal_reciprocal():
    rng = np.random.default_rng(5)
    n = 6
    q = rng.standard_normal((4, n)) + np.array([[2.0], [0], [0], [0]])
    A = np.zeros((4, n, n))
    A[:, np.arange(n), np.arange(n)] = q
    X, info = oracle.solve(A, "qsai", tol=1e-15)
    inv = np.array([q[0], -q[1], -q[2], -q[3]]) / (q ** 2).sum(axis=0)
    want = np.zeros_like(A)
    want[:, np.arange(n), np.arange(n)] = inv
    assert rel(X, want) <= 1e-14


@pytest.mark.parametrize("method,tol_x", [("ns", 1e-10), ("qsai", 1e-10), ("qhpi19", 1e-10),
                                          ("qrapid", 1e-9), ("qhpim", 1e-10)])
@pytest.mark.parametrize("side", ["right", "left"])
def test_rank_deficient_matches_lapack_pinv(method, tol_x, side):
    A, QL, s, QR = I.rank_deficient(20, 14, 6, 1e-2, seed_l=8, seed_r=9)
    X, info = oracle.solve(A, method, tol=1e-13, side=side, max_iter=300)
    assert info["status"] in ("converged", "plateau"), info
    want = np.linalg.pinv(I.chi(A), rcond=1e-8)
    assert rel(I.chi(X), want) <= tol_x, rel(I.chi(X), want)
    # generator-known pseudoinverse V Sigma^+ U^H agrees with LAPACK
    assert rel(I.chi(oracle.pinv_from_svd(QL, s, QR)), want) <= 1e-12
    assert info["E_rel"][0] <= 1e-12


@pytest.mark.parametrize("method", ["ns", "qsai", "qrapid", "qhpi19", "qhpim"])
def test_proposition1_invariants(method):
    A, QL, s, QR = I.rank_deficient(11, 9, 5, 1e-1, seed_l=12, seed_r=13)
    C = I.chi(A)
    Ad = np.linalg.pinv(C, rcond=1e-10)
    X = oracle.init_x0(A, oracle.alpha(A, "safe"))
    for _ in range(4):
        X = oracle.step(A, X, method, N=1)
        cx = I.chi(X)
        AX, XA = C @ cx, cx @ C
        scale = np.linalg.norm(cx)
        assert np.linalg.norm(AX - AX.conj().T) <= 1e-13 * max(1, np.linalg.norm(AX))   # (c)
        assert np.linalg.norm(XA - XA.conj().T) <= 1e-13 * max(1, np.linalg.norm(XA))   # (d)
        assert np.linalg.norm(Ad @ C @ cx - cx) <= 1e-12 * scale                         # (a)
        assert np.linalg.norm(cx @ C @ Ad - cx) <= 1e-12 * scale                         # (b)


def test_convergence_order_measured():
    # scalar case: log r_{j+1} / log r_j equals the order for every method
    for method, p in [("ns", 2), ("qsai", 10), ("qhpi19", 19), ("qhpim", 7), ("qhpim", 12)]:
        A = np.zeros((4, 1, 1))
        A[0, 0, 0] = 1.0
        X = oracle.init_x0(A, 0.5)
        r0 = 1 - X[0, 0, 0]
        X = oracle.step(A, X, method, order=p)
        r1 = 1 - X[0, 0, 0]
        assert math.isclose(math.log(r1) / math.log(r0), p, rel_tol=1e-9)


def test_stop_rule_outcomes():
    A = I.gaussian_quaternion(8, 6, 17)
    X, info = oracle.solve(A, "ns", tol=1e-14, max_iter=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    smax = oracle.sigma_max(A)
    X, info = oracle.solve(A, "qhpi19", tol=1e-14, max_iter=50, alpha_mode="user",
                           alpha_user=3.0 / smax ** 2)
    assert info["status"] == "diverged"
    assert np.all(np.isfinite(X))
    X, info = oracle.solve(A, "qhpi19", tol=1e-10, stop="paper_abs", max_iter=50)
    assert info["status"] == "converged" and info["delta"] < 1e-10


def test_warm_start_resume_is_bitwise():
    A = I.gaussian_quaternion(9, 7, 23)
    Xa, ia = oracle.solve(A, "qsai", tol=1e-30, max_iter=4, stop="paper_abs")
    X2, _ = oracle.solve(A, "qsai", tol=1e-30, max_iter=2, stop="paper_abs")
    Xb, _ = oracle.solve(A, "qsai", tol=1e-30, max_iter=2, stop="paper_abs", x0=X2)
    assert np.array_equal(Xa, Xb)


@pytest.mark.parametrize("mutation,check", [
    (1, check_hamilton), (1, check_matmul_chi), (2, check_adjoint_chi),
    (2, lambda: check_example1("qsai", 1)), (3, check_coefficients),
    (3, lambda: check_matrix_recurrence("qhpi19")),
    (3, lambda: check_diagonal_recurrence("qhpi19")),
    (4, lambda: check_matrix_recurrence("qhpim", 5)),
    (4, lambda: check_diagonal_recurrence("qhpim", 7))])
def test_planted_mistakes_are_caught(mutation, check):
    oracle.set_mutation(mutation)
    try:
        with pytest.raises(AssertionError):
            check()
    finally:
        oracle.set_mutation(0)


@pytest.mark.parametrize("method", ["ns", "qsai", "qhpi19", "qhpim"])
def test_initialization_theorem_threshold(method):
    # Thm. 1: X_0 = alpha A^H converges iff rho(R_0) = max |1 - alpha sigma_i^2| < 1,
    # i.e. alpha < 2 / sigma_1^2 (sigma_1 from LAPACK on the complex representation)
    A = I.gaussian_quaternion(12, 9, 43)
    s1 = np.linalg.svd(I.chi(A), compute_uv=False)[0]
    _, below = oracle.solve(A, method, tol=1e-13, max_iter=400, alpha_mode="user", alpha_user=1.9 / s1 ** 2,
                            order=5)
    assert below["status"] in ("converged", "plateau") and max(below["E_rel"]) <= 1e-12, below
    _, above = oracle.solve(A, method, tol=1e-13, max_iter=400, alpha_mode="user", alpha_user=2.1 / s1 ** 2,
                            order=5)
    assert above["status"] == "diverged", above
