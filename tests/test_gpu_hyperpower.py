"""GPU parity of the unfactorized hyperpower iteration QHPIM(k) (Definition 1;
the QHONSchultz(k) solvers of Example 3) against the FP64 oracle, which
evaluates the sum I + R + ... + R^(k-1) from its powers while the CUDA path
uses Horner's rule.

Tolerances (relative Frobenius error of X against the oracle's X), as for
the factorized methods: FP64 products, or mixed precision with the FP64
polish: 1e-10; tensor-core products only: 1e-5.  Batched (double-FP32):
1e-10 + 1e-12 k kappa_eff^2 against the exact pseudoinverse (null-space
noise grows by the order k per extra iteration)."""
import numpy as np
import pytest

import oracle
from paper_2605_01464_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01464_gb300 import build, qpinv
    build.build()
    return qpinv


@pytest.fixture()
def ctx(qp):
    c = qp.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("k", [2, 3, 10, 19])
@pytest.mark.parametrize("precision,tol_x", [("fp64", 1e-10), ("mixed", 1e-10), ("emu", 1e-10), ("tc", 1e-5)])
def test_qhpim_dense_gaussian_64x48(ctx, k, precision, tol_x):
    A = I.dense_gaussian(64, 48, seed=0)
    ctx.configure(precision=precision, hyper_order=k)
    X, info = ctx.solve(dev(A), "qhpim", tol=1e-12, max_iter=200)
    Xo, _ = oracle.solve(A, "qhpim", tol=1e-12, max_iter=200, order=k)
    assert info["status"] in ("converged", "plateau", "not_converged"), info
    assert rel(X.cpu().numpy(), Xo) <= tol_x, (rel(X.cpu().numpy(), Xo), info)
    if precision != "tc":
        assert info["E_rel"][0] <= 1e-12, info


@pytest.mark.parametrize("k", [4, 19])
@pytest.mark.parametrize("shape,side", [((40, 96), "auto"), ((96, 40), "auto"), ((96, 40), "right"),
                                        ((40, 96), "left"), ((70, 70), "left"), ((130, 130), "right")])
def test_qhpim_sides_and_shapes(ctx, k, shape, side):
    m, n = shape
    A = I.gaussian_quaternion(m, n, 7)
    ctx.configure(precision="mixed", side=side, hyper_order=k)
    X, info = ctx.solve(dev(A), "qhpim", tol=1e-13, max_iter=200)
    Xo, _ = oracle.solve(A, "qhpim", tol=1e-13, max_iter=200, order=k)
    assert rel(X.cpu().numpy(), Xo) <= 1e-10, info


@pytest.mark.parametrize("k,factorized", [(2, "ns"), (10, "qsai"), (19, "qhpi19")])
def test_qhpim_iterates_equal_factorized(ctx, k, factorized):
    """Three FP64 steps of QHPIM(k) and of the factorized method of the same
    polynomial agree to rounding, and each matches the oracle's steps."""
    A = I.gaussian_quaternion(50, 36, 19)
    ctx.configure(precision="fp64", hyper_order=k, stop="paper_abs", penrose=False)
    Xh, ih = ctx.solve(dev(A), "qhpim", tol=0.0, max_iter=3)
    Xf, _ = ctx.solve(dev(A), factorized, tol=0.0, max_iter=3)
    assert ih["iters"] == 3 and ih["status"] == "not_converged"
    Xo = oracle.init_x0(A, oracle.alpha(A, "safe"))
    for _ in range(3):
        Xo = oracle.step(A, Xo, "qhpim", side="left", order=k)
    assert rel(Xh.cpu().numpy(), Xo) <= 1e-12
    assert rel(Xh.cpu().numpy(), Xf.cpu().numpy()) <= 1e-12


def test_qhpim_gemm_counts_per_iteration(ctx):
    A = I.gaussian_quaternion(24, 24, 14)
    ctx.configure(precision="tc", penrose=False, stop="paper_abs")
    for k in (2, 3, 10, 19, 64):
        ctx.configure(hyper_order=k)
        _, info = ctx.solve(dev(A), "qhpim", tol=0.0, max_iter=3)
        assert info["gemms"] == 3 * k, (k, info)


@pytest.mark.parametrize("precision", ["emu", "fp64"])
def test_qhpim_rank_deficient(ctx, precision):
    """Rank-deficient input (kappa_eff = 1e3): X within 1e-8 of the exact
    V Sigma^+ U^H, as for the factorized methods."""
    A, QL, s, QR = I.rank_deficient(80, 60, 20, 1e-3, seed_l=4, seed_r=5)
    ctx.configure(precision=precision, hyper_order=7)
    X, info = ctx.solve(dev(A), "qhpim", tol=1e-13, max_iter=300)
    want = oracle.pinv_from_svd(QL, s, QR)
    assert info["status"] in ("converged", "plateau"), info
    assert rel(X.cpu().numpy(), want) <= 1e-8, (rel(X.cpu().numpy(), want), info)
    assert info["E_rel"][0] <= 1e-12


@pytest.mark.parametrize("k", [10, 19])
def test_qhpim_logspaced_kappa_1e6(ctx, k):
    A, U, s, V = I.logspaced_square(256, 1e-6, seed_u=1, seed_v=2)
    ctx.configure(hyper_order=k)
    X, info = ctx.solve(dev(A), "qhpim", tol=1e-12, max_iter=200)
    want = oracle.pinv_from_svd(U, s, V)
    assert info["E_rel"][0] <= 1e-10, info
    assert rel(X.cpu().numpy(), want) <= 1e-8, (rel(X.cpu().numpy(), want), info)


def test_example3_iteration_counts(ctx):
    """Example 3's setup: 800 x 800 Gaussian quaternion matrix (each component
    N(0, 1); seed 0 here), alpha = 7.8798e-5, ||X_{j+1} - X_j||_F <= 1e-10,
    FP64-accurate products.  The unfactorized solvers take as many iterations
    as the factorized ones of the same order; order 19 takes 8, as in the
    example's table.  (Order 10 takes 9 on this matrix, the table's 10 on the
    paper's: the count is 1 + ceil(log(c / (alpha sigma_min^2)) / log 10) and
    alpha sigma_min^2 = 3.6e-7 here.)"""
    A = I.gaussian_quaternion(800, 800, 0)
    ctx.configure(precision="emu", alpha="user", alpha_user=7.8798e-5, stop="paper_abs")
    iters = {}
    for method, k in [("qhpi19", 19), ("qhpim", 19), ("qsai", 10), ("qhpim", 10)]:
        ctx.configure(hyper_order=k)
        _, info = ctx.solve(dev(A), method, tol=1e-10, max_iter=500)
        assert info["status"] == "converged", (method, k, info)
        assert max(info["E"]) <= 2e-10, (method, k, info)  # the table: 6.3e-11 at most
        iters[(method, k)] = info["iters"]
    assert iters[("qhpim", 19)] == iters[("qhpi19", 19)] == 8, iters
    assert iters[("qhpim", 10)] == iters[("qsai", 10)] in (9, 10), iters


def test_qhpim_invalid_order_and_method(ctx, qp):
    for k in (1, 0, 65):
        with pytest.raises(qp.QpinvError) as e:
            ctx.configure(hyper_order=k)
        assert e.value.code == -1
    ctx.configure(hyper_order=19)
    A = dev(I.gaussian_quaternion(8, 8, 1))
    X = torch.empty((4, 8, 8), dtype=torch.float64, device="cuda")
    pa, lda, _ = qp._planes(A)
    px, ldx, _ = qp._planes(X)
    res = qp.qpinv_result()
    assert qp.qpinv_solve(ctx.h, None, 8, 8, pa, lda, 5, 1e-12, 10, px, ldx, res) == -1


@pytest.mark.parametrize("k", [3, 19])
def test_qhpim_batched_matches_exact_pinv(qp, k):
    mats = I.pure_quaternion_batch(16, seed=3, lo=16, hi=96)
    mats += [I.gaussian_quaternion(m, n, 40 + m + n) for (m, n) in [(1, 1), (7, 3), (3, 7), (33, 65)]]
    ctx = qp.Context(0, hyper_order=k)
    Xs, infos = ctx.solve_batched([dev(a) for a in mats], "qhpim", tol=1e-12, max_iter=300)
    for a, x, info in zip(mats, Xs, infos):
        C = I.chi(a)
        sv = np.linalg.svd(C, compute_uv=False)
        kappa = sv[0] / sv[sv > 1e-10 * sv[0]][-1]
        want = I.unchi(np.linalg.pinv(C, rcond=1e-10))
        err = rel(x.cpu().numpy(), want)
        assert info["status"] in ("converged", "plateau"), (a.shape, info)
        assert err <= 1e-10 + 1e-12 * k * kappa ** 2, (a.shape, kappa, err, info)
        assert info["E_rel"][0] <= 1e-10, (a.shape, info)
    ctx.close()


def test_qhpim_batched_agrees_with_oracle_iteration(qp):
    shapes = [(5, 4), (17, 31), (40, 24), (64, 64)]
    mats = [I.gaussian_quaternion(m, n, 70 + m) for (m, n) in shapes]
    ctx = qp.Context(0, hyper_order=6)
    Xs, _ = ctx.solve_batched([dev(a) for a in mats], "qhpim", tol=1e-13)
    for a, x in zip(mats, Xs):
        xo, _ = oracle.solve(a, "qhpim", tol=1e-13, order=6, side="left" if a.shape[1] > a.shape[2] else "right")
        assert rel(x.cpu().numpy(), xo) <= 1e-11
    ctx.close()


def test_example3_mixed_precision_converges(ctx):
    """Example 3's setup in mixed precision: every solver ends CONVERGED under
    the absolute rule (the returned X's residual bounds the next step below
    1e-10 when the last polish step itself did not), with the Penrose
    residuals of the FP64-accurate solve."""
    A = I.gaussian_quaternion(800, 800, 0)
    ctx.configure(precision="mixed", alpha="user", alpha_user=7.8798e-5, stop="paper_abs")
    for method, k in [("qhpi19", 19), ("qhpim", 19), ("qsai", 10), ("qhpim", 10)]:
        ctx.configure(hyper_order=k)
        _, info = ctx.solve(dev(A), method, tol=1e-10, max_iter=500)
        assert info["status"] == "converged", (method, k, info)
        assert max(info["E"]) <= 2e-10, (method, k, info)
        assert info["iters"] <= 11, (method, k, info)
