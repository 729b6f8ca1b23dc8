"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.

Tolerances (relative Frobenius error of X against the oracle's X):
  * FP64 products, or mixed precision with the FP64-residual polish: 1e-10;
  * tensor-core products only (FP32-level accumulation):              1e-5.
Quaternion GEMMs are checked against the oracle product with the error a
BF16 split of L terms allows with FP32 tensor-core accumulation (whose error
grows with K; K <= 1000 here): L = 1: 1e-2, L = 2: 3e-4, L = 3: 5e-5; FP64: 1e-13.
"""
import numpy as np
import pytest

import oracle
from paper_2605_01464_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEMM_TOL = {1: 1e-2, 2: 3e-4, 3: 5e-5}


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


@pytest.mark.parametrize("m,k,n", [(1, 1, 1), (7, 5, 3), (33, 65, 129), (130, 70, 257)])
def test_qgemm_fp64_matches_oracle(ctx, m, k, n):
    A = I.gaussian_quaternion(m, k, 1)
    B = I.gaussian_quaternion(k, n, 2)
    C = ctx.qgemm(dev(A), dev(B), precision="fp64").cpu().numpy()
    assert rel(C, oracle.matmul(A, B)) <= 1e-13


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("m,k,n", [(128, 64, 64), (200, 130, 90), (1, 1, 1), (257, 300, 129), (64, 1000, 40)])
def test_qgemm_tc_matches_oracle(ctx, L, m, k, n):
    A = I.gaussian_quaternion(m, k, 3)
    B = I.gaussian_quaternion(k, n, 4)
    C = ctx.qgemm(dev(A), dev(B), precision="tc", split_level=L).cpu().numpy()
    assert rel(C, oracle.matmul(A, B)) <= GEMM_TOL[L]


def test_qgemm_tc_each_sign_block(ctx):
    """Unit quaternion matrices isolate each (A component, B component) block
    of the real form: A = e_r * ones, B = e_s * eye; C must be e_r e_s."""
    basis = np.eye(4)
    for r in range(4):
        for s in range(4):
            A = np.zeros((4, 16, 16))
            A[r] = 1.0
            B = np.zeros((4, 16, 16))
            B[s] = np.eye(16)
            C = ctx.qgemm(dev(A), dev(B), precision="tc", split_level=1).cpu().numpy()
            want = oracle.qmul(basis[r], basis[s])
            assert np.allclose(C, want[:, None, None] * np.ones((1, 16, 16)), atol=0), (r, s)


METHODS = [("ns", 5), ("qsai", 5), ("qhpi19", 5), ("qrapid", 5), ("qrapid", 0), ("qrapid", 1)]


@pytest.mark.parametrize("method,N", METHODS)
@pytest.mark.parametrize("precision,tol_x", [("fp64", 1e-10), ("mixed", 1e-10), ("emu", 1e-10), ("tc", 1e-5)])
def test_solve_dense_gaussian_64x48(ctx, method, N, precision, tol_x):
    A = I.dense_gaussian(64, 48, seed=0)
    ctx.configure(precision=precision, qrapid_N=N)
    X, info = ctx.solve(dev(A), method, tol=1e-12, max_iter=200)
    Xo, oinfo = oracle.solve(A, method, tol=1e-12, max_iter=200, N=N)
    assert info["status"] in ("converged", "plateau", "not_converged"), info
    assert rel(X.cpu().numpy(), Xo) <= tol_x, (rel(X.cpu().numpy(), Xo), info)
    if precision != "tc":
        assert info["E_rel"][0] <= 1e-12, info
    assert info["side"] == "left"  # 64 x 48 is tall: residual on the 48 side


@pytest.mark.parametrize("method", ["ns", "qsai", "qhpi19", "qrapid"])
@pytest.mark.parametrize("shape,side", [((40, 96), "auto"), ((96, 40), "auto"), ((96, 40), "right"),
                                        ((40, 96), "left"), ((70, 70), "left")])
def test_solve_sides_and_shapes(ctx, method, shape, side):
    m, n = shape
    A = I.gaussian_quaternion(m, n, 7)
    ctx.configure(precision="mixed", side=side, qrapid_N=2)
    X, info = ctx.solve(dev(A), method, tol=1e-13, max_iter=200)
    Xo, _ = oracle.solve(A, method, tol=1e-13, max_iter=200, N=2)
    assert rel(X.cpu().numpy(), Xo) <= 1e-10, info


@pytest.mark.parametrize("method", ["ns", "qsai", "qhpi19", "qrapid"])
@pytest.mark.parametrize("precision", ["emu", "fp64"])
def test_solve_rank_deficient(ctx, method, precision):
    """Rank-deficient input: null-space rounding noise grows by the method's
    order per step -- about kappa^2 over a solve -- so these run with
    FP64-accurate products throughout, and X is accurate to about
    kappa^2 * eps (kappa = 1e3 here); the FP64 oracle agrees to the same level."""
    A, QL, s, QR = I.rank_deficient(80, 60, 20, 1e-3, seed_l=4, seed_r=5)
    ctx.configure(precision=precision, qrapid_N=3)
    X, info = ctx.solve(dev(A), method, tol=1e-13, max_iter=300)
    want = oracle.pinv_from_svd(QL, s, QR)
    assert info["status"] in ("converged", "plateau"), info
    assert rel(X.cpu().numpy(), want) <= 1e-8, (rel(X.cpu().numpy(), want), info)
    Xo, _ = oracle.solve(A, method, tol=1e-13, max_iter=300, N=3)
    assert rel(Xo, want) <= 1e-8
    assert info["E_rel"][0] <= 1e-12


def test_example1_iteration_counts_and_values(ctx):
    from tests.test_oracle_pins import load_example1
    A, P, vals = load_example1()
    ctx.configure(precision="fp64", alpha="spectral", stop="paper_abs")
    for method, N in [("qsai", 5), ("qhpi19", 5), ("qrapid", 1)]:
        ctx.configure(qrapid_N=N)
        X, info = ctx.solve(dev(A), method, tol=1e-10, max_iter=100)
        assert abs(info["alpha"] - vals["alpha"]) <= 0.5e-9
        assert info["iters"] == vals[("iters", method)], (method, info)
        assert np.max(np.abs(X.cpu().numpy() - P)) <= 0.5e-4 + 1e-12
        assert max(info["E"]) <= vals["Emax"]


def test_nonfinite_input_rejected(ctx, qp):
    A = I.gaussian_quaternion(10, 8, 1)
    A[2, 3, 4] = np.nan
    with pytest.raises(qp.QpinvError) as e:
        ctx.solve(dev(A), "qhpi19")
    assert e.value.code == -4


def test_max_iter_one_not_converged(ctx):
    A = I.gaussian_quaternion(20, 12, 2)
    X, info = ctx.solve(dev(A), "ns", tol=1e-14, max_iter=1)
    assert info["status"] == "not_converged" and info["iters"] == 1
    Xo, _ = oracle.solve(A, "ns", tol=1e-14, max_iter=1)
    ctx.configure(precision="fp64")
    X, info = ctx.solve(dev(A), "ns", tol=1e-14, max_iter=1)
    assert rel(X.cpu().numpy(), Xo) <= 1e-13


def test_divergent_alpha_detected(ctx):
    A = I.gaussian_quaternion(16, 12, 5)
    smax = oracle.sigma_max(A)
    ctx.configure(precision="fp64", alpha="user", alpha_user=3.0 / smax ** 2)
    X, info = ctx.solve(dev(A), "qhpi19", tol=1e-14, max_iter=60)
    assert info["status"] == "diverged"
    assert np.all(np.isfinite(X.cpu().numpy()))


def test_host_pointers_match_device(ctx):
    A = I.gaussian_quaternion(50, 30, 11)
    Xd, _ = ctx.solve(dev(A), "qsai", tol=1e-12)
    Xh, _ = ctx.solve(A.copy(), "qsai", tol=1e-12)
    assert isinstance(Xh, np.ndarray)
    assert np.array_equal(Xd.cpu().numpy(), Xh)


def test_penrose_matches_oracle(ctx):
    A = I.gaussian_quaternion(30, 20, 12)
    Xo, _ = oracle.solve(A, "qhpi19", tol=1e-6, max_iter=3)
    E, R = ctx.penrose(dev(A), dev(Xo))
    Eo, Ro = oracle.penrose(A, Xo)
    assert np.allclose(E, Eo, rtol=1e-8, atol=1e-14)
    assert np.allclose(R, Ro, rtol=1e-8, atol=1e-14)


def test_penrose_small_residual_closed_form(ctx):
    """Square unitary A = Q and X = Q^H + d E: E1 = ||Q (d E) Q|| = d ||E||
    and E2 = ||d E + d^2 E Q E|| exactly (unitary invariance), small enough
    that the outer products run on 6 exact slices after their error check."""
    Q = I.orthonormal_columns(64, 64, 21)
    E = I.gaussian_quaternion(64, 64, 22)
    d = 1e-9
    X = oracle.adjoint(Q) + d * E
    ctx.configure(precision="emu")
    got, _ = ctx.penrose(dev(Q), dev(X))
    e1 = d * np.linalg.norm(E)
    e2 = np.linalg.norm(d * E + d * d * oracle.matmul(oracle.matmul(E, Q), E))
    assert abs(got[0] - e1) <= 1e-6 * e1, (got, e1)
    assert abs(got[1] - e2) <= 1e-6 * e2, (got, e2)
    ctx.configure(precision="mixed")


def test_spectral_alpha_matches_oracle(ctx):
    A = I.gaussian_quaternion(40, 25, 13)
    ctx.configure(alpha="spectral")
    _, info = ctx.solve(dev(A), "qhpi19", tol=1e-12)
    assert abs(info["alpha"] - oracle.alpha(A, "spectral")) <= 1e-9 * info["alpha"]


def test_gemm_counts_per_iteration(ctx):
    A = I.gaussian_quaternion(24, 24, 14)
    ctx.configure(precision="tc", penrose=False, stop="paper_abs")
    for method, N, per in [("ns", 0, 2), ("qsai", 0, 6), ("qhpi19", 0, 7), ("qrapid", 2, 12)]:
        ctx.configure(qrapid_N=N)
        _, info = ctx.solve(dev(A), method, tol=0.0, max_iter=3)
        assert info["gemms"] == 3 * per, (method, info)


EMU_TOL = {2: 1e-3, 4: 1e-7, 6: 1e-11, 8: 1e-14}


@pytest.mark.parametrize("S", [2, 4, 6, 8])
@pytest.mark.parametrize("m,k,n", [(130, 300, 257), (64, 1000, 40), (1, 1, 1), (200, 64, 90)])
def test_qgemm_exact_slices_match_oracle(ctx, S, m, k, n):
    """Exact-slice products: S slices of 7 bits per operand; 8 slices give an
    FP64-level product (the oracle's own rounding is the reference)."""
    A = I.gaussian_quaternion(m, k, 5)
    B = I.gaussian_quaternion(k, n, 6)
    C = ctx.qgemm(dev(A), dev(B), precision="emu", split_level=S).cpu().numpy()
    assert rel(C, oracle.matmul(A, B)) <= EMU_TOL[S], rel(C, oracle.matmul(A, B))


@pytest.mark.parametrize("S,k", [(8, 13500), (4, 30000)])
def test_qgemm_exact_slices_long_k(ctx, S, k):
    """K beyond the fused kernel's int32 level sums (13107 for 8 slices,
    21845 for 4): the chunked multi-launch path with int64 epilogues."""
    A = I.gaussian_quaternion(40, k, 9)
    B = I.gaussian_quaternion(k, 24, 10)
    C = ctx.qgemm(dev(A), dev(B), precision="emu", split_level=S).cpu().numpy()
    assert rel(C, oracle.matmul(A, B)) <= EMU_TOL[S] * 4, rel(C, oracle.matmul(A, B))


def test_qgemm_exact_slices_wide_dynamic_range(ctx):
    """Rows and columns spanning 2^-40 .. 2^40: per-row/column power-of-two
    scaling keeps every entry FP64-accurate relative to its row/column scale."""
    rng = np.random.default_rng(3)
    A = I.gaussian_quaternion(96, 128, 7) * np.exp2(rng.integers(-40, 40, size=(1, 96, 1)))
    B = I.gaussian_quaternion(128, 80, 8) * np.exp2(rng.integers(-40, 40, size=(1, 1, 80)))
    C = ctx.qgemm(dev(A), dev(B), precision="emu", split_level=8).cpu().numpy()
    Co = oracle.matmul(A, B)
    scale = np.abs(A).max(axis=(0, 2))[:, None] * np.abs(B).max(axis=(0, 1))[None, :] * 128
    assert np.max(np.abs(C - Co) / scale[None]) <= 1e-15


@pytest.mark.parametrize("m,n", [(640, 320), (320, 640)])
def test_solve_rectangular_full_rank_mixed(ctx, m, n):
    """Full-rank rectangular A with sigma geometric 1..1e-4: MIXED (no EMU
    retry) must reach the FP64 level, which needs the component of X outside
    the pseudoinverse's row / column space (left by the FP32 phase) removed."""
    k = min(m, n)
    s = np.geomspace(1.0, 1e-4, k)
    U = I.orthonormal_columns(m, k, 31)
    V = I.orthonormal_columns(n, k, 32)
    A = I.with_spectrum(U, s, V)
    X, info = ctx.solve(dev(A), "qhpi19", tol=1e-12)
    assert info["precision"] == "mixed", info
    assert info["E_rel"][0] <= 1e-10 and info["E_rel"][1] <= 1e-10, info
    assert rel(X.cpu().numpy(), oracle.pinv_from_svd(U, s, V)) <= 1e-9, info


@pytest.mark.parametrize("method", ["qhpi19", "qsai", "ns"])
def test_solve_logspaced_kappa_1e6(ctx, method):
    """Square A = U diag(sigma) V^H with sigma log-spaced 1..1e-6 (the large
    workload's structure at n = 256): mixed precision must reach the FP64
    level: E1/||A|| <= 1e-10 and X within 1e-8 of the exact V Sigma^-1 U^H."""
    A, U, s, V = I.logspaced_square(256, 1e-6, seed_u=1, seed_v=2)
    X, info = ctx.solve(dev(A), method, tol=1e-12, max_iter=200)
    want = oracle.pinv_from_svd(U, s, V)
    assert info["E_rel"][0] <= 1e-10, info
    assert rel(X.cpu().numpy(), want) <= 1e-8, (rel(X.cpu().numpy(), want), info)
    Eo, Ro = oracle.penrose(A, X.cpu().numpy())
    assert Ro[0] <= 1e-10  # the oracle's own FP64 evaluation of E1 agrees with the bound


@pytest.mark.parametrize("method,N", [("qhpi19", 5), ("qsai", 5), ("qrapid", 2), ("ns", 5), ("qhpim", 5)])
def test_fused_epilogue_matches_separate_combine(ctx, method, N):
    """The combine pass run in the tensor-core GEMM's epilogue and the same
    pass as its own kernel give the same iterates (same FP32 arithmetic in
    the same order; only the FMA contraction of two compilations may
    differ), on ragged shapes (200 x 136: partial row and column tiles)."""
    A = I.gaussian_quaternion(200, 136, 17)
    got = {}
    for fuse in (True, False):
        ctx.configure(precision="tc", qrapid_N=N, hyper_order=7, fuse_epilogue=fuse)
        ctx.reset_stats()
        X, info = ctx.solve(dev(A), method, tol=1e-6, max_iter=60)
        st = ctx.stats()
        assert (st["fused_epilogues"] > 0) == fuse, st
        got[fuse] = (X.cpu().numpy(), info)
    ctx.configure(precision="mixed", fuse_epilogue=True, hyper_order=19)
    (X1, i1), (X2, i2) = got[True], got[False]
    assert i1["iters"] == i2["iters"], (i1, i2)
    assert rel(X1, X2) <= 1e-6, rel(X1, X2)
    Xo, _ = oracle.solve(A, method, tol=1e-6, max_iter=60, N=N, order=7)
    assert rel(X1, Xo) <= 1e-5


@pytest.mark.parametrize("case", ["logspaced256", "gaussian200x136"])
def test_fused_epilogue_fp64_polish(ctx, case):
    """In the FP64 polish steps of the mixed schedule the BF16 R-products
    take their combine pass (FP64 arithmetic on FP64 masters) in the GEMM's
    epilogue: fewer tensor-core products run unfused than the five R-products
    of each QHPI19 polish step, and X equals the separate combine's result up
    to the FMA contraction of two compilations (ragged tiles at 200 x 136)."""
    if case == "logspaced256":
        A, U, s, V = I.logspaced_square(256, 1e-6, seed_u=1, seed_v=2)
        want = oracle.pinv_from_svd(U, s, V)
    else:
        A = I.gaussian_quaternion(200, 136, 17)
        want = None
    runs = {}
    for fuse in (True, False):
        ctx.configure(precision="mixed", fuse_epilogue=fuse)
        ctx.reset_stats()
        X, info = ctx.solve(dev(A), "qhpi19", tol=1e-12, max_iter=200)
        runs[fuse] = (X.cpu().numpy(), info, ctx.stats())
    ctx.configure(precision="mixed", fuse_epilogue=True)
    (X1, i1, s1), (X2, i2, s2) = runs[True], runs[False]
    assert i1["tc_iters"] == i2["tc_iters"] > 0 and i1["polish_iters"] == i2["polish_iters"] > 0, (i1, i2)
    assert s2["fused_epilogues"] == 0, s2
    assert s1["tc_gemm_launches"] - s1["fused_epilogues"] < 5 * i1["polish_iters"], (s1, i1)
    assert i1["E_rel"][0] <= 1e-10 and i2["E_rel"][0] <= 1e-10, (i1, i2)
    assert rel(X1, X2) <= 1e-9, rel(X1, X2)
    if want is not None:
        assert rel(X1, want) <= 1e-8, rel(X1, want)


@pytest.mark.parametrize("precision", ["emu", "fp64"])
@pytest.mark.parametrize("shape", [(96, 64), (64, 96)])
def test_penrose_reuses_final_residual(ctx, precision, shape):
    """A solve whose stop rule rejects its last step (PLATEAU at an
    unreachable tolerance) returns X_j, whose residual I - AX (I - XA on the
    left side) that step formed with FP64-accurate products: the Penrose pass
    takes it instead of forming the product again, and its E1..E4 equal the
    stand-alone Penrose evaluation of the returned X (both sides formed)."""
    m, n = shape
    A = I.gaussian_quaternion(m, n, 23)
    ctx.configure(precision=precision)
    ctx.reset_stats()
    X, info = ctx.solve(dev(A), "qhpi19", tol=1e-30, max_iter=100)
    st = ctx.stats()
    assert info["status"] == "plateau", info
    assert st["penrose_reused"] == 1, st
    E, _ = ctx.penrose(dev(A), X)
    for k in range(4):
        assert abs(info["E"][k] - E[k]) <= 1e-12 * max(E[k], 1e-300) + 1e-300, (k, info["E"], E)
    Eo, Ro = oracle.penrose(A, X.cpu().numpy())
    assert max(Ro) <= 1e-12, Ro


@pytest.mark.parametrize("S", [2, 4, 8])
@pytest.mark.parametrize("m,k,n", [(130, 300, 257), (200, 64, 90), (300, 1000, 40), (513, 96, 200)])
def test_qgemm_exact_slices_on_sm_pairs(ctx, S, m, k, n):
    """The exact-slice product on pairs of SMs (256-row tiles, one M = 256
    MMA for both CTAs, half of B staged per CTA) against the oracle, and
    equal bit for bit to the one-SM kernel (same slices, levels, chunks and
    int64 sums); shapes with partial pair tiles (rows past the second CTA's
    half) and ragged columns."""
    A = I.gaussian_quaternion(m, k, 15)
    B = I.gaussian_quaternion(k, n, 16)
    ctx.configure(emu_pair=True)
    ctx.reset_stats()
    Cp = ctx.qgemm(dev(A), dev(B), precision="emu", split_level=S).cpu().numpy()
    assert ctx.stats()["emu_gemm_launches"] >= 1
    ctx.configure(emu_pair=False)
    C1 = ctx.qgemm(dev(A), dev(B), precision="emu", split_level=S).cpu().numpy()
    ctx.configure(emu_pair="auto")
    assert rel(Cp, oracle.matmul(A, B)) <= EMU_TOL[S], rel(Cp, oracle.matmul(A, B))
    assert np.array_equal(Cp, C1)


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("m,k,n", [(128, 64, 128), (200, 130, 300), (257, 300, 129), (64, 1000, 200)])
def test_qgemm_tc_broad_tiles(ctx, L, m, k, n):
    """BF16-split products on 128-column tiles (one CTA per SM, a 512-column
    accumulator) against the oracle, and equal bit for bit to the 64-column
    tiles (same MMAs per K step into the same FP32 accumulator entries)."""
    A = I.gaussian_quaternion(m, k, 25)
    B = I.gaussian_quaternion(k, n, 26)
    ctx.configure(tc_broad=True)
    Cb = ctx.qgemm(dev(A), dev(B), precision="tc", split_level=L).cpu().numpy()
    ctx.configure(tc_broad=False)
    Cw = ctx.qgemm(dev(A), dev(B), precision="tc", split_level=L).cpu().numpy()
    ctx.configure(tc_broad="auto")
    Co = oracle.matmul(A, B)
    tol = {1: 1e-2, 2: 3e-4}.get(L, 5e-5 * max(1.0, k / 1000.0))
    assert rel(Cb, Co) <= tol, rel(Cb, Co)
    assert np.array_equal(Cb, Cw)


@pytest.mark.parametrize("method", ["qhpi19", "qsai"])
def test_solve_tc_broad_tiles_match(ctx, method):
    """A mixed-precision solve with the fused epilogues on 64-column tiles
    (two CTAs per SM), on the broad 128-column tiles, and on the persistent
    component-pair items (the default for fused products) gives the same
    iterates: the products are the same bit for bit, only the stop norms'
    partial sums are grouped differently."""
    A, U, s, V = I.logspaced_square(256, 1e-6, seed_u=1, seed_v=2)
    got = {}
    for broad in (False, True, "auto"):
        ctx.configure(tc_broad=broad)
        ctx.reset_stats()
        X, info = ctx.solve(dev(A), method, tol=1e-12, max_iter=200)
        assert ctx.stats()["fused_epilogues"] > 0
        got[broad] = (X.cpu().numpy(), info)
    ctx.configure(tc_broad="auto")
    Xw, iw = got[False]
    for key in (True, "auto"):
        Xb, ib = got[key]
        assert iw["iters"] == ib["iters"] and iw["status"] == ib["status"], (key, iw, ib)
        assert rel(Xb, Xw) <= 1e-12, (key, rel(Xb, Xw))
        assert ib["E_rel"][0] <= 1e-10, ib


@pytest.mark.parametrize("m,k,n", [(200, 130, 300), (300, 257, 136), (640, 512, 520)])
def test_fused_epilogue_component_pairs_match_wide(ctx, m, k, n):
    """One Newton-Schulz step's fused residual product on the persistent
    component-pair shape equals the 64-column shape's, bit for bit in X
    (several items per CTA at 640 x 520: 5 x 5 tiles x 2 pairs)."""
    A = I.gaussian_quaternion(m, n, 27)
    out = {}
    for broad in (False, "auto"):
        ctx.configure(precision="tc", tc_broad=broad)
        X, info = ctx.solve(dev(A), "ns", tol=1e-30, max_iter=2)
        out[broad] = X.cpu().numpy()
    ctx.configure(precision="mixed", tc_broad="auto")
    assert np.array_equal(out[False], out["auto"])
