"""qpinv_solve_batched (one persistent launch, double-FP32 arithmetic) against
LAPACK's pseudoinverse of the complex representation and the single-matrix
solver, on pure-quaternion rank-deficient blocks (A = B W, Dirichlet mixing)
and odd-shaped Gaussian matrices.

Tolerance: rank-deficient blocks amplify null-space rounding noise by about
kappa_eff^2 over a solve (kappa_eff = sigma_1 / sigma_r), and every extra
iteration before the plateau stop multiplies it by the method's order p, so
X must match the exact pseudoinverse to 1e-10 + 1e-12 p kappa_eff^2
(double-FP32 eps is ~1.4e-14); E1/||A|| <= 1e-10 for every matrix."""

ORDER = {"qhpi19": 19, "qsai": 10, "ns": 2, "qrapid": 5}
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


def exact_pinv(A):
    C = I.chi(A)
    sv = np.linalg.svd(C, compute_uv=False)
    return I.unchi(np.linalg.pinv(C, rcond=1e-10)), sv[0] / sv[sv > 1e-10 * sv[0]][-1]


def batch_inputs():
    mats = I.pure_quaternion_batch(20, seed=3, lo=16, hi=96)
    mats += [I.gaussian_quaternion(m, n, 40 + m + n) for (m, n) in [(1, 1), (7, 3), (3, 7), (33, 65), (65, 33)]]
    return mats


@pytest.mark.parametrize("method", ["qhpi19", "qsai", "ns", "qrapid"])
def test_batched_matches_exact_pinv(qp, method):
    mats = batch_inputs()
    ctx = qp.Context(0, qrapid_N=2)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, infos = ctx.solve_batched(As, method, tol=1e-12, max_iter=200)
    for a, x, info in zip(mats, Xs, infos):
        want, kappa = exact_pinv(a)
        err = np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want)
        assert info["status"] in ("converged", "plateau"), (a.shape, info)
        assert err <= 1e-10 + 1e-12 * ORDER[method] * kappa ** 2, (a.shape, kappa, err, info)
        assert info["E_rel"][0] <= 1e-10, (a.shape, info)
    ctx.close()


@pytest.mark.parametrize("tile", [-1, 5])
def test_batched_agrees_with_oracle_iteration(qp, tile):
    """Full-rank odd shapes: the batched X equals the FP64 oracle's X (autotuned
    engine, and the tensor-core engine with its 128 x 64 tiles spanning
    two row tiles and four column tiles at 256 x 200)."""
    shapes = [(5, 4), (17, 31), (40, 24), (64, 64), (256, 200), (130, 256)]
    mats = [I.gaussian_quaternion(m, n, 70 + m) for (m, n) in shapes]
    ctx = qp.Context(0, batched_tile=tile)
    Xs, infos = ctx.solve_batched([torch.from_numpy(a).cuda() for a in mats], "qhpi19", tol=1e-13)
    for a, x in zip(mats, Xs):
        xo, _ = oracle.solve(a, "qhpi19", tol=1e-13)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-11
    ctx.close()


def test_batched_nonfinite_matrix_is_isolated(qp):
    mats = batch_inputs()[:6]
    mats[2] = mats[2].copy()
    mats[2][1, 0, 0] = np.nan
    ctx = qp.Context(0)
    Xs, infos = ctx.solve_batched([torch.from_numpy(a).cuda() for a in mats], "qhpi19", tol=1e-12)
    assert infos[2]["status"] == "nonfinite_input"
    for b in (0, 1, 3, 4, 5):
        assert infos[b]["status"] in ("converged", "plateau") and infos[b]["E_rel"][0] <= 1e-10
    ctx.close()


def test_batched_rejects_oversize(qp):
    ctx = qp.Context(0)
    with pytest.raises(qp.QpinvError) as e:
        ctx.solve_batched([torch.zeros((4, 257, 3), dtype=torch.float64, device="cuda")], "ns")
    assert e.value.code == -1
    ctx.close()


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
def test_batched_every_tile_shape(qp, tile):
    """Each CTA GEMM engine -- the CUDA-core tile shapes 16x16 .. 64x64 and the
    tensor-core exact-slice engine (5) -- gives the same accuracy."""
    mats = batch_inputs()[:12] + [I.gaussian_quaternion(70, 130, 91), I.gaussian_quaternion(200, 90, 92)]
    ctx = qp.Context(0, batched_tile=tile)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, infos = ctx.solve_batched(As, "qhpi19", tol=1e-12, max_iter=200)
    assert ctx.stats()["batched_tile"] == tile
    for a, x, info in zip(mats, Xs, infos):
        want, kappa = exact_pinv(a)
        err = np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want)
        assert err <= 1e-10 + 1e-12 * ORDER["qhpi19"] * kappa ** 2, (a.shape, kappa, err, info)
    ctx.close()


def test_batched_autotune_and_graph_replay(qp):
    """Autotuning picks a tile once per batch signature; the second identical
    call replays the captured CUDA graph and reproduces X bit for bit."""
    mats = batch_inputs()
    ctx = qp.Context(0)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs1, _ = ctx.solve_batched(As, "qhpi19", tol=1e-12, max_iter=200)
    X1 = [x.clone() for x in Xs1]
    st1 = ctx.stats()
    assert 0 <= st1["batched_tile"] < 6 and st1["batched_tune_ms"] > 0
    Xs2, _ = ctx.solve_batched(As, "qhpi19", tol=1e-12, max_iter=200, Xs=Xs1)
    st2 = ctx.stats()
    assert st2["batched_tune_ms"] == st1["batched_tune_ms"]  # signature cached
    assert st2["batched_graph_replays"] == st1["batched_graph_replays"] + 1
    for a, b in zip(X1, Xs2):
        assert torch.equal(a, b)
    ctx.close()
