"""GPU parity of CUR image completion (Sec. 5.1, qpinv_cur_complete) against
the FP64 oracle (oracle/cur.py) on the same seeded image, mask and index sets.

Tolerance: the products are FP64-accurate on both sides, so C^(T) differs
only through the pseudoinverses, which the solver delivers at the FP64 level
(relative tol 1e-12 with the Penrose check): about kappa(C_J) 1e-13 per
iteration, kappa ~1e2..1e3 for these images, through a loop that does not
amplify it (the reconstruction is a pair of projections) -> 1e-8 relative
over the image; the FP64-precision context (CUDA-core products) meets 1e-9.
Observed pixels must come back bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import cur
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def workload(m, n, r, T, seed=16):
    A = I.synthetic_rgb_image(m, n, seed)
    mask = I.completion_mask(m, n, 0.3, seed + 1)
    Is, Js = I.cur_index_sets(m, n, r, T, seed + 2)
    return A, mask, Is, Js


@pytest.mark.parametrize("method", ["qhpi19", "qsai", "qrapid", "ns", "qhpim"])
@pytest.mark.parametrize("sigma", [0.0, 0.5])
@pytest.mark.parametrize("shape", [(48, 64, 8, 6), (70, 45, 11, 4)])
def test_cur_matches_oracle(ctx, method, sigma, shape):
    m, n, r, T = shape
    A, mask, Is, Js = workload(m, n, r, T)
    M = A * mask
    ctx.configure(qrapid_N=2, hyper_order=7)
    C, info = ctx.cur_complete(dev(M), dev(mask), Is, Js, method, tol=1e-12, max_iter=200, sigma=sigma)
    Co, hist = cur.cur_complete(M, mask, Is, Js, method, tol=1e-12, max_iter=200, sigma=sigma, N=2, order=7)
    C = C.cpu().numpy()
    assert rel(C, Co) <= 1e-8, (rel(C, Co), info)
    assert np.array_equal(C[:, mask != 0], M[:, mask != 0])
    assert info["pinv_solves"] == 2 * T and info["pinv_worst_status"] in ("converged", "plateau"), info
    assert info["pinv_max_E1_rel"] <= 1e-12, info


def test_cur_fp64_precision_matches_oracle(ctx):
    A, mask, Is, Js = workload(40, 52, 6, 5, seed=30)
    M = A * mask
    ctx.configure(precision="fp64")
    C, _ = ctx.cur_complete(dev(M), dev(mask), Is, Js, "qhpi19", sigma=0.5)
    Co, _ = cur.cur_complete(M, mask, Is, Js, "qhpi19", sigma=0.5)
    assert rel(C.cpu().numpy(), Co) <= 1e-9


def test_cur_full_size_example(ctx):
    """The paper's workload shape: 512 x 768 colour image, 70 % of the pixels
    removed, rank 60, 25 iterations, sigma = 0.5, QHPI19 pseudoinverses."""
    A, mask, Is, Js = workload(512, 768, 60, 25)
    M = A * mask
    C, info = ctx.cur_complete(dev(M), dev(mask), Is, Js, "qhpi19", sigma=0.5)
    Co, _ = cur.cur_complete(M, mask, Is, Js, "qhpi19", sigma=0.5)
    C = C.cpu().numpy()
    assert rel(C, Co) <= 1e-8, rel(C, Co)
    assert abs(cur.psnr(C, A) - cur.psnr(Co, A)) <= 1e-6
    assert cur.psnr(C, A) >= 30.0, cur.psnr(C, A)  # masked input: 7.4 dB
    assert info["pinv_solves"] == 50 and info["pinv_max_E1_rel"] <= 1e-12, info


def test_cur_exact_low_rank_reproduced(ctx):
    """Exact rank-3 quaternion matrix with one pixel missing outside every
    chosen row and column: C_J and R_I are exact, so the cross form
    C_J W^+ R_I restores the pixel in one iteration (CUR identity, r = rank);
    the optimal form projects the filled matrix, whose error at the pixel
    shrinks by the product of its row and column leverages each iteration."""
    A = oracle.matmul(I.gaussian_quaternion(30, 3, 7), I.gaussian_quaternion(3, 44, 8))
    Is, Js = I.cur_index_sets(30, 44, 3, 10, 8)
    i = min(set(range(30)) - set(Is.ravel().tolist()))
    j = min(set(range(44)) - set(Js.ravel().tolist()))
    mask = np.ones((30, 44), dtype=np.uint8)
    mask[i, j] = 0
    ctx.configure(precision="emu")
    for cross, T in ((True, 1), (False, 10)):
        C, _ = ctx.cur_complete(dev(A * mask), dev(mask), Is[:T], Js[:T], "qhpi19", tol=1e-14, sigma=0.0,
                                cross=cross)
        got = C.cpu().numpy()[:, i, j]
        assert np.max(np.abs(got - A[:, i, j])) <= 1e-9 * np.abs(A).max(), (cross, got, A[:, i, j])


def test_cur_host_pointers_match_device(ctx):
    A, mask, Is, Js = workload(32, 40, 5, 3, seed=40)
    M = A * mask
    Cd, _ = ctx.cur_complete(dev(M), dev(mask), Is, Js, "qsai", sigma=0.5)
    Ch, _ = ctx.cur_complete(M.copy(), mask.copy(), Is, Js, "qsai", sigma=0.5)
    assert isinstance(Ch, np.ndarray)
    assert np.array_equal(Cd.cpu().numpy(), Ch)


def test_cur_invalid_arguments(ctx, qp):
    A, mask, Is, Js = workload(16, 20, 4, 2, seed=50)
    M, mk = dev(A * mask), dev(mask)
    bad_I = Is.copy()
    bad_I[1, 2] = 16
    for kwargs in (dict(I=bad_I, J=Js), dict(I=Is[:, :2], J=Js[:, :2], sigma=9.0),
                   dict(I=np.zeros((1, 17), np.int32), J=np.zeros((1, 17), np.int32))):
        args = dict(I=Is, J=Js, sigma=0.5)
        args.update(kwargs)
        with pytest.raises(qp.QpinvError) as e:
            ctx.cur_complete(M, mk, args["I"], args["J"], "qhpi19", sigma=args["sigma"])
        assert e.value.code == -1
