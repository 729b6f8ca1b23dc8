"""GPU parity of quaternion signal filtering (Sec. 5.2,
qpinv_toeplitz_filter) against the FP64 oracle (oracle/lorenz.py).

Tolerances: the data matrices here are invertible with kappa up to ~1e5,
and h = X^dagger s is computed to the FP64 level on both sides (relative
tol 1e-12, FP64-accurate products), so h agrees to ~kappa 1e-14 -> 1e-8;
the filter error eps = ||X h - s|| / ||s|| is at the rounding level on both
(the paper reports 8e-15 .. 6e-12): <= 1e-10."""
import numpy as np
import pytest

import oracle
from oracle import lorenz
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


def test_known_filter_recovered(ctx):
    p = 40
    x = I.gaussian_quaternion(1, 2 * p + 1, 5)[:, 0, :]
    h_true = I.gaussian_quaternion(p + 1, 1, 6)
    S = oracle.matmul(lorenz.data_matrix(x, p, p), h_true)
    s = np.zeros_like(x)
    s[:, p:] = S[:, :, 0]
    h, s_hat, err, info = ctx.toeplitz_filter(dev(x), dev(s), p, method="qsai", tol=1e-13)
    assert rel(h.cpu().numpy(), h_true) <= 1e-10, info
    assert err <= 1e-12
    ho, _, eo, _ = lorenz.design(x, s, p, p, "qsai", tol=1e-13)
    assert rel(h.cpu().numpy(), ho) <= 1e-10


@pytest.mark.parametrize("method", ["qsai", "ns", "qhpi19", "qrapid", "qhpim"])
@pytest.mark.parametrize("dt", [0.2, 0.1])
def test_lorenz_matches_oracle(ctx, method, dt):
    x, s = I.lorenz_signals(dt=dt)
    p = (x.shape[1] - 1) // 2
    ctx.configure(qrapid_N=2, hyper_order=7)
    h, s_hat, err, info = ctx.toeplitz_filter(dev(x), dev(s), p, method=method, tol=1e-12, max_iter=2000)
    ho, sho, eo, oinfo = lorenz.design(x, s, p, p, method, tol=1e-12, max_iter=2000, N=2, order=7)
    assert info["status"] in ("converged", "plateau"), info
    assert rel(h.cpu().numpy(), ho) <= 1e-8, (rel(h.cpu().numpy(), ho), info, oinfo)
    assert rel(s_hat.cpu().numpy(), sho) <= 1e-10
    assert err <= 1e-10 and eo <= 1e-10, (err, eo)


def test_lorenz_full_size_sampled(ctx):
    """The example's finest step, dt = 0.01 over [0, 40]: N = 4001 samples,
    a 2001 x 2001 data matrix.  The oracle cannot invert it in seconds, so
    the output is checked row by row: s_hat(i) = sum_j x(t0 + i - j) h_j
    for sampled i with the oracle's product, and eps <= 1e-10."""
    x, s = I.lorenz_signals(dt=0.01)
    p = (x.shape[1] - 1) // 2
    h, s_hat, err, info = ctx.toeplitz_filter(dev(x), dev(s), p, method="qsai", tol=1e-12)
    assert info["status"] in ("converged", "plateau") and info["E_rel"][0] <= 1e-10, info
    assert err <= 1e-10, err
    hh, sh = h.cpu().numpy(), s_hat.cpu().numpy()
    rows = [0, 1, 777, p // 2, p - 1, p]
    X = lorenz.data_matrix(x, p, p)
    want = oracle.matmul(X[:, rows, :], hh)
    assert np.max(np.abs(sh[:, rows, :] - want)) <= 1e-12 * np.abs(want).max()
    assert np.max(np.abs(want[:, :, 0] - s[:, p + np.array(rows)])) <= 1e-9 * np.abs(s).max()


def test_filter_host_pointers_match_device(ctx):
    x, s = I.lorenz_signals(dt=0.2)
    p = 50
    hd, _, ed, _ = ctx.toeplitz_filter(dev(x), dev(s), p, t0=70)
    hh, _, eh, _ = ctx.toeplitz_filter(x.copy(), s.copy(), p, t0=70)
    assert isinstance(hh, np.ndarray) and np.array_equal(hd.cpu().numpy(), hh) and ed == eh


def test_filter_invalid_arguments(ctx, qp):
    x, s = I.lorenz_signals(dt=0.2)
    N = x.shape[1]
    for p, t0 in ((10, 9), (100, N - 100), (-1, 5)):
        with pytest.raises(qp.QpinvError) as e:
            ctx.toeplitz_filter(dev(x), dev(s), p, t0=t0)
        assert e.value.code == -1
