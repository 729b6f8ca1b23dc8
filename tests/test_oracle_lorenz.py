"""Pins of the quaternion filtering oracle (Sec. 5.2): the data matrix's
Toeplitz structure (eq. (conv) in matrix form), exact recovery of a known
filter from its own output, the error level of the Lorenz example, and the
signal generator against scipy's high-order integrator.  A planted mistake
shows the pins bite."""
import numpy as np
import pytest

import oracle
from oracle import lorenz
from paper_2605_01464_gb300 import inputs as I


def check_structure(p=6, t0=9):
    x = I.gaussian_quaternion(1, 20, 3)[:, 0, :]
    X = lorenz.data_matrix(x, p, t0)
    for i in range(p + 1):
        for j in range(p + 1):
            assert np.array_equal(X[:, i, j], x[:, t0 + i - j])
    # rows are the delayed samples x(t + i), x(t + i - 1), ..., x(t + i - p)
    assert np.array_equal(X[:, :, 0], x[:, t0:t0 + p + 1])
    assert np.array_equal(X[:, 0, :], x[:, t0 - np.arange(p + 1)])


def check_recovery(p=20, seed=5):
    N = 2 * p + 1
    x = I.gaussian_quaternion(1, N, seed)[:, 0, :]
    t0 = p
    h_true = I.gaussian_quaternion(p + 1, 1, seed + 1)
    S = oracle.matmul(lorenz.data_matrix(x, p, t0), h_true)
    s = np.zeros((4, N))
    s[:, t0:t0 + p + 1] = S[:, :, 0]
    h, s_hat, eps, info = lorenz.design(x, s, p, t0, "qsai", tol=1e-14)
    assert np.linalg.norm(h - h_true) / np.linalg.norm(h_true) <= 1e-10, info
    assert eps <= 1e-13


def test_data_matrix_is_the_delay_toeplitz_matrix():
    check_structure()


def test_known_filter_is_recovered():
    check_recovery()


@pytest.mark.parametrize("method", ["qsai", "ns", "qhpi19"])
def test_lorenz_example_error_level(method):
    # Sec. 5.2 with dt = 0.2 (N = 201, p = 100): the square data matrix is
    # invertible, so the filter output matches the target to rounding
    # (the paper's errors: 1e-14 .. 6e-12)
    x, s = I.lorenz_signals(dt=0.2)
    p = (x.shape[1] - 1) // 2
    h, s_hat, eps, info = lorenz.design(x, s, p, p, method, tol=1e-13, max_iter=2000)
    assert info["status"] in ("converged", "plateau"), info
    assert eps <= 1e-10, eps


def test_lorenz_trajectory_matches_scipy():
    integrate = pytest.importorskip("scipy.integrate")
    tr = I.lorenz_trajectory(0.01, 2.0)

    def f(t, y):
        return [10.0 * (y[1] - y[0]), y[0] * (28.0 - y[2]) - y[1], y[0] * y[1] - 8.0 / 3.0 * y[2]]
    ref = integrate.solve_ivp(f, (0.0, 2.0), [1.0, 1.0, 1.0], method="DOP853", rtol=1e-12, atol=1e-12,
                              t_eval=np.linspace(0.0, 2.0, 201))
    assert np.max(np.abs(tr - ref.y.T)) <= 1e-6


def test_signals_are_pure_and_delayed():
    x, s = I.lorenz_signals(dt=0.1, tau=1.0, noise=0.0)
    assert not x[0].any() and not s[0].any()
    assert np.array_equal(x[:, 10:], s[:, :-10])  # x(t) = s(t - tau), tau = 10 samples


def test_planted_mistake_is_caught(monkeypatch):
    raw = lorenz.data_matrix
    monkeypatch.setattr(lorenz, "data_matrix", lambda x, p, t0: raw(x, p, t0).transpose(0, 2, 1).copy())
    with pytest.raises(AssertionError):
        check_structure()


def test_single_tap_filter_is_the_quaternion_quotient():
    # p = 0: X = [x(t0)], h_0 = x(t0)^-1 s(t0) and s_hat = s exactly
    x = I.gaussian_quaternion(1, 5, 61)[:, 0, :]
    s = I.gaussian_quaternion(1, 5, 62)[:, 0, :]
    h, s_hat, eps, info = lorenz.design(x, s, 0, 2, "qsai", tol=1e-15)
    q = x[:, 2]
    qinv = np.array([q[0], -q[1], -q[2], -q[3]]) / np.dot(q, q)
    assert np.allclose(h[:, 0, 0], oracle.qmul(qinv, s[:, 2]), rtol=0, atol=1e-14)
    assert eps <= 1e-15
