"""FP64 CPU oracle of quaternion signal filtering (Sec. 5.2).

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py``
may use this module; the product library never does.

The filter s(t) ~ sum_{m=0}^{p} x(t - m) h_m (eq. (conv)) in matrix form
X h = s with the (p+1) x (p+1) data matrix X(i, j) = x(t + i - j) and
s(i) = s(t + i), i, j = 0..p; h = X^dagger s, the output s_hat = X h and the
error eps = ||s_hat - s|| / ||s|| (Sec. 5.2).  Signals are (4, N) planes;
sample index t0 plays the role of t.  X^dagger comes from this package's
iterations (``oracle.solve``), products from its naive C product.
"""
import numpy as np

from . import matmul, solve


def data_matrix(x, p, t0):
    """X(i, j) = x(t0 + i - j), i, j = 0..p, written out entry by entry."""
    x = np.asarray(x, dtype=np.float64)
    X = np.empty((4, p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            X[:, i, j] = x[:, t0 + i - j]
    return X


def design(x, s, p, t0, method="qsai", tol=1e-12, max_iter=500, N=5, order=19):
    """Returns (h (4, p+1, 1), s_hat (4, p+1, 1), eps, info of the solve)."""
    X = data_matrix(x, p, t0)
    S = np.asarray(s, dtype=np.float64)[:, t0:t0 + p + 1, None]
    Xp, info = solve(X, method, tol=tol, max_iter=max_iter, N=N, order=order)
    h = matmul(Xp, S)
    s_hat = matmul(X, h)
    eps = np.linalg.norm(s_hat - S) / np.linalg.norm(S)
    return h, s_hat, eps, info
