"""FP64 CPU oracle of quaternion CUR image completion (Sec. 5.1).

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py``
may use this module; the product library never does.  Pseudoinverses come
from this package's own iterations (``oracle.solve``) and every quaternion
product from its naive C matrix product (``oracle.matmul``).

The impute-reconstruct loop (eq. (update) of Sec. 5.1):
    C^(0) = Omega . M  (+ (1 - Omega) . X_init when a start is given)
    X^(t) = L(C^(t)),   C^(t+1) = Omega . M + (1 - Omega) . X^(t)
with the CUR reconstruction L(C) = C_J U R_I, C_J = C(:, J_t), R_I = C(I_t, :),
and U = C_J^dagger C R_I^dagger (eq. (Uopt) with A the current filled
matrix), evaluated left to right; optionally followed by a 2-D Gaussian
filter of standard deviation sigma on every plane (the spatial regulariser of
Sec. 5.1).  Readings (the paper is silent on them):
  * U: the optimal form (Uopt).  The cross form U = W^dagger, W = C(I, J)
    (eq. (Ucross)) is offered too; with index sets drawn uniformly at random
    it diverges on smooth images (the paper notes that its accuracy depends
    on the choice of rows and columns);
  * the index sets are drawn afresh for every iteration (passed in);
  * the filter is the sampled Gaussian on |x| <= ceil(2 sigma) (3 taps for
    sigma = 0.5), normalised to sum 1, with replicated borders;
  * missing pixels start at 0; no projection onto pure quaternions or
    clipping is applied inside the loop; the result is C^(T).
"""
import math

import numpy as np

from . import matmul, solve


def gaussian_weights(sigma):
    """Sampled Gaussian exp(-x^2 / (2 sigma^2)) on the integers |x| <= ceil(2 sigma),
    normalised to sum 1."""
    R = int(math.ceil(2.0 * sigma))
    x = np.arange(-R, R + 1, dtype=np.float64)
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def gaussian_filter(X, sigma):
    """2-D Gaussian filter of every plane of X (4, m, n): out(i, j) = sum over
    offsets (a, b) of g_a g_b X(clamp(i + a), clamp(j + b))."""
    g = gaussian_weights(sigma)
    R = (g.size - 1) // 2
    m, n = X.shape[1], X.shape[2]
    P = np.pad(X, ((0, 0), (R, R), (R, R)), mode="edge")
    out = np.zeros_like(X)
    for a in range(2 * R + 1):
        for b in range(2 * R + 1):
            out += (g[a] * g[b]) * P[:, a:a + m, b:b + n]
    return out


def pinv(A, method, tol, max_iter, N, order):
    """A^dagger by the chosen iteration, residual on the smaller side."""
    side = "left" if A.shape[1] > A.shape[2] else "right"
    return solve(A, method, tol=tol, max_iter=max_iter, side=side, N=N, order=order)


def cur_reconstruct(C, I, J, method="qhpi19", tol=1e-12, max_iter=200, N=5, order=19, cross=False):
    """L(C) = C_J U R_I with U = C_J^dagger C R_I^dagger (or W^dagger, W = C(I, J),
    when cross).  Returns (X, [info of each pseudoinverse solve])."""
    CJ = C[:, :, J]
    RI = C[:, I, :]
    if cross:
        U, info = pinv(C[:, I][:, :, J], method, tol, max_iter, N, order)
        infos = [info]
    else:
        CJp, i1 = pinv(CJ, method, tol, max_iter, N, order)
        RIp, i2 = pinv(RI, method, tol, max_iter, N, order)
        U = matmul(matmul(CJp, C), RIp)
        infos = [i1, i2]
    return matmul(matmul(CJ, U), RI), infos


def cur_complete(M, mask, I, J, method="qhpi19", tol=1e-12, max_iter=200, sigma=0.5, N=5, order=19,
                 x_init=None, cross=False):
    """Runs len(I) completion iterations.  M: (4, m, n) planes (values at
    unobserved pixels are ignored); mask: (m, n), nonzero = observed; I, J:
    (iters, r) index sets.  Returns (C^(T), list of per-iteration solve infos)."""
    obs = (np.asarray(mask) != 0)[None, :, :]
    C = np.where(obs, M, 0.0 if x_init is None else x_init)
    history = []
    for t in range(len(I)):
        X, infos = cur_reconstruct(C, I[t], J[t], method, tol, max_iter, N, order, cross)
        if sigma > 0:
            X = gaussian_filter(X, sigma)
        C = np.where(obs, M, X)
        history.append(infos)
    return C, history


def psnr(X, ref, peak=1.0):
    """Peak signal-to-noise ratio over the colour planes (x, y, z = R, G, B)."""
    mse = np.mean((np.asarray(X)[1:] - np.asarray(ref)[1:]) ** 2)
    return 10.0 * math.log10(peak * peak / mse) if mse > 0 else math.inf
