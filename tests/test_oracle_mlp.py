"""Pins of the FP64 reference network used to check the GPU learned-alpha
kernels: the chain-rule gradient against central differences, a closed form
of the forward pass, the optimal alpha of Thm. 1 against a brute-force scan,
and complete Lanczos runs against LAPACK eigenvalues."""
import numpy as np
import pytest

from oracle import mlp
from paper_2605_01464_gb300 import inputs as I


def random_weights(seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(0, 0.3, mlp.NWEIGHTS)
    w[mlp.OFF_MU:mlp.OFF_SD] = rng.normal(0, 1, mlp.NF)
    w[mlp.OFF_SD:] = rng.uniform(0.5, 2.0, mlp.NF)
    return w


def test_gradient_matches_central_differences():
    w = random_weights(1)
    rng = np.random.default_rng(2)
    X, T = rng.normal(size=(17, mlp.NF)), rng.normal(size=17)
    g = mlp.gradient(w, X, T)
    idx = list(rng.choice(mlp.NTRAIN, 60, replace=False)) + [mlp.OFF_B3, mlp.OFF_W3, mlp.OFF_B1, mlp.OFF_B2]
    num = mlp.numeric_gradient(w, X, T, idx)
    assert np.allclose(g[idx], num, rtol=1e-6, atol=1e-9)


def test_forward_closed_form_with_zero_matrices():
    w = random_weights(3)
    w[mlp.OFF_W1:mlp.OFF_B1] = 0.0
    w[mlp.OFF_W2:mlp.OFF_B2] = 0.0
    p = mlp.unpack(w)
    y, _ = mlp.forward(w, np.ones((3, mlp.NF)))
    assert np.allclose(y, p["b3"] + p["w3"] @ np.tanh(p["b2"]))


def test_optimal_alpha_minimises_thm1_radius():
    sigma = np.array([2.0, 1.3, 0.4, 0.05])
    a_star = mlp.optimal_alpha(sigma)
    grid = np.linspace(1e-4, 2.0 / sigma.max() ** 2, 20001)
    rho = np.max(np.abs(1.0 - grid[:, None] * sigma[None, :] ** 2), axis=1)
    assert abs(grid[np.argmin(rho)] - a_star) <= 2 * (grid[1] - grid[0])


def test_complete_lanczos_gives_the_spectrum():
    A = I.gaussian_quaternion(9, 6, 4)
    C = I.chi(A)
    start = np.random.default_rng(5).normal(size=12) + 1j * np.random.default_rng(6).normal(size=12)
    ritz = mlp.lanczos_ritz(C, 6, start)  # 6 distinct eigenvalues: the Krylov space is exhausted
    ev = np.sort(np.linalg.eigvalsh(C.conj().T @ C))[::-1][::2]  # each quaternion eigenvalue twice
    assert np.allclose(ritz[:6], ev, rtol=1e-8)
