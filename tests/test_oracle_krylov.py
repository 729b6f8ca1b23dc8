"""Pins of the global Krylov oracle (Gl-QGMRES / Gl-QFOM with the QSAI
preconditioner): the minimal-residual and Galerkin definitions checked by
brute force over the real Krylov space, one-step convergence with an exact
preconditioner, monotone GMRES residuals, restart equivalence, and
convergence on a small reservoir system.  A planted mistake shows the pins
bite."""
import numpy as np
import pytest

import oracle
from oracle import krylov
from paper_2605_01464_gb300 import inputs as I


def small_system(n=12, m=2, seed=3):
    A = I.gaussian_quaternion(n, n, seed)
    A[0] += 3.0 * np.sqrt(n) * np.eye(n)  # well conditioned, nonsymmetric
    B = I.gaussian_quaternion(n, m, seed + 1)
    return A, B


def krylov_basis(A, R0, k):
    K = [R0]
    for _ in range(k - 1):
        K.append(oracle.matmul(A, K[-1]))
    return np.stack([v.ravel() for v in K], axis=1)  # real coefficients


def check_gmres_minimal_residual(k=5):
    A, B = small_system()
    X, info = krylov.global_krylov(A, B, "gmres", restart=None, tol=0.0, max_iter=k)
    assert info["iters"] == k
    K = krylov_basis(A, B, k)
    AK = np.stack([oracle.matmul(A, K[:, i].reshape(B.shape)).ravel() for i in range(k)], axis=1)
    c, *_ = np.linalg.lstsq(AK, B.ravel(), rcond=None)
    want = (K @ c).reshape(B.shape)
    assert np.linalg.norm(X - want) <= 1e-10 * np.linalg.norm(want), np.linalg.norm(X - want)


def check_fom_galerkin(k=5):
    A, B = small_system(seed=7)
    X, info = krylov.global_krylov(A, B, "fom", restart=None, tol=0.0, max_iter=k)
    K = krylov_basis(A, B, k)
    AK = np.stack([oracle.matmul(A, K[:, i].reshape(B.shape)).ravel() for i in range(k)], axis=1)
    c = np.linalg.solve(K.T @ AK, K.T @ B.ravel())  # <K_i, B - A K c> = 0
    want = (K @ c).reshape(B.shape)
    assert np.linalg.norm(X - want) <= 1e-9 * np.linalg.norm(want)


def test_gmres_is_the_minimal_residual_iterate():
    check_gmres_minimal_residual()


def test_fom_satisfies_the_galerkin_condition():
    check_fom_galerkin()


def test_gmres_residual_history_is_monotone():
    A, B = small_system(n=20, seed=11)
    _, info = krylov.global_krylov(A, B, "gmres", restart=None, tol=1e-12, max_iter=60)
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-12) and info["converged"]


def test_restart_longer_than_the_run_changes_nothing():
    A, B = small_system(n=16, seed=13)
    X1, i1 = krylov.global_krylov(A, B, "gmres", restart=None, tol=0.0, max_iter=8)
    X2, i2 = krylov.global_krylov(A, B, "gmres", restart=50, tol=0.0, max_iter=8)
    assert np.array_equal(X1, X2)


def test_exact_preconditioner_converges_in_one_step():
    # 40 QSAI iterations make M = A^-1 to rounding: M A = I
    A, B = small_system(n=10, seed=17)
    X, info = krylov.global_krylov(A, B, "gmres", tol=1e-10, max_iter=50, precond_iters=40)
    assert info["iters"] == 1 and info["true_rel_res"] <= 1e-12, info


@pytest.mark.parametrize("kind", ["gmres", "fom"])
@pytest.mark.parametrize("precond", [0, 2])
def test_small_reservoir_system_converges(kind, precond):
    A, B = I.krylov_system(m=2, nx=6, ny=7)
    X, info = krylov.global_krylov(A, B, kind, tol=1e-8, max_iter=500, precond_iters=precond)
    assert info["converged"] and info["rel_res"] <= 1e-8, info
    if precond == 0:
        assert abs(info["true_rel_res"] - info["rel_res"]) <= 1e-12


def test_system_structure():
    A, B = I.krylov_system(m=4)
    assert A.shape == (4, 238, 238) and B.shape == (4, 238, 4)
    assert np.array_equal(A[1], -A[0]) and np.array_equal(A[2], 2 * A[0]) and np.array_equal(A[3], 1.5 * A[0])
    assert B.min() >= 0.0 and B.max() < 1.0


def test_planted_mistake_is_caught(monkeypatch):
    # an inner product that ignores the imaginary planes
    monkeypatch.setattr(np, "tensordot", _real_plane_tensordot)
    with pytest.raises(AssertionError):
        check_gmres_minimal_residual()


_tensordot = np.tensordot


def _real_plane_tensordot(a, b, axes=2):
    if axes == ([1, 2, 3], [0, 1, 2]):
        return _tensordot(a[:, :1], b[:1], axes=axes)
    return _tensordot(a, b, axes=axes)
