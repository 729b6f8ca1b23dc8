"""FP64 CPU oracle of the global quaternion Krylov solvers with the QSAI
preconditioner (Sec. 3.5, Example 4).

TEST INFRASTRUCTURE ONLY: the tests and the CPU-baseline leg of ``bench.py``
may use this module; the product library never does.

System A X = B, A n x n, B n x m quaternion (planes (4, n, m)).  Global
methods work on whole n x m blocks with the real Frobenius inner product
<V, W> = Re tr(V^H W) = sum over the four planes of the entrywise products,
so the Krylov space K_k = span_R{R0, A R0, ..., A^{k-1} R0} has real
coefficients and the Hessenberg matrix is real:
  global Arnoldi: V_1 = R0 / beta, beta = ||R0||_F; W = A V_j;
    h_ij = <V_i, W>, W -= sum_i h_ij V_i (i = 1..j; classical Gram-Schmidt,
    applied twice); h_{j+1,j} = ||W||_F; V_{j+1} = W / h_{j+1,j};
  Gl-QGMRES: y = argmin ||beta e_1 - H_bar y||, X = X0 + sum y_j V_j;
  Gl-QFOM:   H y = beta e_1 (the square part), X = X0 + sum y_j V_j;
restarted every `restart` steps from the current X (or not at all).  The QSAI
preconditioner M is the iterate X_k of k QSAI iterations on A (Alg. 2,
X_0 = alpha A^H, safe alpha); the preconditioned system is M A X = M B.
Stop: the relative residual of the system being solved,
||B' - A' X_j||_F / ||B' - A' X_0||_F <= tol (X_0 = 0), tracked through the
Hessenberg least-squares residual and recomputed explicitly at each restart
and at the end; at most max_iter Arnoldi steps in all.
"""
import numpy as np

from . import matmul, solve


def inner(V, W):
    """Re tr(V^H W) for quaternion blocks in planes."""
    return float(np.sum(V * W))


def qsai_preconditioner(A, iters):
    """M = X_iters of QSAI (Alg. 2) from X_0 = alpha A^H, safe alpha."""
    M, _ = solve(A, "qsai", tol=0.0, max_iter=iters, stop="paper_abs")
    return M


def global_krylov(A, B, kind="gmres", restart=None, tol=1e-6, max_iter=3000, precond_iters=0):
    """Returns (X, info): info has iters (Arnoldi steps), converged, rel_res
    (of the solved system, explicit), true_rel_res (||B - A X|| / ||B||) and
    history (the relative residual estimate after every step).  restart =
    None: no restart (the basis grows up to max_iter blocks)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if precond_iters > 0:
        M = qsai_preconditioner(A, precond_iters)
        As, Bs = matmul(M, A), matmul(M, B)
    else:
        As, Bs = A, B
    cycle = max_iter if restart is None else restart
    X = np.zeros_like(Bs)
    r0 = np.linalg.norm(Bs)  # X_0 = 0
    steps, hist, converged = 0, [], r0 == 0.0
    R = Bs.copy()
    while steps < max_iter and not converged:
        beta = np.linalg.norm(R)
        if beta / r0 <= tol:
            converged = True
            break
        V = np.zeros((cycle + 1,) + Bs.shape)
        V[0] = R / beta
        H = np.zeros((cycle + 1, cycle))
        cs, sn = np.zeros(cycle), np.zeros(cycle)
        g = np.zeros(cycle + 1)
        g[0] = beta
        k = 0
        for j in range(cycle):
            W = matmul(As, V[j])
            for _ in range(2):  # classical Gram-Schmidt, applied twice
                h = np.tensordot(V[:j + 1], W, axes=([1, 2, 3], [0, 1, 2]))
                W = W - np.tensordot(h, V[:j + 1], axes=(0, 0))
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(W)
            k = j + 1
            steps += 1
            # Givens rotations reduce H_bar to upper triangular form; |g[k]|
            # is the GMRES residual, |g[k]| / |c_k| the FOM residual
            col = H[:j + 2, j].copy()
            for i in range(j):
                col[i], col[i + 1] = cs[i] * col[i] + sn[i] * col[i + 1], -sn[i] * col[i] + cs[i] * col[i + 1]
            rho = np.hypot(col[j], col[j + 1])
            cs[j], sn[j] = (col[j] / rho, col[j + 1] / rho) if rho > 0 else (1.0, 0.0)
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            res = abs(g[j + 1]) if kind == "gmres" else (abs(g[j + 1]) / abs(cs[j]) if cs[j] != 0 else np.inf)
            hist.append(res / r0)
            if res / r0 <= tol or steps >= max_iter or H[j + 1, j] == 0.0:
                break
            V[j + 1] = W / H[j + 1, j]
        if kind == "gmres":
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], beta * np.eye(k + 1)[0], rcond=None)
        else:
            y = np.linalg.solve(H[:k, :k], beta * np.eye(k)[0])
        X = X + np.tensordot(y, V[:k], axes=(0, 0))
        R = Bs - matmul(As, X)
        converged = np.linalg.norm(R) / r0 <= tol
    info = dict(iters=steps, converged=bool(converged), rel_res=float(np.linalg.norm(Bs - matmul(As, X)) / r0),
                true_rel_res=float(np.linalg.norm(B - matmul(A, X)) / np.linalg.norm(B)), history=hist)
    return X, info
