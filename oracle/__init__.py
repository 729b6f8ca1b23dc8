"""FP64 CPU oracle for the quaternion hyperpower pseudoinverse iterations.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never does.  The arithmetic lives in ``qoracle.c`` (plain C, FP64, its own
scalar quaternion type); this module only marshals numpy arrays.

Matrices cross this interface as ``(4, rows, cols)`` float64 arrays of real
component planes (s, x, y, z) -- the same convention the inputs module uses.
Internally the C code stores interleaved quaternion structs.
"""
import ctypes
import os

import numpy as np

from . import build as _build

METHODS = {"ns": 0, "qsai": 1, "qrapid": 2, "qhpi19": 3, "qhpim": 4}
ALPHA = {"safe": 0, "spectral": 1, "fro": 2, "user": 3}
STOP = {"paper_abs": 0, "rel_plateau": 1}
STATUS = {0: "converged", 1: "plateau", 2: "not_converged", 3: "diverged"}


class QoResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("alpha", ctypes.c_double), ("delta", ctypes.c_double),
                ("delta_rel", ctypes.c_double), ("E", ctypes.c_double * 4),
                ("E_rel", ctypes.c_double * 4), ("gemms", ctypes.c_longlong)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(ctypes.c_double)
        i, d = ctypes.c_int, ctypes.c_double
        L.qo_qmul.argtypes = [P, P, P]
        L.qo_matmul.argtypes = [i, i, i, P, P, P]
        L.qo_adjoint.argtypes = [i, i, P, P]
        L.qo_norms.argtypes = [i, i, P, P]
        L.qo_sigma_max.argtypes = [i, i, P]
        L.qo_sigma_max.restype = d
        L.qo_alpha.argtypes = [i, i, P, i, d]
        L.qo_alpha.restype = d
        L.qo_init_x0.argtypes = [i, i, P, d, P]
        L.qo_step.argtypes = [i, i, P, P, i, i, i, P]
        L.qo_penrose.argtypes = [i, i, P, P, P, P]
        L.qo_solve.argtypes = [i, i, P, i, i, i, d, i, d, i, i, P, P, P,
                               ctypes.POINTER(QoResult)]
        L.qo_pinv_from_svd.argtypes = [i, i, i, P, P, P, P]
        L.qo_constants.argtypes = [P]
        L.qo_gemm_count.restype = ctypes.c_longlong
        L.qo_set_mutation.argtypes = [i]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _to_q(planes):
    """(4, r, c) planes -> C-contiguous (r, c, 4) interleaved quaternions."""
    planes = np.asarray(planes, dtype=np.float64)
    assert planes.ndim == 3 and planes.shape[0] == 4, planes.shape
    return np.ascontiguousarray(planes.transpose(1, 2, 0))


def _from_q(q):
    return np.ascontiguousarray(q.transpose(2, 0, 1))


def qmul(p, q):
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.zeros(4)
    lib().qo_qmul(_ptr(p), _ptr(q), _ptr(r))
    return r


def matmul(A, B):
    a, b = _to_q(A), _to_q(B)
    m, k = a.shape[:2]
    assert b.shape[0] == k
    n = b.shape[1]
    c = np.zeros((m, n, 4))
    lib().qo_matmul(m, k, n, _ptr(a), _ptr(b), _ptr(c))
    return _from_q(c)


def adjoint(A):
    a = _to_q(A)
    m, n = a.shape[:2]
    h = np.zeros((n, m, 4))
    lib().qo_adjoint(m, n, _ptr(a), _ptr(h))
    return _from_q(h)


def norms(A):
    """(||A||_1, ||A||_inf, ||A||_F) with quaternion moduli."""
    a = _to_q(A)
    out = np.zeros(3)
    lib().qo_norms(a.shape[0], a.shape[1], _ptr(a), _ptr(out))
    return tuple(out)


def sigma_max(A):
    a = _to_q(A)
    return lib().qo_sigma_max(a.shape[0], a.shape[1], _ptr(a))


def alpha(A, mode="safe", user=0.0):
    a = _to_q(A)
    return lib().qo_alpha(a.shape[0], a.shape[1], _ptr(a), ALPHA[mode], float(user))


def init_x0(A, alpha_value):
    a = _to_q(A)
    m, n = a.shape[:2]
    x = np.zeros((n, m, 4))
    lib().qo_init_x0(m, n, _ptr(a), float(alpha_value), _ptr(x))
    return _from_q(x)


def _param(method, N, order):
    """The C interface's method parameter: QRAPID's N, or QHPIM's order k."""
    return int(order if method == "qhpim" else N)


def step(A, X, method="qhpi19", N=5, side="right", order=19):
    a, x = _to_q(A), _to_q(X)
    m, n = a.shape[:2]
    assert x.shape[:2] == (n, m)
    y = np.zeros((n, m, 4))
    lib().qo_step(m, n, _ptr(a), _ptr(x), METHODS[method], _param(method, N, order),
                  int(side == "left"), _ptr(y))
    return _from_q(y)


def penrose(A, X):
    """Returns (E[4], E_rel[4]): ||AXA-A||, ||XAX-X||, ||(AX)^H-AX||, ||(XA)^H-XA||
    (Frobenius), and the same divided by ||A||, ||X||, ||AX||, ||XA||."""
    a, x = _to_q(A), _to_q(X)
    E, R = np.zeros(4), np.zeros(4)
    lib().qo_penrose(a.shape[0], a.shape[1], _ptr(a), _ptr(x), _ptr(E), _ptr(R))
    return E, R


def solve(A, method="qhpi19", tol=1e-12, max_iter=500, alpha_mode="safe", alpha_user=0.0,
          stop="rel_plateau", side="right", N=5, x0=None, trace=False, order=19):
    """Runs the chosen iteration to the stop rule.  Returns (X, info).
    N: QRAPID's step parameter; order: the order k of QHPIM."""
    a = _to_q(A)
    m, n = a.shape[:2]
    x = np.zeros((n, m, 4))
    res = QoResult()
    tr = np.full(max(max_iter, 1), np.nan)
    x0p = None
    if x0 is not None:
        x0q = _to_q(x0)
        x0p = _ptr(x0q)
    lib().qo_solve(m, n, _ptr(a), METHODS[method], _param(method, N, order), ALPHA[alpha_mode],
                   float(alpha_user), STOP[stop], float(tol), int(max_iter), int(side == "left"), x0p, _ptr(x),
                   _ptr(tr), ctypes.byref(res))
    info = dict(status=STATUS[res.status], iters=res.iters, alpha=res.alpha, delta=res.delta,
                delta_rel=res.delta_rel, E=list(res.E), E_rel=list(res.E_rel), gemms=res.gemms)
    if trace:
        info["delta_trace"] = tr[: max_iter]
    return _from_q(x), info


def pinv_from_svd(U, sigma, V):
    """A^dagger = V Sigma^dagger U^H for A = U diag(sigma) V^H (U: (4,m,r), V: (4,n,r))."""
    u, v = _to_q(U), _to_q(V)
    m, r = u.shape[:2]
    n = v.shape[0]
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    assert s.shape == (r,) and v.shape[1] == r
    x = np.zeros((n, m, 4))
    lib().qo_pinv_from_svd(m, n, r, _ptr(u), _ptr(s), _ptr(v), _ptr(x))
    return _from_q(x)


CONSTANT_NAMES = ("beta1", "beta2", "a1", "a2", "a3", "b1", "b2", "c1", "c2",
                  "d1", "d2", "d3", "e1", "e2")


def constants():
    out = np.zeros(14)
    lib().qo_constants(_ptr(out))
    return dict(zip(CONSTANT_NAMES, out))


def gemm_count():
    return lib().qo_gemm_count()


def set_mutation(k):
    """Plants a known mistake in the oracle (0 = none).  Tests only."""
    lib().qo_set_mutation(int(k))
