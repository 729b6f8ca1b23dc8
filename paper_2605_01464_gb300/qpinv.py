"""Thin ctypes binding of libqpinv (include/qpinv.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  The functions mirror the C entry points (qpinv_init, qpinv_solve,
qpinv_solve_batched, qpinv_free, qpinv_qgemm, qpinv_penrose, ...) and the
`Context` class wraps them for tensors.

A quaternion matrix is a (4, rows, cols) float64 array of component planes
(s, x, y, z): a CUDA torch tensor (device pointers) or a CPU torch tensor /
numpy array (host pointers; the library copies through its own device
buffers inside the call).  The library must be built (``build.py``); there is
no fallback -- a missing library raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqpinv.so")

METHODS = {"ns": 0, "qsai": 1, "qrapid": 2, "qhpi19": 3, "qhpim": 4}
PRECISION = {"fp64": 0, "mixed": 1, "tc": 2, "emu": 3}
PRECISION_NAME = {0: "fp64", 1: "mixed", 2: "tc", 3: "emu", 4: "df32"}
ALPHA = {"safe": 0, "spectral": 1, "fro": 2, "user": 3, "learned": 4}
SIDE = {"auto": 0, "right": 1, "left": 2}
STOP = {"paper_abs": 0, "rel_plateau": 1}
STATUS = {0: "converged", 1: "plateau", 2: "not_converged", 3: "diverged", 4: "nonfinite_input"}
ERRORS = {0: "ok", -1: "invalid", -2: "cuda", -3: "nomem", -4: "nonfinite", -5: "timeout", -6: "unsupported",
          -7: "noalloc_limit"}
NOALLOC_MAX_DIM = 256


class qpinv_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("split_level", ctypes.c_int), ("polish_iters", ctypes.c_int),
                ("alpha_mode", ctypes.c_int), ("alpha_user", ctypes.c_double), ("qrapid_N", ctypes.c_int),
                ("side", ctypes.c_int), ("stop_rule", ctypes.c_int), ("penrose", ctypes.c_int),
                ("profile", ctypes.c_int), ("batched_tile", ctypes.c_int), ("hyper_order", ctypes.c_int),
                ("fuse_epilogue", ctypes.c_int), ("emu_pair", ctypes.c_int), ("tc_broad", ctypes.c_int)]


class qpinv_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("tc_iters", ctypes.c_int),
                ("polish_iters", ctypes.c_int), ("alpha", ctypes.c_double), ("alpha_source", ctypes.c_int),
                ("side", ctypes.c_int), ("precision", ctypes.c_int), ("delta", ctypes.c_double),
                ("delta_rel", ctypes.c_double), ("E", ctypes.c_double * 4), ("E_rel", ctypes.c_double * 4),
                ("gemms", ctypes.c_longlong), ("time_ms", ctypes.c_double), ("alpha_fallback", ctypes.c_int)]


class qpinv_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("tc_gemm_launches", ctypes.c_longlong),
                ("tc_gemm_ms", ctypes.c_double), ("tc_gemm_flops", ctypes.c_double),
                ("tc_gemm_flops_issued", ctypes.c_double), ("f64_gemm_launches", ctypes.c_longlong),
                ("f64_gemm_ms", ctypes.c_double), ("f64_gemm_flops", ctypes.c_double),
                ("ew_launches", ctypes.c_longlong), ("ew_ms", ctypes.c_double), ("ew_bytes", ctypes.c_double),
                ("emu_gemm_launches", ctypes.c_longlong), ("emu_gemm_ms", ctypes.c_double),
                ("emu_gemm_flops", ctypes.c_double), ("emu_gemm_flops_issued", ctypes.c_double),
                ("batched_tile", ctypes.c_longlong), ("batched_tune_ms", ctypes.c_double),
                ("batched_graph_replays", ctypes.c_longlong), ("fused_epilogues", ctypes.c_longlong),
                ("penrose_reused", ctypes.c_longlong)]


class qpinv_cur_result(ctypes.Structure):
    _fields_ = [("pinv_solves", ctypes.c_int), ("pinv_iters", ctypes.c_int), ("pinv_worst_status", ctypes.c_int),
                ("pinv_max_E1_rel", ctypes.c_double), ("time_ms", ctypes.c_double)]


class qpinv_krylov_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("true_rel_res", ctypes.c_double), ("time_ms", ctypes.c_double)]


PTR4 = ctypes.c_void_p * 4
_lib = None

# every symbol include/qpinv.h declares (checked by the tests)
EXPORTS = ("qpinv_default_options", "qpinv_init", "qpinv_set_options", "qpinv_solve", "qpinv_solve_batched",
           "qpinv_free", "qpinv_last_error", "qpinv_qgemm", "qpinv_penrose", "qpinv_get_stats",
           "qpinv_reset_stats", "qpinv_qgemm_noalloc", "qpinv_alpha_features", "qpinv_alpha_train",
           "qpinv_alpha_predict", "qpinv_alpha_gradient", "qpinv_alpha_weights", "qpinv_cur_complete",
           "qpinv_toeplitz_filter", "qpinv_global_krylov")
ALPHA_NFEAT, ALPHA_NWEIGHTS, ALPHA_NTRAIN = 32, 6401, 6337


def lib():
    """Loads libqpinv.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqpinv.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
        L.qpinv_default_options.argtypes = [ctypes.POINTER(qpinv_options)]
        L.qpinv_default_options.restype = None
        L.qpinv_init.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(qpinv_options)]
        L.qpinv_set_options.argtypes = [vp, ctypes.POINTER(qpinv_options)]
        L.qpinv_solve.argtypes = [vp, vp, i, i, PTR4, l, i, d, i, PTR4, l, ctypes.POINTER(qpinv_result)]
        L.qpinv_solve_batched.argtypes = [vp, vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(vp),
                                          ctypes.POINTER(l), i, d, i, ctypes.POINTER(vp), ctypes.POINTER(l),
                                          ctypes.POINTER(qpinv_result)]
        L.qpinv_free.argtypes = [vp]
        L.qpinv_free.restype = None
        L.qpinv_last_error.argtypes = [vp]
        L.qpinv_last_error.restype = ctypes.c_char_p
        L.qpinv_qgemm.argtypes = [vp, vp, i, i, i, PTR4, l, PTR4, l, PTR4, l, i, i]
        L.qpinv_penrose.argtypes = [vp, vp, i, i, PTR4, l, PTR4, l, ctypes.POINTER(d), ctypes.POINTER(d)]
        L.qpinv_get_stats.argtypes = [vp, ctypes.POINTER(qpinv_stats)]
        L.qpinv_reset_stats.argtypes = [vp]
        L.qpinv_qgemm_noalloc.argtypes = [vp, i, i, i, PTR4, l, PTR4, l, PTR4, l, i]
        fp = ctypes.POINTER(ctypes.c_float)
        dp = ctypes.POINTER(d)
        L.qpinv_alpha_features.argtypes = [vp, vp, i, i, PTR4, l, fp, dp]
        L.qpinv_alpha_train.argtypes = [vp, vp, i, fp, fp, i, i, ctypes.c_float, ctypes.c_ulonglong, dp]
        L.qpinv_alpha_predict.argtypes = [vp, vp, fp, dp]
        L.qpinv_alpha_gradient.argtypes = [vp, vp, i, fp, fp, fp, dp]
        L.qpinv_alpha_weights.argtypes = [vp, fp, i, i]
        ip = ctypes.POINTER(i)
        L.qpinv_cur_complete.argtypes = [vp, vp, i, i, PTR4, l, vp, l, i, i, ip, ip, i, i, d, i, d, PTR4, l,
                                         ctypes.POINTER(qpinv_cur_result)]
        L.qpinv_toeplitz_filter.argtypes = [vp, vp, i, PTR4, PTR4, i, i, i, d, i, PTR4, PTR4,
                                            ctypes.POINTER(qpinv_result), dp]
        L.qpinv_global_krylov.argtypes = [vp, vp, i, i, PTR4, l, PTR4, l, i, i, i, d, i, PTR4, l,
                                          ctypes.POINTER(qpinv_krylov_result)]
        _lib = L
    return _lib


# ---------------------------------------------------------------- raw names

def qpinv_default_options():
    o = qpinv_options()
    lib().qpinv_default_options(ctypes.byref(o))
    return o


def qpinv_init(device=0, options=None):
    h = ctypes.c_void_p()
    rc = lib().qpinv_init(ctypes.byref(h), int(device), ctypes.byref(options) if options is not None else None)
    _check(None, rc, "qpinv_init")
    return h


def qpinv_free(ctx):
    lib().qpinv_free(ctx)


def qpinv_solve(ctx, stream, m, n, A, lda, method, tol, max_iter, X, ldx, result):
    return lib().qpinv_solve(ctx, stream, m, n, A, lda, method, tol, max_iter, X, ldx, ctypes.byref(result))


def qpinv_solve_batched(ctx, stream, batch, m, n, A, lda, method, tol, max_iter, X, ldx, results):
    return lib().qpinv_solve_batched(ctx, stream, batch, m, n, A, lda, method, tol, max_iter, X, ldx, results)


def qpinv_qgemm_noalloc(A, B, C, split_level=3, stream=None):
    """C = A B through the allocation-free entry point (CUDA tensors of
    shape (4, m, k), (4, k, n), (4, m, n), float64).  Returns the C-ABI code."""
    m, k = A.shape[1], A.shape[2]
    n = B.shape[2]
    pa, lda, _ka = _planes(A)
    pb, ldb, _kb = _planes(B)
    pc, ldc, _kc = _planes(C)
    return lib().qpinv_qgemm_noalloc(_stream_handle(stream), m, k, n, pa, lda, pb, ldb, pc, ldc, int(split_level))


def _check(ctx, rc, what):
    if rc != 0:
        msg = lib().qpinv_last_error(ctx).decode() if ctx is not None else ""
        raise QpinvError(rc, "%s failed: %s (%s)" % (what, ERRORS.get(rc, rc), msg))


class QpinvError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(msg)
        self.code = code


# ---------------------------------------------------------------- marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _planes(x):
    """(4, r, c) float64 array/tensor -> (PTR4, ld, keepalive)."""
    if _is_torch(x):
        assert x.dtype.is_floating_point and x.element_size() == 8 and x.dim() == 3 and x.shape[0] == 4
        assert x.stride(2) == 1 and x.stride(1) >= x.shape[2], "rows must be contiguous"
        base, es = x.data_ptr(), 8
        p = PTR4(*[base + c * x.stride(0) * es for c in range(4)])
        return p, x.stride(1), x
    a = np.asarray(x)
    assert a.dtype == np.float64 and a.ndim == 3 and a.shape[0] == 4
    if not (a.flags.c_contiguous):
        a = np.ascontiguousarray(a)
    base = a.ctypes.data
    p = PTR4(*[base + c * a.strides[0] for c in range(4)])
    return p, a.strides[1] // 8, a


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Context:
    """A libqpinv context bound to one CUDA device."""

    def __init__(self, device=0, precision="mixed", split_level=0, polish_iters=2, alpha="safe",
                 alpha_user=0.0, qrapid_N=5, side="auto", stop="rel_plateau", penrose=True, profile=False,
                 batched_tile=-1, hyper_order=19):
        self.options = qpinv_default_options()
        self.device = device
        self.configure(precision=precision, split_level=split_level, polish_iters=polish_iters, alpha=alpha,
                       alpha_user=alpha_user, qrapid_N=qrapid_N, side=side, stop=stop, penrose=penrose,
                       profile=profile, batched_tile=batched_tile, hyper_order=hyper_order, _apply=False)
        self.h = qpinv_init(device, self.options)

    def configure(self, precision=None, split_level=None, polish_iters=None, alpha=None, alpha_user=None,
                  qrapid_N=None, side=None, stop=None, penrose=None, profile=None, batched_tile=None,
                  hyper_order=None, fuse_epilogue=None, emu_pair=None, tc_broad=None, _apply=True):
        o = self.options
        if precision is not None: o.precision = PRECISION[precision]
        if split_level is not None: o.split_level = int(split_level)
        if polish_iters is not None: o.polish_iters = int(polish_iters)
        if alpha is not None: o.alpha_mode = ALPHA[alpha]
        if alpha_user is not None: o.alpha_user = float(alpha_user)
        if qrapid_N is not None: o.qrapid_N = int(qrapid_N)
        if side is not None: o.side = SIDE[side]
        if stop is not None: o.stop_rule = STOP[stop]
        if penrose is not None: o.penrose = int(bool(penrose))
        if profile is not None: o.profile = int(bool(profile))
        if batched_tile is not None: o.batched_tile = int(batched_tile)
        if hyper_order is not None: o.hyper_order = int(hyper_order)
        if fuse_epilogue is not None: o.fuse_epilogue = int(bool(fuse_epilogue))
        if emu_pair is not None: o.emu_pair = -1 if emu_pair == "auto" else int(bool(emu_pair))
        if tc_broad is not None: o.tc_broad = -1 if tc_broad == "auto" else int(bool(tc_broad))
        if _apply:
            _check(self.h, lib().qpinv_set_options(self.h, ctypes.byref(o)), "qpinv_set_options")

    def close(self):
        if getattr(self, "h", None):
            qpinv_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, A, method="qhpi19", tol=1e-12, max_iter=500, X=None, stream=None):
        """Returns (X, info).  X is allocated like A (same device) unless given."""
        m, n = A.shape[1], A.shape[2]
        if X is None:
            if _is_torch(A):
                import torch
                X = torch.empty((4, n, m), dtype=torch.float64, device=A.device)
            else:
                X = np.empty((4, n, m))
        pa, lda, ka = _planes(A)
        px, ldx, kx = _planes(X)
        res = qpinv_result()
        rc = qpinv_solve(self.h, _stream_handle(stream), m, n, pa, lda, METHODS[method], float(tol),
                         int(max_iter), px, ldx, res)
        _check(self.h, rc, "qpinv_solve")
        if kx is not X:  # host copy made for contiguity
            X[...] = kx
        return X, result_dict(res)

    def cur_complete(self, M, mask, I, J, method="qhpi19", tol=1e-12, max_iter=200, sigma=0.5, cross=False,
                     C=None, stream=None):
        """CUR image completion (qpinv_cur_complete).  M: (4, m, n) planes;
        mask: (m, n) uint8 (nonzero = observed), a tensor on M's device or a
        numpy array; I, J: (iters, r) integer index sets.  Returns (C, info)."""
        m, n = M.shape[1], M.shape[2]
        I = np.ascontiguousarray(I, dtype=np.int32)
        J = np.ascontiguousarray(J, dtype=np.int32)
        assert I.shape == J.shape and I.ndim == 2
        iters, r = I.shape
        if C is None:
            if _is_torch(M):
                import torch
                C = torch.empty((4, m, n), dtype=torch.float64, device=M.device)
            else:
                C = np.empty((4, m, n))
        pm, ldm, km = _planes(M)
        pc, ldc, kc = _planes(C)
        if _is_torch(mask):
            assert mask.dtype.itemsize == 1 and mask.stride(1) == 1
            mp, ldk = mask.data_ptr(), mask.stride(0)
        else:
            mask = np.ascontiguousarray(mask, dtype=np.uint8)
            mp, ldk = mask.ctypes.data, mask.shape[1]
        res = qpinv_cur_result()
        ip = ctypes.POINTER(ctypes.c_int)
        rc = lib().qpinv_cur_complete(self.h, _stream_handle(stream), m, n, pm, ldm, mp, ldk, r, iters,
                                      I.ctypes.data_as(ip), J.ctypes.data_as(ip), 1 if cross else 0,
                                      METHODS[method], float(tol), int(max_iter), float(sigma), pc, ldc,
                                      ctypes.byref(res))
        _check(self.h, rc, "qpinv_cur_complete")
        if kc is not C:
            C[...] = kc
        return C, dict(pinv_solves=res.pinv_solves, pinv_iters=res.pinv_iters,
                       pinv_worst_status=STATUS.get(res.pinv_worst_status, res.pinv_worst_status),
                       pinv_max_E1_rel=res.pinv_max_E1_rel, time_ms=res.time_ms)

    def toeplitz_filter(self, x, s, p, t0=None, method="qsai", tol=1e-12, max_iter=500, stream=None):
        """Quaternion filter design (qpinv_toeplitz_filter).  x, s: (4, N)
        sample planes (tensors or numpy arrays); t0 defaults to p.  Returns
        (h, s_hat, err, info of the pseudoinverse solve); h and s_hat are
        (4, p + 1, 1), allocated like x."""
        N = x.shape[1]
        t0 = p if t0 is None else t0
        if _is_torch(x):
            import torch
            h = torch.empty((4, p + 1, 1), dtype=torch.float64, device=x.device)
            sh = torch.empty_like(h)
        else:
            h, sh = np.empty((4, p + 1, 1)), np.empty((4, p + 1, 1))
        px, _, kx = _planes(x[:, None, :])
        ps, _, ks = _planes(s[:, None, :])
        ph, _, kh = _planes(h)
        psh, _, ksh = _planes(sh)
        res, err = qpinv_result(), ctypes.c_double()
        rc = lib().qpinv_toeplitz_filter(self.h, _stream_handle(stream), N, px, ps, int(p), int(t0), METHODS[method],
                                         float(tol), int(max_iter), ph, psh, ctypes.byref(res), ctypes.byref(err))
        _check(self.h, rc, "qpinv_toeplitz_filter")
        return h, sh, err.value, result_dict(res)

    def global_krylov(self, A, B, kind="gmres", restart=0, precond_iters=0, tol=1e-6, max_iter=3000, X=None,
                      stream=None):
        """Gl-QGMRES / Gl-QFOM (qpinv_global_krylov) for A X = B; restart 0 =
        none; precond_iters > 0: QSAI left preconditioner.  Returns (X, info)."""
        n, m = A.shape[1], B.shape[2]
        if X is None:
            if _is_torch(B):
                import torch
                X = torch.empty((4, n, m), dtype=torch.float64, device=B.device)
            else:
                X = np.empty((4, n, m))
        pa, lda, ka = _planes(A)
        pb, ldb, kb = _planes(B)
        px, ldx, kx = _planes(X)
        res = qpinv_krylov_result()
        rc = lib().qpinv_global_krylov(self.h, _stream_handle(stream), n, m, pa, lda, pb, ldb,
                                       0 if kind == "gmres" else 1, int(restart), int(precond_iters), float(tol),
                                       int(max_iter), px, ldx, ctypes.byref(res))
        _check(self.h, rc, "qpinv_global_krylov")
        if kx is not X:
            X[...] = kx
        return X, dict(iters=res.iters, converged=bool(res.converged), rel_res=res.rel_res,
                       true_rel_res=res.true_rel_res, time_ms=res.time_ms)

    def solve_batched(self, As, method="qhpi19", tol=1e-6, max_iter=100, Xs=None, stream=None):
        import torch
        b = len(As)
        if Xs is None:
            Xs = [torch.empty((4, a.shape[2], a.shape[1]), dtype=torch.float64, device=a.device) for a in As]
        m = (ctypes.c_int * b)(*[a.shape[1] for a in As])
        n = (ctypes.c_int * b)(*[a.shape[2] for a in As])
        ap = (ctypes.c_void_p * (4 * b))()
        xp = (ctypes.c_void_p * (4 * b))()
        lda = (ctypes.c_long * b)()
        ldx = (ctypes.c_long * b)()
        for t, (a, x) in enumerate(zip(As, Xs)):
            pa, la, _ = _planes(a)
            px, lx, _ = _planes(x)
            for c in range(4):
                ap[4 * t + c] = pa[c]
                xp[4 * t + c] = px[c]
            lda[t], ldx[t] = la, lx
        res = (qpinv_result * b)()
        rc = qpinv_solve_batched(self.h, _stream_handle(stream), b, m, n, ap, lda, METHODS[method], float(tol),
                                 int(max_iter), xp, ldx, res)
        _check(self.h, rc, "qpinv_solve_batched")
        return Xs, [result_dict(r) for r in res]

    def qgemm(self, A, B, precision="tc", split_level=3, C=None, stream=None):
        m, k = A.shape[1], A.shape[2]
        n = B.shape[2]
        if C is None:
            if _is_torch(A):
                import torch
                C = torch.empty((4, m, n), dtype=torch.float64, device=A.device)
            else:
                C = np.empty((4, m, n))
        pa, lda, _ka = _planes(A)
        pb, ldb, _kb = _planes(B)
        pc, ldc, _kc = _planes(C)
        rc = lib().qpinv_qgemm(self.h, _stream_handle(stream), m, k, n, pa, lda, pb, ldb, pc, ldc,
                               PRECISION[precision], int(split_level))
        _check(self.h, rc, "qpinv_qgemm")
        return C

    def penrose(self, A, X, stream=None):
        m, n = A.shape[1], A.shape[2]
        pa, lda, _ka = _planes(A)
        px, ldx, _kx = _planes(X)
        E = (ctypes.c_double * 4)()
        R = (ctypes.c_double * 4)()
        rc = lib().qpinv_penrose(self.h, _stream_handle(stream), m, n, pa, lda, px, ldx, E, R)
        _check(self.h, rc, "qpinv_penrose")
        return list(E), list(R)

    # ---- learned alpha ----
    def alpha_features(self, A, stream=None):
        """(features[32] float32, theta_1) of A."""
        m, n = A.shape[1], A.shape[2]
        pa, lda, _ka = _planes(A)
        f = np.zeros(ALPHA_NFEAT, dtype=np.float32)
        t1 = ctypes.c_double()
        rc = lib().qpinv_alpha_features(self.h, _stream_handle(stream), m, n, pa, lda, _fptr(f), ctypes.byref(t1))
        _check(self.h, rc, "qpinv_alpha_features")
        return f, t1.value

    def alpha_train(self, feats, labels, epochs=200, batch=128, lr=1e-3, seed=0, stream=None):
        X = np.ascontiguousarray(feats, dtype=np.float32)
        T = np.ascontiguousarray(labels, dtype=np.float32)
        assert X.ndim == 2 and X.shape[1] == ALPHA_NFEAT and T.shape == (X.shape[0],)
        loss = ctypes.c_double()
        rc = lib().qpinv_alpha_train(self.h, _stream_handle(stream), X.shape[0], _fptr(X), _fptr(T), int(epochs),
                                     int(batch), float(lr), int(seed), ctypes.byref(loss))
        _check(self.h, rc, "qpinv_alpha_train")
        return loss.value

    def alpha_predict(self, feat, stream=None):
        f = np.ascontiguousarray(feat, dtype=np.float32)
        y = ctypes.c_double()
        _check(self.h, lib().qpinv_alpha_predict(self.h, _stream_handle(stream), _fptr(f), ctypes.byref(y)),
               "qpinv_alpha_predict")
        return y.value

    def alpha_gradient(self, feats, labels, stream=None):
        X = np.ascontiguousarray(feats, dtype=np.float32)
        T = np.ascontiguousarray(labels, dtype=np.float32)
        g = np.zeros(ALPHA_NTRAIN, dtype=np.float32)
        loss = ctypes.c_double()
        rc = lib().qpinv_alpha_gradient(self.h, _stream_handle(stream), X.shape[0], _fptr(X), _fptr(T), _fptr(g),
                                        ctypes.byref(loss))
        _check(self.h, rc, "qpinv_alpha_gradient")
        return g, loss.value

    def alpha_weights(self, w=None):
        """Returns the weight block, or loads `w` (QPINV_ALPHA_NWEIGHTS floats)."""
        if w is None:
            out = np.zeros(ALPHA_NWEIGHTS, dtype=np.float32)
            _check(self.h, lib().qpinv_alpha_weights(self.h, _fptr(out), ALPHA_NWEIGHTS, 0), "qpinv_alpha_weights")
            return out
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(self.h, lib().qpinv_alpha_weights(self.h, _fptr(w), ALPHA_NWEIGHTS, 1), "qpinv_alpha_weights")
        return w

    def stats(self):
        s = qpinv_stats()
        _check(self.h, lib().qpinv_get_stats(self.h, ctypes.byref(s)), "qpinv_get_stats")
        return {f: getattr(s, f) for f, _ in qpinv_stats._fields_}

    def reset_stats(self):
        _check(self.h, lib().qpinv_reset_stats(self.h), "qpinv_reset_stats")


def result_dict(r):
    return dict(status=STATUS.get(r.status, r.status), iters=r.iters, tc_iters=r.tc_iters,
                polish_iters=r.polish_iters, alpha=r.alpha, alpha_source=r.alpha_source,
                side="left" if r.side == 2 else "right", precision=PRECISION_NAME.get(r.precision, r.precision),
                delta=r.delta, delta_rel=r.delta_rel,
                E=list(r.E), E_rel=list(r.E_rel), gemms=r.gemms, time_ms=r.time_ms,
                alpha_fallback=r.alpha_fallback)
