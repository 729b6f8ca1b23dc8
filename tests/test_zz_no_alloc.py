"""The allocation-free quaternion GEMM (qpinv_qgemm_noalloc) against the
context-based tensor-core GEMM (qpinv_qgemm, QPINV_PREC_TC) on the same
inputs, through the C ABI.  It keeps its scratch in one fixed device array
shared by every call, so each case makes two calls in a row with different
inputs: the second result must not depend on what the first left behind.
This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2605_01464_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GEMM_TOL = {1: 1e-2, 2: 3e-4, 3: 5e-5}  # same bounds as the other tensor-core GEMM tests


@pytest.fixture(scope="module")
def qp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_01464_gb300 import build, qpinv
    build.build()
    return qpinv


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("m,k,n", [(200, 130, 90), (256, 256, 256), (1, 1, 1), (37, 256, 5)])
def test_noalloc_matches_context_gemm_twice(qp, L, m, k, n):
    ctx = qp.Context(0)
    try:
        for call, seed in enumerate((11, 12)):
            A = torch.from_numpy(I.gaussian_quaternion(m, k, seed)).cuda()
            B = torch.from_numpy(I.gaussian_quaternion(k, n, seed + 50)).cuda()
            C = torch.full((4, m, n), float("nan"), dtype=torch.float64, device="cuda")
            rc = qp.qpinv_qgemm_noalloc(A, B, C, split_level=L)
            assert rc == 0, (call, rc)
            ref = ctx.qgemm(A, B, precision="tc", split_level=L)
            assert torch.isfinite(C).all()
            assert rel(C, ref) <= GEMM_TOL[L], (call, rel(C, ref))
    finally:
        ctx.close()


def test_noalloc_rejects_oversize_and_host_pointers(qp):
    big = qp.NOALLOC_MAX_DIM + 1
    A = torch.zeros((4, big, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((4, big, 8), dtype=torch.float64, device="cuda")
    assert qp.qpinv_qgemm_noalloc(A, B, C) == -7
    Ah = np.zeros((4, 8, 8))
    Ch = np.zeros((4, 8, 8))
    assert qp.qpinv_qgemm_noalloc(Ah, np.zeros((4, 8, 8)), Ch) == -1
