"""The allocation-free quaternion GEMM (qpinv_qgemm_noalloc) against the FP64
oracle product on the same inputs, through the C ABI.  It serves callers that
cannot allocate device memory when they need a product (code inside a memory
pool or arena that forbids new cudaMalloc calls, loops that must not touch the
allocator after start-up, callers without a library context).  It keeps its
scratch in one fixed device array shared by every call, so each case makes two
calls in a row with different inputs into NaN-filled outputs: the second
result must not depend on what the first left behind.  The tolerances are the
BF16-split bounds of the other tensor-core GEMM tests.  This file is collected
last on purpose."""
import numpy as np
import pytest

import oracle
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("L", [1, 2, 3])
@pytest.mark.parametrize("m,k,n", [(200, 130, 90), (256, 256, 256), (1, 1, 1), (37, 256, 5)])
def test_noalloc_matches_oracle_twice(qp, L, m, k, n):
    for call, seed in enumerate((11, 12)):
        A = I.gaussian_quaternion(m, k, seed)
        B = I.gaussian_quaternion(k, n, seed + 50)
        C = torch.full((4, m, n), float("nan"), dtype=torch.float64, device="cuda")
        rc = qp.qpinv_qgemm_noalloc(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, split_level=L)
        assert rc == 0, (call, rc)
        got = C.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = rel(got, oracle.matmul(A, B))
        assert err <= GEMM_TOL[L], (call, err)


def test_noalloc_rejects_oversize_and_host_pointers(qp):
    big = qp.NOALLOC_MAX_DIM + 1
    A = torch.zeros((4, big, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((4, 8, 8), dtype=torch.float64, device="cuda")
    C = torch.zeros((4, big, 8), dtype=torch.float64, device="cuda")
    assert qp.qpinv_qgemm_noalloc(A, B, C) == -7
    Ah = np.zeros((4, 8, 8))
    Ch = np.zeros((4, 8, 8))
    assert qp.qpinv_qgemm_noalloc(Ah, np.zeros((4, 8, 8)), Ch) == -1
