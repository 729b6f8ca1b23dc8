"""Host-side helpers of bench.py (no GPU): the roofline entries computed from
kernel statistics, the SSIM used to report image quality, and the
workload description."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def stats(emu_n=0, emu_ms=0.0, emu_fl=0.0, emu_iss=0.0, tc_n=0, tc_ms=0.0, tc_fl=0.0, tc_iss=0.0):
    return {"emu_gemm_launches": emu_n, "emu_gemm_ms": emu_ms, "emu_gemm_flops": emu_fl,
            "emu_gemm_flops_issued": emu_iss, "tc_gemm_launches": tc_n, "tc_gemm_ms": tc_ms,
            "tc_gemm_flops": tc_fl, "tc_gemm_flops_issued": tc_iss}


def test_rooflines_dominant_first_and_arithmetic():
    st = stats(emu_n=10, emu_ms=100.0, emu_fl=10 * 5.5e11, emu_iss=10 * 36 * 5.5e11,
               tc_n=20, tc_ms=30.0, tc_fl=20 * 5.5e11, tc_iss=20 * 3 * 5.5e11)
    r = bench.kernel_rooflines(st)
    assert [e["kernel"].split()[0] for e in r] == ["k_qgemm_emu", "k_qgemm_tc"]
    e = r[0]
    # achieved = algorithmic flops per launch / mean launch time
    assert e["achieved"] == pytest.approx(5.5e11 / 10e-3 / 1e12)
    assert e["achieved_issued"] == pytest.approx(36 * 5.5e11 / 10e-3 / 1e12)
    assert e["frac"] == pytest.approx(e["achieved"] / e["peak"])
    assert e["bound"] == "tensor" and e["unit"] == "TFLOP/s"
    # traffic estimate scales with the issued flops of a launch
    assert e["traffic"] == pytest.approx(bench.TRAFFIC_PER_ISSUED_FLOP["k_qgemm_emu"] * 36 * 5.5e11)


def test_rooflines_without_gemm_launches():
    assert bench.kernel_rooflines(stats()) == [None]


def test_elementwise_entry_is_hbm_bytes_over_time():
    st = stats(emu_n=1, emu_ms=5.0, emu_fl=1e11, emu_iss=3.6e12)
    st.update(ew_launches=40, ew_ms=8.0, ew_bytes=16e9)
    r = bench.kernel_rooflines(st)
    e = r[-1]
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx(16e9 / 8e-3 / 1e9)  # 2000 GB/s
    assert e["frac"] == pytest.approx(e["achieved"] / e["peak"])
    assert r[0]["kernel"].startswith("k_qgemm_emu")  # GEMMs first, the HBM entry last


def test_ssim_of_identical_images_is_one_and_drops_with_noise():
    pytest.importorskip("scipy")
    rng = np.random.default_rng(0)
    A = np.zeros((4, 40, 50))
    A[1:] = rng.uniform(0, 1, (3, 40, 50))
    assert bench._ssim(A, A) == pytest.approx(1.0, abs=1e-12)
    B = A.copy()
    B[1:] += 0.2 * rng.standard_normal((3, 40, 50))
    assert bench._ssim(B, A) < 0.9


def test_paper_tables_are_consistent():
    # Example 3: unfactorized slower than factorized; Example 4: preconditioning
    # reduces both the steps and the time for every m
    s = bench.PAPER_EX3_SECONDS
    assert s["qhpim19"] > s["qhpi19"] and s["qhpim10"] > s["qsai"]
    for m, rows in bench.PAPER_KRYLOV.items():
        (it_f, t_f), (it_g, t_g), (it_pf, t_pf), (it_pg, t_pg) = rows
        assert it_pf < it_f and it_pg < it_g and t_pf < t_f and t_pg < t_g
    for dt, (qsvd, qns, qsai) in bench.PAPER_LORENZ_SECONDS.items():
        assert qsai < qns < qsvd
