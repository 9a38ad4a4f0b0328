"""Host-side helpers of bench.py: the success criteria of Section 4.2 on hand-made fits, and the
whole-job rate."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_success_criteria_by_hand():
    truth = np.array([[0.0, 20.0, 0.2, 6.2, 1.0, 0.5]] * 4)
    best = truth.copy()
    best[1, 3] = 0.1  # alpha wraps: 6.2 -> 0.1 is 0.183 rad, 2.9% of 2 pi
    best[2, 0] = 2.5  # t0 off by 2.5 d = 12.5% of tE
    best[3, 5] = 0.56  # q off by 12%
    chi_true = np.array([100.0, 100.0, 100.0, 100.0])
    chi = np.array([100.5, 150.0, 190.0, 201.0])  # delta chi^2 0.5, 50, 90, 101 with nu = 100 - 6 = 94
    s = bench._success(best, chi, chi_true, truth, 100)
    assert s["dchi2_per_dof_lt_1"] == 0.75  # 101/94 > 1 fails
    assert s["dchi2_le_1"] == 0.25
    assert s["strict"] == 0.5  # rows 0 and 1; row 2 fails on t0, row 3 on chi^2


def test_whole_job_rate():
    # units processed by all ranks over the slowest rank's time per step
    assert bench.whole_job_rate(4, 1000, 2.0) == 4 * 1000 / 2.0 * 1e3


def test_pipe_time_fraction():
    # 80 TFLOP of FP32 at 80 TFLOP/s is 1 s, 1.25 TFLOP of FP64 at 1.25 TFLOP/s another 1 s: at
    # those peaks the pass would take 2 s; measured 8 s gives 0.25
    assert bench.pipe_time_fraction(80e12, 1.25e12, 80.0, 1.25, 8.0) == 0.25
    # no FP64 work: the plain FP32 fraction
    assert bench.pipe_time_fraction(40e12, 0.0, 80.0, 1.25, 1.0) == 0.5


def test_budget_runs_what_fits_and_reports_the_rest():
    import time

    out = {}
    b = bench.Budget(time.perf_counter() + 10.0)
    assert b.run(out, "small", 1.0, lambda: {"ok": 1}) == {"ok": 1}
    assert b.run(out, "large", 100.0, lambda: {"ok": 2}) is None
    assert out["small"] == {"ok": 1} and out["large"]["skipped"].startswith("time budget")

    def fails():
        raise ValueError("boom")

    b.run(out, "broken", 1.0, fails)  # a failing section is reported, not raised
    assert out["broken"] == {"error": "ValueError: boom"}
