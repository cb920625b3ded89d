"""Host-side logic of bench.py that the bench line's numbers rest on, checked on the
CPU: the algorithmic FLOP model of tracking (the roofline's `achieved`), and the
clock summary that flags throttled runs (fed nvidia-smi rows as the sampler reads
them, no GPU)."""
import numpy as np

import bench


def test_flop_model_counts():
    """Per Gauss-Newton iteration 41 flop per support sample + 55 for the 4x4 solve
    (5,016 at 11x11); per level set-up 33 per sample + 10 (4,003); model 2: 24 per
    sample + 10."""
    assert bench.flops_model(5, 4) == (41 * 121 + 55, 33 * 121 + 10) == (5016, 4003)
    assert bench.flops_model(4, 2) == (24 * 81 + 10, 33 * 81 + 10)


def test_algorithmic_flops_counts_iterations_and_setups():
    """Tracked points (TRACKED or MAXITER) pay one set-up per level, lost points one."""
    iters = np.array([10, 30, 3, 0], dtype=np.uint8)
    status = np.array([0, 4, 1, 2], dtype=np.uint8)  # tracked, max-iter, lost (OOB, small eig)
    per_iter, per_setup = bench.flops_model(5, 4)
    got = bench.algorithmic_flops(iters, status, levels=5, radius=5, model=4)
    assert got == 43 * per_iter + (5 + 5 + 1 + 1) * per_setup


def sampler(rows):
    s = bench.ClockSampler(0)
    s.rows = [[x.strip() for x in r.split(",")] for r in rows]
    return s.summary()


def test_clock_summary_flags_throttling():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1950, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1390.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = sampler([ok, ok, capped])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3
    s = sampler([ok, hot, hot])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_thermal_slowdown"]
    assert sampler([])["reasons"] == ["nvidia-smi unavailable"]
