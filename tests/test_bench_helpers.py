"""Host logic of bench.py (no GPU): the expected pair count of the roofline
(the probability that two uniform points of the unit cube lie within r),
the FP32 rounding that keeps points inside the half-open box, and the
clock-sample summary (samples taken during the timed region, throttle
reasons)."""
from __future__ import annotations

import os

import numpy as np

import bench


def test_pair_fraction_matches_monte_carlo():
    rng = np.random.default_rng(11)
    n = 2_000_000
    d = np.linalg.norm(rng.random((n, 3)) - rng.random((n, 3)), axis=1)
    for r in (0.05, 0.1, 0.3):
        p = bench.pair_fraction_unit_cube(r)
        mc = float((d <= r).mean())
        assert abs(mc - p) <= 5.0 * np.sqrt(p / n) + 1e-7, (r, mc, p)
    # small r: the boundary terms vanish against the ball volume
    r = 1e-3
    assert abs(bench.pair_fraction_unit_cube(r) / (4 * np.pi / 3 * r**3) - 1.0) < 2e-3
    # r = 1 keeps the polynomial's value at the cube's side
    assert 0.0 < bench.pair_fraction_unit_cube(1.0) < 1.0


def test_f32_in_box_stays_in_the_half_open_box():
    x = np.array([[0.0, 0.5, 1.0 - 1e-12], [1.0 - 1e-9, 0.25, 0.999999999]])
    y = bench.f32_in_box(x)
    assert y.dtype == np.float32
    assert np.all(y >= 0.0) and np.all(y < 1.0)
    np.testing.assert_allclose(y, x.astype(np.float32), atol=1e-7)


def test_clock_summary_keeps_the_timed_samples(tmp_path):
    cs = bench.ClockSampler(0)
    cs.proc = object()  # as if nvidia-smi were running
    lines = ["0, 1800, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active"] * 2 + \
            ["0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active"] * 3
    with open(cs.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs.skip = 2  # two samples were there before the timed region
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(cs.path)
