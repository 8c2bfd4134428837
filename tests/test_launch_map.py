"""Host logic of the launch-condition map (Section 5, Table 1's power-law fit)."""
import math

import pytest

from paper_1811_08282_gb300 import launch_map as LM


def test_power_fit_recovers_exact_power_law():
    xs = [2.0 ** e for e in range(14, 25)]
    ys = [1.33e-4 * x ** 0.937 for x in xs]
    A, b, r2 = LM.power_fit(xs, ys)
    assert A == pytest.approx(1.33e-4, rel=1e-9)
    assert b == pytest.approx(0.937, rel=1e-12)
    assert r2 == pytest.approx(1.0, abs=1e-12)


def test_power_fit_r2_drops_with_scatter():
    xs = [2.0 ** e for e in range(14, 25)]
    ys = [6.77e-3 * x ** 0.97 * (1.5 if i % 2 else 1 / 1.5) for i, x in enumerate(xs)]
    A, b, r2 = LM.power_fit(xs, ys)
    # alternating factor 1.5^(+-1) in log space: residual variance log(1.5)^2 against the trend's spread
    assert 0.9 < r2 < 1.0
    assert b == pytest.approx(0.97, abs=0.05)


def test_power_fit_two_points_is_the_line_through_them():
    A, b, r2 = LM.power_fit([10.0, 1000.0], [2.0, 200.0])
    assert b == pytest.approx(1.0)
    assert A == pytest.approx(0.2)
    assert r2 == pytest.approx(1.0)


def test_steps_cover_four_phases_of_the_widest_tile_and_respect_the_cap():
    # heat: W/2 levels = W/2 steps per phase; four phases of W = 1024 is 2048 steps
    assert LM.steps_for("heat", 1 << 24, 2.0 ** 32, 1024, 20000) == 2048
    assert LM.steps_for("heat", 1 << 14, 2.0 ** 32, 1024, 20000) == 20000
    assert LM.steps_for("heat", 1 << 20, 2.0 ** 32, 1024, 20000) == 4096
    # Euler: 4 levels per step, so four phases of W = 1024 is 512 steps
    assert LM.steps_for("euler", 1 << 22, 2.0 ** 28, 1024, 20000) == 512
    assert LM.steps_for("euler", 1 << 14, 2.0 ** 28, 1024, 20000) == 16384
    # the floor wins over the cap
    assert LM.steps_for("heat", 1 << 14, 2.0 ** 32, 1024, 100) == 2048
    assert math.isfinite(LM.steps_for("heat", 1 << 10, 2.0 ** 32, 32, 20000))
