"""The seeded input generators shared by tests and benchmark (no scheme arithmetic)."""
import os

import numpy as np

from paper_1811_08282_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_reference_outputs():
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        want = [int(x, 16) for x in f.read().split() if x.startswith("0x")]
    got = [int(v) for v in I.splitmix64(0, len(want))]
    assert got == want


def test_generators_are_deterministic_and_in_range():
    a = I.uniform(42, 1000, -1, 1)
    assert np.array_equal(a, I.uniform(42, 1000, -1, 1))
    assert a.min() >= -1 and a.max() < 1
    k = I.randint(42, 1000, 1, 64)
    assert k.min() >= 1 and k.max() <= 64 and len(np.unique(k)) > 50
    m = I.heat_modes(1 << 14, 8, seed=3)
    assert m.amps.shape == (8,) and np.all((m.ks >= 1) & (m.ks <= 64))
    r = I.heat_r(7)
    assert 0.1 <= r < 0.45


def test_sod_layout():
    q = I.sod(16)
    assert q.shape == (3, 16)
    np.testing.assert_array_equal(q[0], [1.0] * 8 + [0.125] * 8)
    np.testing.assert_array_equal(q[1], 0.0)
    np.testing.assert_allclose(q[2], [2.5] * 8 + [0.25] * 8)


def test_riemann_segments_ranges():
    seg = I.riemann_segments(1 << 12, 64, 1)
    assert np.all((seg.rho >= 0.1) & (seg.rho <= 1.0))
    assert np.all((seg.p >= 0.1) & (seg.p <= 1.0))
    assert np.all(np.abs(seg.u) <= 0.5)
    q = I.riemann_initial(seg)
    assert q.shape == (3, 1 << 12)
