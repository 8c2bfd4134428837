"""Pins of the FTCS heat oracle (Section 4.2) to mathematics it cannot fake.

- the dense matrix power (I + r L)^s u0 in extended precision (textbook linear algebra),
- the exact discrete decay G(k)^s of Fourier modes, G(k) = 1 - 4 r sin^2(pi k/n),
- the vanishing of the Nyquist mode k = n/2 after one step at r = 1/4,
- conservation of total heat, exact translation invariance.
A dropped term, a wrong sign, a wrong neighbour index or a wrong factor fails one of these.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I


def _ftcs_matrix(n, r, boundary):
    """(I + r L) with L the second-difference matrix (periodic or zero-gradient ends)."""
    a = np.zeros((n, n), dtype=np.longdouble)
    for j in range(n):
        a[j, j] += 1 - 2 * np.longdouble(r)
        for nb in (j - 1, j + 1):
            if boundary == oracle.PERIODIC:
                nb %= n
            else:
                nb = min(max(nb, 0), n - 1)
            a[j, nb] += np.longdouble(r)
    return a


def _matpow_apply(a, u0, s):
    u = np.asarray(u0, dtype=np.longdouble)
    for _ in range(s):
        u = a.dot(u)
    return u


@pytest.mark.parametrize("boundary", [oracle.PERIODIC, oracle.TRANSMISSIVE])
@pytest.mark.parametrize("r", [0.1, 0.25, 0.45])
def test_heat_matches_matrix_power(boundary, r):
    n, s = 24, 60
    u0 = I.uniform(7, n, -1.0, 1.0)
    got = oracle.heat_run(u0, r, s, boundary)
    want = _matpow_apply(_ftcs_matrix(n, r, boundary), u0, s)
    err = np.max(np.abs(got - want.astype(np.float64)))
    assert err < 50 * s * np.finfo(np.float64).eps


def test_closed_form_matches_matrix_power():
    n, s, r = 32, 40, 0.3
    modes = I.heat_modes(n, 5, seed=3, kmax=15)
    u0 = I.heat_initial(modes)
    want = _matpow_apply(_ftcs_matrix(n, r, oracle.PERIODIC), u0, s).astype(np.float64)
    got = oracle.heat_modes(n, r, s, modes.amps, modes.ks)
    assert np.max(np.abs(got - want)) < 1e-13


def test_closed_form_at_zero_steps_is_initial_state():
    n = 4096
    modes = I.heat_modes(n, 32, seed=11)
    u0 = I.heat_initial(modes)
    got = oracle.heat_modes(n, 0.3, 0, modes.amps, modes.ks)
    assert np.max(np.abs(got - u0)) < 1e-13


@pytest.mark.parametrize("n,s,r,seed", [(1024, 500, 0.25, 0), (16384, 200, 0.4, 1), (4096, 3000, 0.45, 2)])
def test_stepper_matches_mode_decay(n, s, r, seed):
    modes = I.heat_modes(n, 8, seed=seed)
    u0 = I.heat_initial(modes)
    got = oracle.heat_run(u0, r, s)
    want = oracle.heat_modes(n, r, s, modes.amps, modes.ks)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) / scale < 1e-12


def test_single_high_mode_decay_factor():
    # one mode with strong decay: the ratio after s steps is G(k)^s exactly
    n, k, r, s = 256, 37, 0.3, 25
    u0 = I.heat_initial(I.HeatModes(n=n, amps=np.array([1.0]), ks=np.array([k])))
    got = oracle.heat_run(u0, r, s)
    g = 1.0 - 4.0 * r * np.sin(np.pi * k / n) ** 2
    np.testing.assert_allclose(got, (g ** s) * u0, rtol=0, atol=1e-13)


def test_nyquist_mode_vanishes_at_r_quarter():
    # mode k = n/2 has G = 1 - 4 r sin^2(pi/2) = 1 - 4r, which is 0 at r = 1/4
    n = 64
    j = np.arange(n)
    u0 = np.cos(np.pi * j)  # mode k = n/2 (alternating +-1), exact in binary
    got = oracle.heat_run(u0, 0.25, 1)
    assert np.max(np.abs(got)) == 0.0


@pytest.mark.parametrize("boundary", [oracle.PERIODIC, oracle.TRANSMISSIVE])
def test_total_heat_conserved(boundary):
    n, s = 8192, 2000
    u0 = I.uniform(5, n, -1.0, 1.0)
    got = oracle.heat_run(u0, 0.4, s, boundary)
    s0 = np.sum(u0.astype(np.longdouble))
    s1 = np.sum(got.astype(np.longdouble))
    assert abs(float(s1 - s0)) < 1e-9


def test_translation_invariance_is_bitwise():
    n, s, shift = 2048, 300, 517
    u0 = I.uniform(9, n, -1.0, 1.0)
    a = oracle.heat_run(u0, 0.33, s)
    b = oracle.heat_run(np.roll(u0, shift), 0.33, s)
    assert np.array_equal(np.roll(a, shift), b)


def test_zero_steps_is_identity():
    u0 = I.uniform(1, 100, -1.0, 1.0)
    assert np.array_equal(oracle.heat_run(u0, 0.2, 0), u0)
