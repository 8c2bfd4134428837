"""Pins of the 2D FTCS oracle (the 5-point extension of Section 6's future work) against
what the mathematics fixes, independent of the oracle's own code:

- the dense matrix power (I + rx Lx + ry Ly)^s in extended precision on tiny grids,
  periodic and transmissive (a brute-force restatement of the operator);
- a state constant along y is advanced, row by row, bit for bit as the 1D oracle (already
  pinned by its own tests) with r = rx; the same for x with ry after a transpose;
- the exact eigen-decomposition: separable sin/cos modes decay by
  G = 1 - 4 rx sin^2(pi kx/nx) - 4 ry sin^2(pi ky/ny) per step (closed form), and the
  closed form at s = 0 is the input generator's state;
- total heat conserved on periodic grids; a periodic shift in x and y commutes with a
  run bitwise; swapping x and y (and rx, ry) transposes the result bitwise.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I


def _lap1d(n, periodic):
    L = np.zeros((n, n), dtype=np.longdouble)
    for i in range(n):
        L[i, i] -= 2
        for d in (-1, 1):
            k = i + d
            if periodic:
                k %= n
            else:
                k = min(max(k, 0), n - 1)
            L[i, k] += 1
    return L


def _dense(u0, rx, ry, steps, periodic):
    ny, nx = u0.shape
    Lx = np.kron(np.eye(ny, dtype=np.longdouble), _lap1d(nx, periodic))
    Ly = np.kron(_lap1d(ny, periodic), np.eye(nx, dtype=np.longdouble))
    A = np.eye(nx * ny, dtype=np.longdouble) + np.longdouble(rx) * Lx + np.longdouble(ry) * Ly
    v = u0.reshape(-1).astype(np.longdouble)
    for _ in range(steps):
        v = A @ v
    return v.astype(np.float64).reshape(ny, nx)


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.TRANSMISSIVE])
@pytest.mark.parametrize("shape,rx,ry,steps", [((4, 5), 0.2, 0.15, 7), ((6, 6), 0.1, 0.3, 20), ((3, 8), 0.24, 0.01, 13)])
def test_matches_dense_matrix_power(bc, shape, rx, ry, steps):
    rng = np.random.default_rng(sum(shape) + steps)
    u0 = rng.uniform(-1, 1, shape)
    got = oracle.heat2d_run(u0, rx, ry, steps, bc)
    want = _dense(u0, rx, ry, steps, bc == oracle.PERIODIC)
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("bc", [oracle.PERIODIC, oracle.TRANSMISSIVE])
def test_constant_in_y_reduces_to_1d_bitwise(bc):
    nx, ny, rx, ry, steps = 96, 7, 0.31, 0.2, 45
    row = I.heat_initial(I.heat_modes(nx, 5, seed=2))
    got = oracle.heat2d_run(np.tile(row, (ny, 1)), rx, ry, steps, bc)
    want = oracle.heat_run(row, rx, steps, bc)
    for j in range(ny):
        assert np.array_equal(got[j], want)
    # and along x after a transpose, with ry
    col = I.heat_initial(I.heat_modes(ny * 9, 3, seed=5))
    got = oracle.heat2d_run(np.tile(col[:, None], (1, 5)), rx, ry, steps, bc)
    want = oracle.heat_run(col, ry, steps, bc)
    for i in range(5):
        assert np.array_equal(got[:, i], want)


def test_separable_modes_decay_by_the_exact_factor():
    nx, ny, rx, ry, steps = 64, 48, 0.2, 0.17, 100
    m = I.heat2d_modes(nx, ny, 6, seed=3, kmax=4)
    u0 = I.heat2d_initial(m)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    at0 = oracle.heat2d_modes(nx, ny, rx, ry, 0, m.amps, m.kx, m.ky, m.fx, m.fy, ii.ravel(), jj.ravel())
    assert np.max(np.abs(at0.reshape(ny, nx) - u0)) <= 1e-14
    got = oracle.heat2d_run(u0, rx, ry, steps)
    want = oracle.heat2d_modes(nx, ny, rx, ry, steps, m.amps, m.kx, m.ky, m.fx, m.fy, ii.ravel(), jj.ravel())
    # rounding: a few ulps of the initial magnitude per step
    assert np.max(np.abs(got.ravel() - want)) <= steps * 4 * 2.0 ** -52 * np.max(np.abs(u0))
    assert np.max(np.abs(want)) > 1e-3 * np.max(np.abs(u0))  # the modes are still there
    # one mode alone: u^s = G^s u^0 exactly in the closed form; check the factor directly
    k = (3, 5)
    g = 1 - 4 * rx * np.sin(np.pi * k[0] / nx) ** 2 - 4 * ry * np.sin(np.pi * k[1] / ny) ** 2
    one = oracle.heat2d_modes(nx, ny, rx, ry, 10, [1.0], [k[0]], [k[1]], [1], [0], [7], [11])
    base = np.cos(2 * np.pi * k[0] * 7 / nx) * np.sin(2 * np.pi * k[1] * 11 / ny)
    assert one[0] == pytest.approx(g ** 10 * base, rel=1e-13)


def test_conservation_shift_and_transpose():
    nx, ny, rx, ry, steps = 40, 24, 0.22, 0.13, 60
    rng = np.random.default_rng(9)
    u0 = rng.uniform(-1, 1, (ny, nx))
    got = oracle.heat2d_run(u0, rx, ry, steps)
    assert abs(float(got.sum(dtype=np.longdouble) - u0.sum(dtype=np.longdouble))) < 1e-12
    shifted = oracle.heat2d_run(np.roll(u0, (5, 11), axis=(0, 1)), rx, ry, steps)
    assert np.array_equal(shifted, np.roll(got, (5, 11), axis=(0, 1)))
    tr = oracle.heat2d_run(np.ascontiguousarray(u0.T), ry, rx, steps)
    assert np.array_equal(tr, got.T)
