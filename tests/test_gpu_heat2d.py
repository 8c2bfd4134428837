"""The swept rule in two dimensions (Section 6's future work) for FTCS heat, through the
C ABI (sw2d_*): swept == per-step bitwise in FP64 and FP32 (same per-cell function),
FP64 within 1e-12 of the oracle, a state constant along y bitwise equal to the 1D library
run of its row, the exact mode solution at a larger size, and the launch plan (one Up
launch, two per phase, the remaining steps per step).

Errors are taken relative to the initial state's largest magnitude: rounding errors scale
with the data, and on these small grids the modes decay by orders of magnitude within a
few steps, so the final state's own size says little about them."""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def run2d(p: S.Heat2D, u0, steps):
    import torch
    dt = torch.float64 if p.precision == S.SW_FP64 else torch.float32
    st = torch.as_tensor(np.ascontiguousarray(u0), device="cuda").to(dt).reshape(-1).clone()
    with S.Handle2D(p) as h:
        h.sw2d_run(st, steps)
        launches = h.sw2d_last_launch_count()
    torch.cuda.synchronize()
    return st.double().cpu().numpy().reshape(p.ny, p.nx), launches


CASES = [
    # nx, ny, W, steps
    (16, 16, 8, 9),        # two tiles each way, a ragged tail
    (48, 32, 8, 40),       # non-square tiling
    (64, 96, 16, 33),
    (128, 64, 32, 100),
    (256, 256, 64, 200),
    (192, 128, 64, 31),    # fewer steps than one phase: per-step only
    (160, 96, 32, 16),     # exactly one phase
]


@pytest.mark.parametrize("nx,ny,W,steps", CASES)
@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32])
def test_swept_equals_perstep_and_oracle(nx, ny, W, steps, prec):
    m = I.heat2d_modes(nx, ny, 6, seed=nx + ny + steps, kmax=8)
    u0 = I.heat2d_initial(m)
    rx, ry = 0.21, 0.17
    sw, ls = run2d(S.Heat2D(precision=prec, method=S.SW_SWEPT, tile_width=W, nx=nx, ny=ny, rx=rx, ry=ry), u0, steps)
    ps, lp = run2d(S.Heat2D(precision=prec, method=S.SW_PERSTEP, nx=nx, ny=ny, rx=rx, ry=ry), u0, steps)
    assert np.array_equal(sw, ps)
    H = W // 2
    P, R = steps // H, steps % H
    assert ls == (1 + 2 * P + R if P >= 1 else steps) and lp == steps
    want = oracle.heat2d_run(u0, rx, ry, steps)
    err = np.max(np.abs(sw - want)) / np.max(np.abs(u0))
    assert err <= (1e-12 if prec == S.SW_FP64 else 1e-5), err


@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32])
def test_constant_along_y_equals_the_1d_run(prec):
    # the y-difference of a state constant along y is exactly zero: each row must come out
    # as the 1D library's run of that row, bit for bit
    nx, ny, W, steps, r = 512, 64, 32, 77, 0.3
    row = I.heat_initial(I.heat_modes(nx, 6, seed=4))
    got, _ = run2d(S.Heat2D(precision=prec, method=S.SW_SWEPT, tile_width=W, nx=nx, ny=ny, rx=r, ry=0.11),
                   np.tile(row, (ny, 1)), steps)
    one = run_gpu(S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=S.SW_SWEPT, n=nx, r=r,
                            tile_width=64), row[None], steps)[0]
    for j in range(ny):
        assert np.array_equal(got[j], one)


@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32])
@pytest.mark.parametrize("W", [16, 32, 64, 128])
def test_threads_per_cta_give_the_same_bits(prec, W):
    # every thread count computes the same cells with the same arithmetic (the FP32 walker's
    # bands and the strip lines change with it; with 128 threads a warp takes several lines)
    if prec == S.SW_FP64 and W > 118:
        pytest.skip("an FP64 frame of W = 128 exceeds the shared memory (FP64 holds W <= 118)")
    nx, ny, steps = 4 * W, 3 * W, 3 * (W // 2) + 5
    u0 = I.heat2d_initial(I.heat2d_modes(nx, ny, 6, seed=W, kmax=8))
    p = S.Heat2D(precision=prec, method=S.SW_SWEPT, tile_width=W, nx=nx, ny=ny, rx=0.19, ry=0.23)
    ref, _ = run2d(S.Heat2D(precision=prec, method=S.SW_PERSTEP, nx=nx, ny=ny, rx=0.19, ry=0.23), u0, steps)
    import torch
    dt = torch.float64 if prec == S.SW_FP64 else torch.float32
    for nt, nb in ((128, 128), (256, 128), (128, 256), (256, 256), (1024, 256), (256, 1024)):
        st = torch.as_tensor(u0.reshape(-1), device="cuda").to(dt).clone()
        with S.Handle2D(p) as h:
            h.sw2d_set_threads(nt, nb)
            assert h.sw2d_threads() == nt and h.sw2d_threads(bridges=True) == nb
            h.sw2d_run(st, steps)
        torch.cuda.synchronize()
        assert np.array_equal(st.double().cpu().numpy().reshape(ny, nx), ref), (nt, nb)


def test_set_threads_refuses_other_counts():
    p = S.Heat2D(precision=S.SW_FP32, method=S.SW_SWEPT, tile_width=32, nx=128, ny=128, rx=0.2, ry=0.2)
    with S.Handle2D(p) as h:
        assert h.sw2d_threads() == 128 and h.sw2d_threads(bridges=True) == 128
        for bad in (64, 512, 100, -1):
            for args in ((bad, 0), (0, bad)):
                with pytest.raises(S.SweptError) as ei:
                    h.sw2d_set_threads(*args)
                assert ei.value.code == S.SW_ERR_BAD_ARG
        h.sw2d_set_threads(128, 1024)
        h.sw2d_set_threads(0, 0)
        assert h.sw2d_threads() == 128 and h.sw2d_threads(bridges=True) == 128
    p64 = S.Heat2D(precision=S.SW_FP64, method=S.SW_SWEPT, tile_width=32, nx=128, ny=128, rx=0.2, ry=0.2)
    with S.Handle2D(p64) as h:
        assert h.sw2d_threads() == 256 and h.sw2d_threads(bridges=True) == 256
    p128 = S.Heat2D(precision=S.SW_FP32, method=S.SW_SWEPT, tile_width=128, nx=256, ny=256, rx=0.2, ry=0.2)
    with S.Handle2D(p128) as h:
        assert h.sw2d_threads() == 1024 and h.sw2d_threads(bridges=True) == 256
    with S.Handle2D(S.Heat2D(precision=S.SW_FP32, method=S.SW_PERSTEP, nx=128, ny=128, rx=0.2, ry=0.2)) as h:
        with pytest.raises(S.SweptError):
            h.sw2d_set_threads(256)
        assert h.sw2d_threads() == 0


def test_transmissive_perstep_matches_oracle():
    nx, ny, steps = 96, 80, 60
    rng = np.random.default_rng(5)
    u0 = rng.uniform(-1, 1, (ny, nx))
    got, _ = run2d(S.Heat2D(precision=S.SW_FP64, boundary=S.SW_TRANSMISSIVE, method=S.SW_PERSTEP, nx=nx, ny=ny,
                            rx=0.2, ry=0.25), u0, steps)
    want = oracle.heat2d_run(u0, 0.2, 0.25, steps, oracle.TRANSMISSIVE)
    assert np.max(np.abs(got - want)) / np.max(np.abs(u0)) <= 1e-12


def test_exact_modes_at_2048_squared():
    nx = ny = 2048
    steps, rx, ry = 3000, 0.2, 0.2
    m = I.heat2d_modes(nx, ny, 16, seed=2, kmax=16)
    u0 = I.heat2d_initial(m)
    got, _ = run2d(S.Heat2D(precision=S.SW_FP64, method=S.SW_SWEPT, tile_width=64, nx=nx, ny=ny, rx=rx, ry=ry),
                   u0, steps)
    rng = np.random.default_rng(0)
    ii, jj = rng.integers(0, nx, 4096), rng.integers(0, ny, 4096)
    want = oracle.heat2d_modes(nx, ny, rx, ry, steps, m.amps, m.kx, m.ky, m.fx, m.fy, ii, jj)
    assert np.max(np.abs(got[jj, ii] - want)) <= 1e-12 * np.max(np.abs(u0))


def test_bad_arguments_are_refused():
    for bad in (dict(tile_width=6), dict(tile_width=48, nx=96, ny=100), dict(nx=64, ny=64, tile_width=64),
                dict(boundary=S.SW_TRANSMISSIVE), dict(rx=0.0), dict(precision=S.SW_FP32_COMP),
                dict(tile_width=256, precision=S.SW_FP64, nx=1024, ny=1024)):
        p = S.Heat2D(**{**dict(precision=S.SW_FP64, method=S.SW_SWEPT, tile_width=16, nx=128, ny=128), **bad})
        with pytest.raises(S.SweptError) as ei:
            S.Handle2D(p)
        assert ei.value.code in (S.SW_ERR_BAD_ARG, S.SW_ERR_UNSUPPORTED)
