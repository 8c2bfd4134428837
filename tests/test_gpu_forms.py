"""GPU parity of the two data-structure strategies of Section 4.3 (Fig. 2) for the Euler
step, through the C ABI: swept lengthened (SW_FLAG_LENGTHENED), swept flattened
(SW_FLAG_FLATTENED: two 5-point stages per step on radius-2 windows; the default when
W % 4 == 0 and W >= 8), per-step flattened (default) and per-step lengthened
(SW_FLAG_LENGTHENED: four 3-point launches per step) evaluate the same per-cell
functions and must agree bitwise, and (FP64) with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, run_gpu

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _prob(n, W, lam, bc, method, prec, flags=0):
    return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=bc, method=method, n=n, dt_dx=lam, gamma=GAMMA,
                     tile_width=W if method == S.SW_SWEPT else 0, flags=flags)


CASES = [
    # n, W, steps, boundary, init: single-level halves, ragged ends, wide tiles, many tiles
    (64, 8, 5, S.SW_TRANSMISSIVE, "sod"),
    (64, 8, 6, S.SW_PERIODIC, "riemann"),
    (256, 16, 21, S.SW_TRANSMISSIVE, "riemann"),
    (1024, 64, 100, S.SW_PERIODIC, "riemann"),
    (2048, 256, 301, S.SW_TRANSMISSIVE, "sod"),
    (3072, 96, 150, S.SW_PERIODIC, "riemann"),
    (4096, 1024, 600, S.SW_TRANSMISSIVE, "riemann"),
    (1000, 40, 77, S.SW_TRANSMISSIVE, "sod"),
    (1 << 18, 512, 333, S.SW_TRANSMISSIVE, "riemann"),
]


def _init(kind, n, seed):
    if kind == "sod":
        return I.sod(n), I.sod_lambda()
    return I.riemann_initial(I.riemann_segments(n, max(2, min(64, n // 128)), seed)), I.riemann_lambda()


@pytest.mark.parametrize("n,W,steps,bc,kind", CASES)
@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
def test_four_forms_agree_bitwise(n, W, steps, bc, kind, prec):
    q0, lam = _init(kind, n, seed=n + steps)
    swept_len = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, prec, S.SW_FLAG_LENGTHENED), q0, steps)
    swept_default = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, prec), q0, steps)
    swept_flat = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, prec, S.SW_FLAG_FLATTENED), q0, steps)
    per_flat = run_gpu(_prob(n, W, lam, bc, S.SW_PERSTEP, prec), q0, steps)
    per_len = run_gpu(_prob(n, W, lam, bc, S.SW_PERSTEP, prec, S.SW_FLAG_LENGTHENED), q0, steps)
    assert np.array_equal(swept_flat, swept_len)
    assert np.array_equal(swept_default, swept_len)
    assert np.array_equal(per_len, per_flat)
    assert np.array_equal(swept_len, per_flat)
    if prec == S.SW_FP64 and n <= 4096:
        want = oracle.euler_run(q0, lam, GAMMA, steps, oracle.PERIODIC if bc == S.SW_PERIODIC else oracle.TRANSMISSIVE)
        assert np.array_equal(swept_flat, want)


def test_flattened_launch_count():
    # W/4 levels per phase half, two levels per step: W/8 steps per phase, as lengthened
    n, W, steps = 4096, 128, 160
    q0, lam = _init("riemann", n, 1)
    import torch
    for flags in (0, S.SW_FLAG_LENGTHENED, S.SW_FLAG_FLATTENED):
        p = _prob(n, W, lam, S.SW_TRANSMISSIVE, S.SW_SWEPT, S.SW_FP32, flags)
        st = S.to_state(p, torch.as_tensor(q0.reshape(-1), device="cuda"))
        with S.Handle(p) as h:
            h.sw_run(st, steps)
            assert h.sw_last_launch_count() == steps // (W // 8) + 1
    p = _prob(n, W, lam, S.SW_TRANSMISSIVE, S.SW_PERSTEP, S.SW_FP32, S.SW_FLAG_LENGTHENED)
    st = S.to_state(p, torch.as_tensor(q0.reshape(-1), device="cuda"))
    with S.Handle(p) as h:
        h.sw_run(st, 10)
        assert h.sw_last_launch_count() == 40


@pytest.mark.parametrize("flags,W,shift", [(S.SW_FLAG_LENGTHENED, 64, 37), (S.SW_FLAG_FLATTENED, 64, 37),
                                           (S.SW_FLAG_FLATTENED, 128, 6), (0, 32, 37),
                                           (0, 256, 130)])
def test_translation_invariance_across_seams_bitwise(flags, W, shift):
    # periodic: shifting the initial state by s cells (s not a multiple of W) shifts the result
    # by s, bitwise -- every cell sits at a different place in its tile, so this pins the seams
    n, steps = 2048, 97
    q0, lam = _init("riemann", n, seed=11)
    p = _prob(n, W, lam, S.SW_PERIODIC, S.SW_SWEPT, S.SW_FP32, flags)
    a = run_gpu(p, q0, steps)
    b = run_gpu(p, np.roll(q0, shift, axis=1), steps)
    assert np.array_equal(np.roll(a, shift, axis=1), b)
