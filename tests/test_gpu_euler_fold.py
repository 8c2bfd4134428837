"""GPU parity of the register-resident Euler phase kernel (k_euler_fold) through the C ABI.

With SW_FLAG_EULER_FOLD the folded kernel runs the Up Triangle, every Diamond and the
Down Triangle at W = 128 (FP64, FP32, FP32 hi/lo) and W = 256 (FP32 forms); a truncated
upper half still runs on the generic kernel. It must agree bitwise with the generic
phase kernel (forced by SW_FLAG_GENERIC) and with the per-step kernel, on periodic and
transmissive grids, for step counts that end inside a phase, and (FP64) with the oracle.
"""
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


def _prob(n, W, lam, bc, method, prec, flags=S.SW_FLAG_EULER_FOLD):
    return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=bc, method=method, n=n, dt_dx=lam, gamma=GAMMA,
                     tile_width=W if method == S.SW_SWEPT else 0, flags=flags)


def _init(kind, n, seed):
    if kind == "sod":
        return I.sod(n), I.sod_lambda()
    return I.riemann_initial(I.riemann_segments(n, max(2, min(64, n // 128)), seed)), I.riemann_lambda()


CASES = [
    # n, W, steps, boundary, init: whole phases, ragged ends, one tile pair, long chains per warp
    (256, 128, 3, S.SW_TRANSMISSIVE, "sod"),
    (256, 128, 16, S.SW_PERIODIC, "riemann"),
    (512, 128, 40, S.SW_TRANSMISSIVE, "riemann"),
    (1024, 128, 100, S.SW_PERIODIC, "riemann"),
    (2048, 128, 161, S.SW_TRANSMISSIVE, "sod"),
    (4096, 256, 200, S.SW_TRANSMISSIVE, "riemann"),
    (4096, 256, 96, S.SW_PERIODIC, "riemann"),
    (8192, 256, 333, S.SW_TRANSMISSIVE, "sod"),
    (1 << 17, 128, 250, S.SW_TRANSMISSIVE, "riemann"),
    (1 << 18, 256, 130, S.SW_PERIODIC, "riemann"),
]

PRECS = [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP]


@pytest.mark.parametrize("n,W,steps,bc,kind", CASES)
@pytest.mark.parametrize("prec", PRECS)
def test_fold_equals_generic_and_perstep(n, W, steps, bc, kind, prec):
    if prec == S.SW_FP64 and W != 128:
        pytest.skip("the FP64 folded kernel is instantiated at W = 128 only")
    q0, lam = _init(kind, n, seed=n + steps)
    fold = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, prec), q0, steps)
    generic = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, prec, flags=S.SW_FLAG_GENERIC), q0, steps)
    per = run_gpu(_prob(n, W, lam, bc, S.SW_PERSTEP, prec), q0, steps)
    assert np.array_equal(fold, generic)
    assert np.array_equal(fold, per)
    assert np.all(np.isfinite(fold))


@pytest.mark.parametrize("n,W,steps,bc,kind", [c for c in CASES if c[0] <= 4096 and c[1] == 128])
def test_fold_fp64_equals_oracle(n, W, steps, bc, kind):
    q0, lam = _init(kind, n, seed=n + steps)
    got = run_gpu(_prob(n, W, lam, bc, S.SW_SWEPT, S.SW_FP64), q0, steps)
    want = oracle.euler_run(q0, lam, GAMMA, steps, oracle.PERIODIC if bc == S.SW_PERIODIC else oracle.TRANSMISSIVE)
    assert np.array_equal(got, want)


def test_fold_resume_is_bitwise_continuation():
    # run(a); run(b) == run(a + b): the state between runs is Q alone
    n, W = 4096, 128
    q0, lam = _init("riemann", n, seed=5)
    p = _prob(n, W, lam, S.SW_TRANSMISSIVE, S.SW_SWEPT, S.SW_FP32)
    once = run_gpu(p, q0, 90)
    first = run_gpu(p, q0, 37)
    both = run_gpu(p, first, 53)
    assert np.array_equal(once, both)
