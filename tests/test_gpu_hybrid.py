"""GPU parity of the hybrid CPU/GPU swept run (Section 4.2's affinity split, Eq. 1's GPU
work factor) through the C ABI: for every scheme, precision and boundary, sw_run_hybrid
(GPU structures 0 .. gpu_tiles-1, host threads the rest, flank slots crossing once per
phase) gives bitwise the state of sw_run, whatever the work factor, the thread count and
the kernel the GPU share runs (folded or generic); FP64 Euler is also the oracle's."""
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


def _heat(n, W, prec, bc, flags=0, r=0.3):
    return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=bc, method=S.SW_SWEPT, n=n, r=r, tile_width=W,
                     flags=flags)


def _euler(n, W, prec, bc, lam, flags=S.SW_FLAG_LENGTHENED):
    # the host engine runs the lengthened form (Section 4.3) only
    return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=bc, method=S.SW_SWEPT, n=n, dt_dx=lam, gamma=GAMMA,
                     tile_width=W, flags=flags)


def run_hybrid(problem, planes_fp64, nsteps, wf, threads):
    import torch
    x = torch.as_tensor(np.ascontiguousarray(planes_fp64, dtype=np.float64).reshape(-1), device="cuda")
    st = S.to_state(problem, x)
    with S.Handle(problem) as h:
        h.sw_run_hybrid(st, nsteps, wf, threads)
        out = S.to_fp64(problem, st)
        assert h.sw_sync_status() == 0
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(problem.nv, problem.n)


HEAT = [
    # n, W, steps, boundary, work factor, host threads, flags
    (1024, 32, 37, S.SW_PERIODIC, 1, 1, 0),
    (1024, 32, 40, S.SW_TRANSMISSIVE, 3, 2, 0),
    (4096, 128, 300, S.SW_PERIODIC, 4, 3, 0),           # GPU share on the folded kernel
    (4096, 128, 301, S.SW_PERIODIC, 4, 3, S.SW_FLAG_GENERIC),
    (8192, 256, 777, S.SW_PERIODIC, 10, 4, 0),
    (6000, 40, 123, S.SW_TRANSMISSIVE, 2, 5, 0),
    (1 << 16, 128, 1000, S.SW_PERIODIC, 30, 8, 0),
]


@pytest.mark.parametrize("n,W,steps,bc,wf,threads,flags", HEAT)
@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
def test_heat_hybrid_equals_gpu(n, W, steps, bc, wf, threads, flags, prec):
    u0 = I.heat_initial(I.heat_modes(n, 8, seed=n + steps))[None]
    p = _heat(n, W, prec, bc, flags)
    assert np.array_equal(run_hybrid(p, u0, steps, wf, threads), run_gpu(p, u0, steps))


EULER = [
    (1024, 32, 9, S.SW_TRANSMISSIVE, "sod", 1, 1),
    (2048, 64, 40, S.SW_PERIODIC, "riemann", 3, 2),
    (4096, 128, 70, S.SW_TRANSMISSIVE, "riemann", 5, 3),
    (3840, 96, 33, S.SW_PERIODIC, "riemann", 2, 4),
    (8192, 256, 130, S.SW_TRANSMISSIVE, "sod", 8, 2),
]


@pytest.mark.parametrize("n,W,steps,bc,kind,wf,threads", EULER)
@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
def test_euler_hybrid_equals_gpu(n, W, steps, bc, kind, wf, threads, prec):
    if kind == "sod":
        q0, lam = I.sod(n), I.sod_lambda()
    else:
        q0, lam = I.riemann_initial(I.riemann_segments(n, max(2, n // 128), 3)), I.riemann_lambda()
    p = _euler(n, W, prec, bc, lam)
    got = run_hybrid(p, q0, steps, wf, threads)
    assert np.array_equal(got, run_gpu(p, q0, steps))
    if prec == S.SW_FP64:
        want = oracle.euler_run(q0, lam, GAMMA, steps, oracle.PERIODIC if bc == S.SW_PERIODIC else oracle.TRANSMISSIVE)
        assert np.array_equal(got, want)


def test_hybrid_euler_fold_share():
    # the GPU share on the register-resident Euler kernel
    n, W, steps = 4096, 128, 64
    q0, lam = I.riemann_initial(I.riemann_segments(n, 32, 9)), I.riemann_lambda()
    p = _euler(n, W, S.SW_FP32, S.SW_TRANSMISSIVE, lam, flags=S.SW_FLAG_EULER_FOLD)
    assert np.array_equal(run_hybrid(p, q0, steps, 4, 2), run_gpu(p, q0, steps))


def test_hybrid_repeated_calls_and_thread_change():
    import torch
    n, W = 8192, 128
    u0 = I.heat_initial(I.heat_modes(n, 8, seed=3))[None]
    p = _heat(n, W, S.SW_FP64, S.SW_PERIODIC)
    want = run_gpu(p, u0, 500)
    st = S.to_state(p, torch.as_tensor(u0.reshape(-1), device="cuda"))
    with S.Handle(p) as h:
        h.sw_run_hybrid(st, 200, 6, 2)
        h.sw_run_hybrid(st, 250, 3, 5)   # new thread count
        h.sw_run(st, 50)                 # then the GPU alone
        got = S.to_fp64(p, st).cpu().numpy().reshape(1, n)
    assert np.array_equal(got, want)


def test_hybrid_rejects_flattened_euler_handle():
    # swept Euler defaults to the flattened form when W allows it; the host share has only
    # the lengthened sub-steps, so such a handle is refused before anything runs
    import torch
    n, W = 1024, 64
    q0, lam = I.sod(n), I.sod_lambda()
    for flags in (0, S.SW_FLAG_FLATTENED):
        p = _euler(n, W, S.SW_FP32, S.SW_TRANSMISSIVE, lam, flags=flags)
        st = S.to_state(p, torch.as_tensor(q0.reshape(-1), device="cuda"))
        before = st.clone()
        with S.Handle(p) as h:
            with pytest.raises(S.SweptError) as ei:
                h.sw_run_hybrid(st, 10, 4, 2)
            assert ei.value.code == S.SW_ERR_BAD_ARG
        torch.cuda.synchronize()
        assert torch.equal(st, before)


def test_hybrid_rejects_bad_split():
    import torch
    p = _heat(1024, 128, S.SW_FP64, S.SW_PERIODIC)   # 8 tiles
    st = S.to_state(p, torch.zeros(1024, dtype=torch.float64, device="cuda"))
    with S.Handle(p) as h:
        with pytest.raises(S.SweptError):
            h.sw_run_hybrid(st, 10, 8, 1)            # 8 // 9 = 0 tiles per thread
        with pytest.raises(S.SweptError):
            h.sw_run_hybrid(st, 10, 0, 2)            # work factor < 1
