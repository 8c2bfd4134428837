"""GPU tests of SW_FLAG_GRAPH: a run captured once into a CUDA graph and replayed gives
bitwise the state of the same run launched directly (swept and per-step, heat and Euler),
replays reuse the graph, and a new state pointer or step count captures again."""
import numpy as np
import pytest

from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _heat(method, prec, flags, n=16384, W=64):
    return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=method, n=n, r=0.25,
                     tile_width=W if method == S.SW_SWEPT else 0, flags=flags)


def _euler(method, prec, flags, n=4096, W=128):
    return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=S.SW_TRANSMISSIVE, method=method, n=n,
                     dt_dx=I.sod_lambda(), gamma=I.GAMMA, tile_width=W if method == S.SW_SWEPT else 0, flags=flags)


@pytest.mark.parametrize("method", [S.SW_SWEPT, S.SW_PERSTEP])
@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
@pytest.mark.parametrize("steps", [1, 57, 1000])
def test_graph_equals_direct_heat(method, prec, steps):
    u0 = I.heat_initial(I.heat_modes(16384, 8, seed=steps))[None]
    assert np.array_equal(run_gpu(_heat(method, prec, S.SW_FLAG_GRAPH), u0, steps),
                          run_gpu(_heat(method, prec, 0), u0, steps))


@pytest.mark.parametrize("method,flags", [(S.SW_SWEPT, 0), (S.SW_PERSTEP, 0), (S.SW_PERSTEP, S.SW_FLAG_LENGTHENED),
                                          (S.SW_SWEPT, S.SW_FLAG_FLATTENED)])
def test_graph_equals_direct_euler(method, flags):
    q0 = I.sod(4096)
    assert np.array_equal(run_gpu(_euler(method, S.SW_FP32, flags | S.SW_FLAG_GRAPH), q0, 77),
                          run_gpu(_euler(method, S.SW_FP32, flags), q0, 77))


def test_replay_and_recapture():
    import torch
    u0 = I.heat_initial(I.heat_modes(16384, 8, seed=1))[None]
    want = run_gpu(_heat(S.SW_PERSTEP, S.SW_FP64, 0), u0, 300)
    p = _heat(S.SW_PERSTEP, S.SW_FP64, S.SW_FLAG_GRAPH)
    x = torch.as_tensor(u0.reshape(-1), device="cuda")
    a, b = S.to_state(p, x), S.to_state(p, x)
    with S.Handle(p) as h:
        for _ in range(3):
            h.sw_run(a, 100)          # captured once, replayed twice
        assert h.sw_last_launch_count() == 100
        h.sw_run(b, 250)              # new pointer and count: captured again
        h.sw_run(b, 50)               # new count
        assert h.sw_sync_status() == 0
        ga, gb = S.to_fp64(p, a).cpu().numpy(), S.to_fp64(p, b).cpu().numpy()
    assert np.array_equal(ga.reshape(1, -1), want)
    assert np.array_equal(gb.reshape(1, -1), want)
