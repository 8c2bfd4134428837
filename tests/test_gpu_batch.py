"""Batches: many independent problems of uneven lengths in one persistent launch.

Each problem of a batch must come out bitwise equal to advancing it alone with
sw_run (same per-structure device code, same arithmetic), FP64 Euler problems
also bitwise equal to the oracle. The launch is replayed from a CUDA graph;
replays are deterministic. A dependency wait that never completes (structure 0
of problem 0 withholds its flag through the test hook) ends after its budget
with SW_ERR_TIMEOUT, and the next run on the same context succeeds.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib

pytestmark = pytest.mark.gpu

WIDTHS = (32, 64, 128, 256)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _problem(item, prec, W, flags=0):
    if item.scheme == "heat":
        return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                         n=item.n, r=item.r, tile_width=W)
    return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=S.SW_TRANSMISSIVE, method=S.SW_SWEPT,
                     n=item.n, dt_dx=I.riemann_lambda(), gamma=I.GAMMA, tile_width=W, flags=flags)


def _setup(prec, count=24, seed=5, hi_exp=14.0, flat_every=0):
    import torch
    items = I.batch_problems(count, seed, lo_exp=10.0, hi_exp=hi_exp)
    probs, states, init = [], [], []
    for i, it in enumerate(items):
        W = WIDTHS[i % len(WIDTHS)]  # n is a multiple of 256 and >= 1024
        flags = S.SW_FLAG_FLATTENED if flat_every and i % flat_every == 0 else S.SW_FLAG_LENGTHENED
        p = _problem(it, prec, W, flags)
        x = torch.as_tensor(it.planes.reshape(-1), device="cuda")
        probs.append(p)
        states.append(S.to_state(p, x))
        init.append(x)
    return items, probs, states, init


def _read(probs, states):
    return [S.to_fp64(p, s).cpu().numpy() for p, s in zip(probs, states)]


@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
@pytest.mark.parametrize("flat_every", [0, 2])
def test_batch_equals_individual_runs(prec, flat_every):
    # flat_every = 2: every other problem in the flattened Euler form (heat ignores it)
    import torch
    nsteps = 150
    items, probs, states, init = _setup(prec, flat_every=flat_every)
    with S.Batch(probs, states, nsteps) as b:
        assert b.sw_batch_items() > 0
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        got = _read(probs, states)
    for i, (p, x) in enumerate(zip(probs, init)):
        st = S.to_state(p, x)
        with S.Handle(p) as h:
            h.sw_run(st, nsteps)
        want = S.to_fp64(p, st).cpu().numpy()
        assert np.array_equal(got[i], want), f"problem {i} ({items[i].scheme}, n={p.n}, W={p.tile_width})"
        if prec == S.SW_FP64 and items[i].scheme == "euler" and i < 8:
            ref = oracle.euler_run(items[i].planes, I.riemann_lambda(), I.GAMMA, nsteps, oracle.TRANSMISSIVE)
            assert np.array_equal(got[i], ref)
    torch.cuda.synchronize()


@pytest.mark.parametrize("threads", [64, 256])
def test_threads_per_cta_give_the_same_bits(threads):
    # the persistent kernel with 64 or 256 threads per CTA (sw_batch_set_threads) against the
    # default 128, set before the first run and changed between runs (the graph is re-captured)
    import torch
    items, probs, states, init = _setup(S.SW_FP32_COMP, count=20, seed=12, flat_every=2)
    nsteps = 90
    with S.Batch(probs, states, nsteps) as b:
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        ref = _read(probs, states)
        for p, st, x in zip(probs, states, init):
            st.copy_(S.to_state(p, x))
        b.sw_batch_set_threads(threads)
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        got = _read(probs, states)
        with pytest.raises(S.SweptError):
            b.sw_batch_set_threads(96)
    for a, c in zip(ref, got):
        assert np.array_equal(a, c)
    torch.cuda.synchronize()


def test_compensated_heat_items_against_the_oracle():
    # FP32 hi/lo heat problems of a batch: within 1e-9 of the initial magnitude of the FP64
    # oracle after 2,000 steps (their Euler neighbours are covered by the precision tests)
    import torch
    items, probs, states, init = _setup(S.SW_FP32_COMP, count=24, seed=13)
    nsteps = 2000
    with S.Batch(probs, states, nsteps) as b:
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        got = _read(probs, states)
    checked = 0
    for i, it in enumerate(items):
        if it.scheme != "heat":
            continue
        want = oracle.heat_run(it.planes[0], it.r, nsteps)
        assert np.max(np.abs(got[i].reshape(-1) - want)) <= 1e-9 * np.max(np.abs(it.planes)), i
        checked += 1
    assert checked >= 10
    torch.cuda.synchronize()


def test_batch_graph_replay_is_deterministic():
    import torch
    items, probs, states, init = _setup(S.SW_FP32_COMP, count=16, seed=9)
    with S.Batch(probs, states, 77) as b:
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        first = _read(probs, states)
        for p, st, x in zip(probs, states, init):  # reset the states and replay the graph
            st.copy_(S.to_state(p, x))
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        second = _read(probs, states)
    for a, c in zip(first, second):
        assert np.array_equal(a, c)
    torch.cuda.synchronize()


def test_dependency_wait_times_out_and_context_recovers():
    import torch
    items, probs, states, init = _setup(S.SW_FP32, count=8, seed=3, hi_exp=12.0)
    with S.Batch(probs, states, 40) as b:
        b.sw_batch_debug(20_000_000, True)  # ~10 ms budget; one structure never publishes
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_ERR_TIMEOUT
        b.sw_batch_debug(2_000_000_000, False)
        for p, st, x in zip(probs, states, init):
            st.copy_(S.to_state(p, x))
        b.sw_batch_run()
        assert b.sw_batch_status() == S.SW_OK
        got = _read(probs, states)
    p, x = probs[1], init[1]
    st = S.to_state(p, x)
    with S.Handle(p) as h:
        h.sw_run(st, 40)
    assert np.array_equal(got[1], S.to_fp64(p, st).cpu().numpy())
    torch.cuda.synchronize()


def test_autotune_picks_a_dividing_width():
    for scheme, n in ((S.SW_HEAT, 1 << 16), (S.SW_EULER, 3 * 4096)):
        p = S.Problem(scheme=scheme, precision=S.SW_FP32_COMP,
                      boundary=S.SW_PERIODIC if scheme == S.SW_HEAT else S.SW_TRANSMISSIVE,
                      method=S.SW_SWEPT, n=n, r=0.3, dt_dx=0.08, gamma=1.4, flags=S.SW_FLAG_GENERIC)
        W = S.sw_autotune(p, 256)
        assert W in (32, 64, 128, 256, 512, 1024) and n % W == 0 and n >= 2 * W
