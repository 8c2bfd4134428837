"""sw_run_noalloc: the swept run for callers that cannot allocate device memory.

Code running inside a framework whose memory pool owns the whole device cannot
call cudaMalloc (it fails, or escapes the pool's accounting), and latency-critical
loops may not allocate after start-up (cudaMalloc / cudaFree can synchronise the
device). sw_run_noalloc serves them: it keeps the flank buffers of the swept
phases in a static 16 MiB device array inside the library instead of allocating.

These tests call it through the C ABI and compare it with the allocating entry
point (sw_run) on consecutive calls -- the shared array keeps the previous call's
contents, which must not leak into the next result -- with the tolerance the
other swept tests use (bitwise: same kernels, same arithmetic), and directly with
the FP64 oracle (heat within 1e-12 norm-relative, Euler bitwise). This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, norm_rel

pytestmark = pytest.mark.gpu


def _case(kind):
    if kind == "heat":
        n = 1 << 16
        p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                      n=n, r=0.31, tile_width=512)
        return p, I.heat_initial(I.heat_modes(n, 8, seed=21))[None], 777
    if kind == "heat_comp":
        n = 1 << 15
        p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP32_COMP, boundary=S.SW_TRANSMISSIVE,
                      method=S.SW_SWEPT, n=n, r=0.4, tile_width=256)
        return p, I.heat_initial(I.heat_modes(n, 8, seed=22))[None], 501
    n = 4096
    # "euler": the default form (flattened at W = 128); "euler_len": the lengthened form
    flags = S.SW_FLAG_LENGTHENED if kind == "euler_len" else 0
    p = S.Problem(scheme=S.SW_EULER, precision=S.SW_FP64, boundary=S.SW_TRANSMISSIVE, method=S.SW_SWEPT,
                  n=n, dt_dx=I.sod_lambda(), gamma=I.GAMMA, tile_width=128, flags=flags)
    return p, I.sod(n), 123


def _both(kind):
    import torch
    p, planes, steps = _case(kind)
    x = torch.as_tensor(np.ascontiguousarray(planes).reshape(-1), device="cuda")
    ref_state = S.to_state(p, x)
    with S.Handle(p) as h:
        h.sw_run(ref_state, steps)
    ref = S.to_fp64(p, ref_state).cpu().numpy()
    st = S.to_state(p, x)
    assert S.sw_run_noalloc(p, st, steps) == S.SW_OK
    got = S.to_fp64(p, st).cpu().numpy()
    torch.cuda.synchronize()
    return got, ref


def test_noalloc_matches_allocating_run_on_consecutive_calls():
    ensure_lib()
    # consecutive calls with different problems reuse the same static array
    for kind in ("heat", "euler", "heat_comp", "euler_len", "heat"):
        got, ref = _both(kind)
        assert np.array_equal(got, ref), f"{kind}: max diff {np.max(np.abs(got - ref))}"


def test_noalloc_matches_oracle():
    import torch
    ensure_lib()
    for kind in ("heat", "euler", "euler_len"):
        p, planes, steps = _case(kind)
        st = S.to_state(p, torch.as_tensor(np.ascontiguousarray(planes).reshape(-1), device="cuda"))
        S.sw_run_noalloc(p, st, steps)
        got = S.to_fp64(p, st).cpu().numpy().reshape(p.nv, p.n)
        torch.cuda.synchronize()
        if p.scheme == S.SW_HEAT:
            want = oracle.heat_run(planes[0], p.r, steps)[None]
            assert norm_rel(got, want) <= 1e-12
        else:
            want = oracle.euler_run(planes, p.dt_dx, p.gamma, steps, oracle.TRANSMISSIVE)
            assert np.array_equal(got, want)


def test_noalloc_warns_unstable_heat_like_sw_create():
    import torch
    ensure_lib()
    n = 4096
    p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                  n=n, r=0.55, tile_width=64)
    u0 = torch.as_tensor(I.heat_initial(I.heat_modes(n, 4, seed=3)), device="cuda")
    st = S.to_state(p, u0)
    assert S.sw_run_noalloc(p, st, 5) == S.SW_WARN_UNSTABLE
    ref = S.to_state(p, u0)
    with S.Handle(p) as h:
        assert h.warning == S.SW_WARN_UNSTABLE
        h.sw_run(ref, 5)
    torch.cuda.synchronize()
    assert torch.equal(st, ref)


def test_noalloc_rejects_problems_beyond_the_static_buffer():
    import torch
    ensure_lib()
    n = 1 << 22  # heat FP64 at W = 1024 needs ~128 MiB of flanks
    p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                  n=n, r=0.3, tile_width=1024)
    st = torch.arange(n, dtype=torch.float64, device="cuda")
    before = st.clone()
    with pytest.raises(S.SweptError) as ei:
        S.sw_run_noalloc(p, st, 10)
    assert ei.value.code == S.SW_ERR_TOO_LARGE
    # the largest grid the field rules allow (2^40 cells) is refused before any size wraps
    big = S.Problem(scheme=S.SW_EULER, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                    n=1 << 40, dt_dx=0.1, gamma=1.4, tile_width=1024)
    with pytest.raises(S.SweptError) as ei:
        S.sw_run_noalloc(big, st, 10)
    assert ei.value.code == S.SW_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert torch.equal(st, before)
    for bad in (dict(method=S.SW_PERSTEP), dict(flags=S.SW_FLAG_GRAPH), dict(n=(1 << 40) + 1024),
                dict(tile_width=6)):
        q = S.Problem(**{**p.__dict__, **bad})
        with pytest.raises(S.SweptError) as ei:
            S.sw_run_noalloc(q, st, 10)
        assert ei.value.code == S.SW_ERR_BAD_ARG
