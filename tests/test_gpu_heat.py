"""GPU parity of the FTCS heat path through the C ABI (swept phases and per-step kernel).

- FP64 swept == FP64 per-step, bitwise (same per-cell arithmetic; Section 4.1 says
  the swept rule uses the same numerical method as the classic decomposition);
- FP64 vs the FP64 oracle: norm-relative error <= 1e-12 (GPU uses fused
  multiply-adds, the oracle plain expressions; FTCS is a contraction for r <= 1/2,
  so rounding differences do not grow);
- FP32 and FP32-compensated: swept == per-step bitwise; error vs the oracle below
  stated bounds. Sizes span several tiles, ragged step counts (not multiples of
  W/2) and both boundary kinds.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, norm_rel, run_gpu

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12

CASES = [
    # n, W, steps, boundary, r
    (16, 4, 1, S.SW_PERIODIC, 0.3),
    (16, 4, 7, S.SW_TRANSMISSIVE, 0.3),
    (64, 8, 37, S.SW_PERIODIC, 0.45),
    (256, 32, 100, S.SW_TRANSMISSIVE, 0.25),
    (1024, 64, 1000, S.SW_PERIODIC, 0.25),
    (4096, 128, 333, S.SW_TRANSMISSIVE, 0.4),
    (6144, 96, 517, S.SW_PERIODIC, 0.2),
    (3000, 100, 250, S.SW_TRANSMISSIVE, 0.35),
    (8192, 1024, 2500, S.SW_PERIODIC, 0.45),
    (2048, 1024, 700, S.SW_TRANSMISSIVE, 0.3),
    (4096, 512, 255, S.SW_PERIODIC, 0.1),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _init(n, seed=0):
    return I.heat_initial(I.heat_modes(n, 8, seed=seed, kmax=min(64, n // 4)))


def _prob(n, W, r, bc, method, prec=S.SW_FP64, flags=0):
    return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=bc, method=method, n=n, r=r,
                     tile_width=W if method == S.SW_SWEPT else 0, flags=flags)


@pytest.mark.parametrize("n,W,steps,bc,r", CASES)
def test_fp64_swept_equals_perstep_and_oracle(n, W, steps, bc, r):
    u0 = _init(n, seed=n + steps)
    sw = run_gpu(_prob(n, W, r, bc, S.SW_SWEPT), u0[None], steps)
    ps = run_gpu(_prob(n, W, r, bc, S.SW_PERSTEP), u0[None], steps)
    assert np.array_equal(sw, ps), f"max diff {np.max(np.abs(sw - ps))}"
    ref = oracle.heat_run(u0, r, steps, oracle.PERIODIC if bc == S.SW_PERIODIC else oracle.TRANSMISSIVE)
    assert norm_rel(sw, ref[None]) <= TOL_FP64


# FP32_COMP keeps the state to ~2^-48 but each increment is still rounded to FP32, so
# its error grows like eps32 * (sum of |increments|): ~1e-9 on these fast-decaying modes
@pytest.mark.parametrize("prec,tol", [(S.SW_FP32, 2e-5), (S.SW_FP32_COMP, 1e-8)])
@pytest.mark.parametrize("n,W,steps,bc,r", [CASES[2], CASES[4], CASES[7], CASES[8]])
def test_fp32_variants_swept_equals_perstep(prec, tol, n, W, steps, bc, r):
    u0 = _init(n, seed=7)
    sw = run_gpu(_prob(n, W, r, bc, S.SW_SWEPT, prec), u0[None], steps)
    ps = run_gpu(_prob(n, W, r, bc, S.SW_PERSTEP, prec), u0[None], steps)
    assert np.array_equal(sw, ps)
    ref = oracle.heat_run(u0, r, steps, oracle.PERIODIC if bc == S.SW_PERIODIC else oracle.TRANSMISSIVE)
    assert norm_rel(sw, ref[None]) <= tol


@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP])
@pytest.mark.parametrize("n,W,steps", [
    (256, 128, 300),       # two diamonds per phase: one per warp
    (1024, 128, 1000),
    (192, 64, 77),         # W = 64 (two cells per lane): three tiles, an odd number of diamonds
    (4096, 64, 31),        # shorter than one Up Triangle
    (4096, 64, 96),        # a multiple of W/2: complete Down Triangle
    (16384, 64, 1000),     # the small-grid workload's shape
    (4096, 256, 777),      # ragged last phases run on the generic kernel
    (1 << 16, 512, 1500),
    (1 << 15, 1024, 2100),
    (2048, 1024, 513),
    (3 * 1024, 1024, 1025),  # odd number of diamonds
    (4096, 256, 1),          # shorter than one Up Triangle
    (4096, 256, 127),        # W/2 - 1: Up truncated, Down
    (4096, 256, 128),        # exactly one Up + Down
    (4096, 256, 129),
    (4096, 256, 640),        # a multiple of W/2: complete Down Triangle
    (8192, 512, 256 * 7 + 5),
    (1 << 21, 128, 200),     # FP64: a smooth field, integer path nearly everywhere
])
def test_register_diamond_kernel_matches_generic_kernel(prec, n, W, steps):
    # periodic heat at W = 32K uses the register-resident Diamond kernel for every complete
    # Diamond phase; SW_FLAG_GENERIC forces the shared-memory kernel everywhere. FP64 at
    # W = 128 and 256 updates half the register cells on the integer pipes, the generic
    # kernel all of them on the FP64 pipe: the two must agree bit for bit
    u0 = _init(n, seed=W + steps)
    fast = run_gpu(_prob(n, W, 0.33, S.SW_PERIODIC, S.SW_SWEPT, prec), u0[None], steps)
    gen = run_gpu(_prob(n, W, 0.33, S.SW_PERIODIC, S.SW_SWEPT, prec, flags=S.SW_FLAG_GENERIC), u0[None], steps)
    assert np.array_equal(fast, gen), f"max diff {np.max(np.abs(fast - gen))}"
    if prec == S.SW_FP64:
        ref = oracle.heat_run(u0, 0.33, steps)
        assert norm_rel(fast, ref[None]) <= TOL_FP64


def test_compensated_beats_plain_fp32_where_fp32_stagnates():
    # smooth low modes on a large grid: the per-step increment is far below half an
    # FP32 ulp, so plain FP32 cannot follow the decay; the hi/lo form can.
    n, steps, r = 1 << 16, 4000, 0.4
    modes = I.heat_modes(n, 4, seed=3, kmax=8)
    u0 = I.heat_initial(modes)
    ref = oracle.heat_modes(n, r, steps, modes.amps, modes.ks)
    e32 = norm_rel(run_gpu(_prob(n, 1024, r, S.SW_PERIODIC, S.SW_SWEPT, S.SW_FP32), u0[None], steps), ref[None])
    ecomp = norm_rel(run_gpu(_prob(n, 1024, r, S.SW_PERIODIC, S.SW_SWEPT, S.SW_FP32_COMP), u0[None], steps),
                     ref[None])
    assert ecomp < 1e-9
    assert ecomp < e32 / 100


def test_zero_steps_is_identity():
    u0 = _init(256)
    for method in (S.SW_SWEPT, S.SW_PERSTEP):
        out = run_gpu(_prob(256, 32, 0.3, S.SW_PERIODIC, method), u0[None], 0)
        assert np.array_equal(out[0], u0)


def test_translation_invariance_across_seams_bitwise():
    # shifting by s (not a multiple of W) moves every seam; the result must shift bitwise
    n, W, steps, shift = 2048, 64, 301, 45
    u0 = _init(n, seed=5)
    a = run_gpu(_prob(n, W, 0.3, S.SW_PERIODIC, S.SW_SWEPT), u0[None], steps)[0]
    b = run_gpu(_prob(n, W, 0.3, S.SW_PERIODIC, S.SW_SWEPT), np.roll(u0, shift)[None], steps)[0]
    assert np.array_equal(np.roll(a, shift), b)


def test_split_runs_equal_one_run():
    # checkpoint/resume: advancing 123 + 456 steps equals 579 steps bitwise
    import torch
    n, W = 4096, 256
    u0 = _init(n, seed=9)
    p = _prob(n, W, 0.37, S.SW_PERIODIC, S.SW_SWEPT)
    one = run_gpu(p, u0[None], 579)
    st = S.to_state(p, torch.as_tensor(u0, device="cuda"))
    with S.Handle(p) as h:
        h.sw_run(st, 123)
        h.sw_run(st, 456)
        two = S.to_fp64(p, st).cpu().numpy()
    assert np.array_equal(one, two)


def test_launch_counts():
    import torch
    n, W, steps = 16384, 64, 1000
    p = _prob(n, W, 0.25, S.SW_PERIODIC, S.SW_SWEPT)
    st = S.to_state(p, torch.as_tensor(_init(n), device="cuda"))
    with S.Handle(p) as h:
        h.sw_run(st, steps)
        # phases 0..ceil(1000/32) = 33 launches (vs 1000 per-step launches)
        assert h.sw_last_launch_count() == 33
        assert h.sw_tile_width() == 64
    q = _prob(n, W, 0.25, S.SW_PERIODIC, S.SW_PERSTEP)
    st = S.to_state(q, torch.as_tensor(_init(n), device="cuda"))
    with S.Handle(q) as h:
        h.sw_run(st, steps)
        assert h.sw_last_launch_count() == steps


def test_conservation_sum_is_deterministic_and_conserved():
    import torch
    n = 1 << 14
    u0 = _init(n, seed=4) + 0.5
    p = _prob(n, 64, 0.3, S.SW_PERIODIC, S.SW_SWEPT)
    st = S.to_state(p, torch.as_tensor(u0, device="cuda"))
    with S.Handle(p) as h:
        s0 = h.sw_conservation(st)
        assert s0 == h.sw_conservation(st)
        h.sw_run(st, 1000)
        s1 = h.sw_conservation(st)
    assert abs(s0[0] - float(np.sum(u0.astype(np.longdouble)))) < 1e-9
    assert abs(s1[0] - s0[0]) < 1e-9


def test_host_buffer_entry_point_matches_device_run():
    n, W, steps = 4096, 128, 200
    u0 = _init(n, seed=2)
    p = _prob(n, W, 0.3, S.SW_PERIODIC, S.SW_SWEPT)
    dev = run_gpu(p, u0[None], steps)[0]
    buf = np.ascontiguousarray(u0.copy())
    out = np.empty_like(buf)
    with S.Handle(p) as h:
        h.sw_run_host(buf.ctypes.data, out.ctypes.data, steps, 0)
    assert np.array_equal(out, dev)


@pytest.mark.parametrize("prec,offset,n", [(S.SW_FP32, 1, 8192), (S.SW_FP32, 4, 8192), (S.SW_FP32, 8, 8192),
                                           (S.SW_FP64, 1, 8192), (S.SW_FP64, 2, 8192), (S.SW_FP32_COMP, 1, 8192),
                                           (S.SW_FP64, 1, 1 << 21), (S.SW_FP64, 2, 1 << 21)])
@pytest.mark.parametrize("steps", [7, 8])
def test_perstep_on_any_state_alignment(prec, offset, n, steps):
    # the caller's state may start at any element: the per-step kernel picks its vector
    # width from the pointer's alignment, and every width gives the same bits. FP64 at
    # 2^21 cells: 4 (aligned), 2 (offset 2) and 1 (offset 1) cells per thread, the first
    # two with half the cells on the integer pipes, the last on the FP64 pipe alone
    import torch
    p = S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=S.SW_PERSTEP, n=n, r=0.3)
    u0 = I.heat_initial(I.heat_modes(n, 8, seed=offset))
    want = run_gpu(p, u0[None], steps)
    st = S.to_state(p, torch.as_tensor(u0, device="cuda"))
    big = torch.zeros(st.numel() + 16, dtype=st.dtype, device="cuda")
    view = big[offset:offset + st.numel()]  # every plane of the layout, starting `offset` elements in
    view.copy_(st)
    with S.Handle(p) as h:
        h.sw_run(view, steps)
        assert h.sw_sync_status() == S.SW_OK
        got = S.to_fp64(p, view.clone()).cpu().numpy().reshape(1, n)
    assert np.array_equal(got, want)
