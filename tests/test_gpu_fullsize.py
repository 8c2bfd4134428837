"""Parity at the full sizes of the configured workloads, in the launch configuration the
benchmark uses (swept with the register-resident Diamond kernel for periodic heat).

Where the oracle cannot step the whole run in seconds, it is checked on outputs it can
compute one by one or on a sub-domain that provably evolves identically, and through
properties that hold at any size:

- heat: the exact discrete solution of a sum of sine modes (closed form, sampled cells);
- Sod: cells outside the numerical domain of dependence (4 cells per step on each side of
  the interface: two 5-point stages) never change, bitwise; the oracle on the sub-domain around the interface
  (transmissive ends copy constant cells) equals the full-domain run bitwise; mass and
  energy are conserved and momentum changes by exactly the boundary pressure impulse;
- random Riemann problems: swept == per-step bitwise, periodic conservation, positivity.
"""
import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import batched
from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib, norm_rel, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _heat(n, W, r, prec=S.SW_FP64, method=S.SW_SWEPT):
    return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=method, n=n, r=r,
                     tile_width=W if method == S.SW_SWEPT else 0)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4])
def test_heat_n16384_r025_1000_steps_w64(seed):
    n, steps, r = 16384, 1000, 0.25
    u0 = I.heat_initial(I.heat_modes(n, 8, seed=seed))
    sw = run_gpu(_heat(n, 64, r), u0[None], steps)
    ps = run_gpu(_heat(n, 64, r, method=S.SW_PERSTEP), u0[None], steps)
    assert np.array_equal(sw, ps)
    assert norm_rel(sw, oracle.heat_run(u0, r, steps)[None]) <= 1e-12


@pytest.mark.parametrize("W", [128, 512])
def test_heat_n2_24_50000_steps(W):
    n, steps = 1 << 24, 50_000
    modes = I.heat_modes(n, 32, seed=2024)
    r = I.heat_r(2024)
    u0 = I.heat_initial(modes)
    sw = run_gpu(_heat(n, W, r), u0[None], steps)[0]
    ps = run_gpu(_heat(n, W, r, method=S.SW_PERSTEP), u0[None], steps)[0]
    assert np.array_equal(sw, ps)
    idx = np.linspace(0, n - 1, 8192).astype(np.int64)
    want = oracle.heat_modes(n, r, steps, modes.amps, modes.ks, idx)
    assert np.max(np.abs(sw[idx] - want)) / np.max(np.abs(want)) <= 1e-12


def test_heat_precision_n2_22_r04_100000_steps():
    n, steps, r = 1 << 22, 100_000, 0.4
    modes = I.heat_modes(n, 32, seed=4)
    u0 = I.heat_initial(modes)
    idx = np.linspace(0, n - 1, 8192).astype(np.int64)
    want = oracle.heat_modes(n, r, steps, modes.amps, modes.ks, idx)
    errs = {}
    for prec in (S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP):
        got = run_gpu(_heat(n, 512, r, prec), u0[None], steps)[0][idx]
        errs[prec] = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert errs[S.SW_FP64] <= 1e-12
    assert errs[S.SW_FP32_COMP] <= 1e-9          # compensated: ~1e-10 measured
    assert errs[S.SW_FP32_COMP] * 100 < errs[S.SW_FP32]  # plain FP32 stagnates on these modes


@pytest.mark.slow
def test_sod_n2_20_20000_steps():
    import torch
    n, steps = 1 << 20, 20_000
    lam = I.sod_lambda()
    q0 = I.sod(n)
    p_sw = S.Problem(scheme=S.SW_EULER, precision=S.SW_FP64, boundary=S.SW_TRANSMISSIVE, method=S.SW_SWEPT,
                     n=n, dt_dx=lam, gamma=I.GAMMA, tile_width=512)
    p_ps = S.Problem(scheme=S.SW_EULER, precision=S.SW_FP64, boundary=S.SW_TRANSMISSIVE, method=S.SW_PERSTEP,
                     n=n, dt_dx=lam, gamma=I.GAMMA)
    sw = run_gpu(p_sw, q0, steps)
    ps = run_gpu(p_ps, q0, steps)
    assert np.array_equal(sw, ps)
    # outside the domain of dependence nothing moves
    reach = 4 * steps + 2
    mid = n // 2
    assert np.array_equal(sw[:, : mid - reach], q0[:, : mid - reach])
    assert np.array_equal(sw[:, mid + reach:], q0[:, mid + reach:])
    # the oracle on the sub-domain around the interface is the full-domain result
    lo, hi = mid - reach - 8, mid + reach + 8
    ref = oracle.euler_run(q0[:, lo:hi].copy(), lam, I.GAMMA, steps, oracle.TRANSMISSIVE)
    assert np.array_equal(sw[:, lo:hi], ref)
    # mass and energy conserved; momentum changes by the pressure difference at the ends
    s0 = q0.sum(axis=1, dtype=np.longdouble)
    s1 = sw.sum(axis=1, dtype=np.longdouble)
    assert abs(float(s1[0] - s0[0])) < 1e-6 and abs(float(s1[2] - s0[2])) < 1e-6
    impulse = steps * lam * (I.SOD_LEFT[2] - I.SOD_RIGHT[2])
    assert abs(float(s1[1] - s0[1]) - impulse) < 1e-6
    torch.cuda.synchronize()


@pytest.mark.slow
def test_random_riemann_n2_22_precisions():
    # the precision workload as the benchmark runs it: N = 2^22, 64 random Riemann segments,
    # 4000 steps, periodic, swept at W = 512 (flattened); FP64 equals the oracle bitwise on
    # sampled windows (each run on the window plus its domain of dependence, 4 cells per
    # step each side); FP32 and hi/lo: error against the FP64 run within the stated
    # bounds, positive, no growth of total variation or extrema
    import torch
    from bench import euler_quality, norm_errors
    n, steps = 1 << 22, 4000
    q0 = I.riemann_initial(I.riemann_segments(n, 64, seed=4))
    lam = I.riemann_lambda()

    def prob(prec, method):
        return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=S.SW_PERIODIC, method=method, n=n,
                         dt_dx=lam, gamma=I.GAMMA, tile_width=512 if method == S.SW_SWEPT else 0)

    f64 = run_gpu(prob(S.SW_FP64, S.SW_SWEPT), q0, steps)
    assert np.array_equal(f64, run_gpu(prob(S.SW_FP64, S.SW_PERSTEP), q0, steps))
    reach, w = 4 * steps + 8, 512
    for a in (0, 1_000_003, 2_500_000, n - w):
        sub = np.ascontiguousarray(np.take(q0, np.arange(a - reach, a + w + reach), axis=1, mode="wrap"))
        ref = oracle.euler_run(sub, lam, I.GAMMA, steps, oracle.TRANSMISSIVE)
        assert np.array_equal(f64[:, a:a + w], ref[:, reach:reach + w]), a
    s0 = q0.sum(axis=1, dtype=np.longdouble)
    s1 = f64.sum(axis=1, dtype=np.longdouble)
    assert np.all(np.abs((s1 - s0).astype(np.float64)) < 1e-8 * np.abs(s0.astype(np.float64)) + 1e-8)
    q_ref = euler_quality(f64)
    bounds = {"rho": (0.4, 3e-2), "m": (0.4, 4e-2), "E": (0.05, 3e-3)}
    for prec in (S.SW_FP32, S.SW_FP32_COMP):
        got = run_gpu(prob(prec, S.SW_SWEPT), q0, steps)
        assert np.array_equal(got, run_gpu(prob(prec, S.SW_PERSTEP), q0, steps))
        err = norm_errors(got, f64, ("rho", "m", "E"))
        for v, (mx, l2) in bounds.items():
            assert err[v]["max_rel"] <= mx and err[v]["l2_rel"] <= l2, (prec, v, err[v])
        q = euler_quality(got)
        assert q["finite"] and q["min_rho"] > 0 and q["min_p"] > 0
        assert q["tv_rho"] <= q_ref["tv_rho"] * (1 + 1e-3) and q["tv_p"] <= q_ref["tv_p"] * (1 + 1e-3)
        assert q["extrema_rho"] <= q_ref["extrema_rho"] + 2
    torch.cuda.synchronize()


@pytest.mark.slow
def test_batched_subset_full_length_10000_steps():
    # 64 problems of the batched workload (lengths 2^10 .. 2^13), FP32 hi/lo, tuned widths,
    # 10,000 steps: every problem bitwise equal to its own run
    import torch
    items = I.batch_problems(64, seed=7, lo_exp=10.0, hi_exp=13.0)
    bt = batched.build(items, 10_000)
    bt.batch.sw_batch_run()
    assert bt.batch.sw_batch_status() == S.SW_OK
    for p, st, it in zip(bt.problems, bt.states, items):
        got = S.to_fp64(p, st).cpu().numpy()
        want = run_gpu(p, it.planes, 10_000)
        assert np.array_equal(got, want)
    bt.batch.close()
    torch.cuda.synchronize()


def test_large_grid_fp32_swept_equals_perstep():
    # 2^27 cells (512 MB of state, 2 GB of flanks at W = 1024)
    n, steps = 1 << 27, 600
    u0 = np.zeros(n)
    u0[: 1 << 20] = I.heat_initial(I.heat_modes(1 << 20, 4, seed=1))
    sw = run_gpu(_heat(n, 1024, 0.3, S.SW_FP32), u0[None], steps)
    ps = run_gpu(_heat(n, 1024, 0.3, S.SW_FP32, S.SW_PERSTEP), u0[None], steps)
    assert np.array_equal(sw, ps)


@pytest.mark.parametrize("prec", [S.SW_FP64, S.SW_FP32])
def test_heat2d_8192_squared_2048_steps(prec):
    # the benchmark's 2D workload in its launch configuration (W = 64): swept == per-step bitwise
    # and the exact mode solution of the oracle at sampled cells (relative to the initial maximum)
    import torch
    n, steps, r = 8192, 2048, 0.2
    m = I.heat2d_modes(n, n, 16, seed=6, kmax=16)
    u0 = I.heat2d_initial(m)
    dt = torch.float64 if prec == S.SW_FP64 else torch.float32
    outs = []
    for method in (S.SW_SWEPT, S.SW_PERSTEP):
        p = S.Heat2D(precision=prec, method=method, tile_width=64 if method == S.SW_SWEPT else 0, nx=n, ny=n,
                     rx=r, ry=r)
        st = torch.as_tensor(u0.reshape(-1), device="cuda").to(dt).clone()
        with S.Handle2D(p) as h:
            h.sw2d_run(st, steps)
        outs.append(st)
    assert torch.equal(outs[0], outs[1])
    rng = np.random.default_rng(11)
    ii, jj = rng.integers(0, n, 4096), rng.integers(0, n, 4096)
    want = oracle.heat2d_modes(n, n, r, r, steps, m.amps, m.kx, m.ky, m.fx, m.fy, ii, jj)
    got = outs[0].double().cpu().numpy().reshape(n, n)[jj, ii]
    err = np.max(np.abs(got - want)) / np.max(np.abs(u0))
    assert err <= (1e-12 if prec == S.SW_FP64 else 1e-5), err
    torch.cuda.synchronize()
