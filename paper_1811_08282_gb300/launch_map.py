"""Launch-condition map and power-law fit of the swept rule on one GPU.

Section 5 maps the time per time step of Swept and Classic over the launch
conditions (threads per block, i.e. tile width W) and grid size N, then takes
the best W per N and fits the Swept time per step to a power law y = A x^b
(Table 1, least squares, with R^2). This module runs that experiment on this
library: every (N, W) for the swept method, and the per-step ("Classic") kernel
once per N (it has no tile width), each timed with CUDA events after one
untimed run. With --work-factors the map gains the paper's third axis, the GPU
work factor of Eq. 1: each (N, W) is also run split between the GPU and
--threads host threads (sw_run_hybrid; 0 = the GPU alone), timed on the host
clock around the synchronous call.

    python -m paper_1811_08282_gb300.launch_map --scheme heat --precision fp64
    python -m paper_1811_08282_gb300.launch_map --scheme euler --precision fp64 --exps 14 20
    python -m paper_1811_08282_gb300.launch_map --scheme heat --exps 19 23 --step 2 \
        --work-factors 0 32 64 96 --threads 16
    python -m paper_1811_08282_gb300.launch_map --scheme euler --forms --exps 14 22

--forms (Euler) is Section 4.3's experiment (Fig. 3): the time per step of the two
data-structure strategies, lengthened (four 3-point sub-steps per step) and
flattened (two 5-point stages), each with the swept rule (best W) and per step.

Output: one JSON line per measurement ({"kind": "point", ...}), one per N with
the best W and the swept speedup over per-step ({"kind": "best", ...}), and one
with the fit ({"kind": "fit", "A_us": A, "b": b, "r2": R^2}), where the fit is
ordinary least squares of log y on log x and R^2 is taken in that log space.
Heat uses 32 sine modes (r = 0.3, periodic); Euler the Sod problem (transmissive).
"""
from __future__ import annotations

import argparse
import json
import math

from . import inputs as I
from . import swept as S

PREC = {"fp64": S.SW_FP64, "fp32": S.SW_FP32, "fp32_comp": S.SW_FP32_COMP}


def power_fit(xs, ys):
    """Least-squares fit of log y = log A + b log x; returns (A, b, R^2 in log space)."""
    lx = [math.log(x) for x in xs]
    ly = [math.log(y) for y in ys]
    n = len(lx)
    mx, my = sum(lx) / n, sum(ly) / n
    sxx = sum((a - mx) ** 2 for a in lx)
    sxy = sum((a - mx) * (b - my) for a, b in zip(lx, ly))
    b = sxy / sxx
    a = my - b * mx
    ss_res = sum((y - (a + b * x)) ** 2 for x, y in zip(lx, ly))
    ss_tot = sum((y - my) ** 2 for y in ly)
    return math.exp(a), b, (1.0 - ss_res / ss_tot) if ss_tot > 0 else 1.0


def steps_for(scheme: str, n: int, target: float, wmax: int, cap: int) -> int:
    """Time steps for one measurement: about `target` cell-steps, at least four
    phases of the widest tile (W/2 levels per phase; Euler has 4 levels per step),
    at most `cap`."""
    lo = 2 * wmax if scheme == "heat" else wmax // 2
    return int(min(max(lo, target // n), max(lo, cap)))


def _problem(scheme, precision, n, method, W, flags=0):
    if scheme == "heat":
        return S.Problem(scheme=S.SW_HEAT, precision=precision, boundary=S.SW_PERIODIC, method=method,
                         n=n, r=0.3, tile_width=W, flags=flags)
    return S.Problem(scheme=S.SW_EULER, precision=precision, boundary=S.SW_TRANSMISSIVE, method=method,
                     n=n, dt_dx=I.sod_lambda(), gamma=I.GAMMA, tile_width=W, flags=flags)


def _initial(scheme, n):
    if scheme == "heat":
        return I.heat_initial(I.heat_modes(n, 32, seed=1))[None]
    return I.sod(n)


def measure(scheme: str, precision: int, n: int, method: int, W: int, steps: int, reps: int,
            work_factor: int = 0, threads: int = 0, flags: int = 0) -> float:
    """Seconds per run of `steps` time steps (minimum over `reps` timed runs after one
    untimed run), state resident on the device, reset from a device copy each run;
    work_factor > 0: the hybrid run with `threads` host threads."""
    import time
    import torch
    p = _problem(scheme, precision, n, method, W, flags)
    x0 = torch.as_tensor(_initial(scheme, n).reshape(-1), device="cuda")
    fresh = S.to_state(p, x0)
    st = fresh.clone()
    ts = []
    with S.Handle(p) as h:
        for i in range(reps + 1):
            st.copy_(fresh)
            if work_factor > 0:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h.sw_run_hybrid(st, steps, work_factor, threads)
                if i:
                    ts.append(time.perf_counter() - t0)
                continue
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            h.sw_run(st, steps)
            b.record()
            b.synchronize()
            if i:
                ts.append(a.elapsed_time(b) / 1e3)
        rc = h.sw_sync_status()
        if rc < 0:
            raise S.SweptError(rc, "launch_map")
    return min(ts)


def run_map(scheme: str, precision: int, exps, widths, target: float, cap: int, reps: int, emit=print,
            fit_exps=None, work_factors=(0,), threads: int = 1):
    """Measure every (N, W) and per-step per N; fit the best swept time per step over
    N in 2^fit_exps[0] .. 2^fit_exps[1] (default: every measured N)."""
    best = []
    for e in exps:
        n = 1 << e
        ws = [W for W in widths if n % W == 0 and n >= 2 * W]
        steps = steps_for(scheme, n, target, max(ws), cap)
        row = {}
        for W in ws:
            for wf in work_factors:
                if wf > 0:
                    try:
                        S.sw_hybrid_split(n // W, wf, threads)
                    except S.SweptError:
                        continue  # too few tiles for this split
                t = measure(scheme, precision, n, S.SW_SWEPT, W, steps, reps, wf, threads)
                row[(W, wf)] = t
                emit(json.dumps({"kind": "point", "scheme": scheme, "precision": precision, "n": n,
                                 "method": "swept" if wf == 0 else "hybrid", "W": W, "work_factor": wf,
                                 "threads": threads if wf else 0, "steps": steps, "us_per_step": t / steps * 1e6,
                                 "gcell_steps_per_s": n * steps / t / 1e9}))
        tc = measure(scheme, precision, n, S.SW_PERSTEP, 0, steps, reps)
        emit(json.dumps({"kind": "point", "scheme": scheme, "precision": precision, "n": n, "method": "perstep",
                         "W": None, "steps": steps, "us_per_step": tc / steps * 1e6,
                         "gcell_steps_per_s": n * steps / tc / 1e9}))
        wb = min(row, key=row.get)
        best.append((n, row[wb] / steps * 1e6))
        emit(json.dumps({"kind": "best", "scheme": scheme, "precision": precision, "n": n, "W": wb[0],
                         "work_factor": wb[1], "swept_us_per_step": row[wb] / steps * 1e6,
                         "perstep_us_per_step": tc / steps * 1e6, "speedup": tc / row[wb]}))
    lo, hi = fit_exps if fit_exps else (0, 62)
    pts = [(n, y) for n, y in best if (1 << lo) <= n <= (1 << hi)]
    A, b, r2 = power_fit([n for n, _ in pts], [y for _, y in pts])
    emit(json.dumps({"kind": "fit", "scheme": scheme, "precision": precision, "A_us": A, "b": b, "r2": r2,
                     "n_range": [pts[0][0], pts[-1][0]]}))
    return best, (A, b, r2)


def run_forms(precision: int, exps, widths, target: float, cap: int, reps: int, emit=print):
    """Section 4.3 / Fig. 3 on this GPU: µs per step of the four Euler forms per N."""
    forms = {"swept_lengthened": (S.SW_SWEPT, S.SW_FLAG_LENGTHENED), "swept_flattened": (S.SW_SWEPT, S.SW_FLAG_FLATTENED),
             "perstep_flattened": (S.SW_PERSTEP, 0), "perstep_lengthened": (S.SW_PERSTEP, S.SW_FLAG_LENGTHENED)}
    for e in exps:
        n = 1 << e
        ws = [W for W in widths if n % W == 0 and n >= 2 * W and W % 4 == 0 and W >= 8]
        steps = steps_for("euler", n, target, max(ws), cap)
        row = {}
        for name, (method, flags) in forms.items():
            if method == S.SW_SWEPT:
                ts = {W: measure("euler", precision, n, method, W, steps, reps, flags=flags) for W in ws}
                W = min(ts, key=ts.get)
                row[name] = (ts[W] / steps * 1e6, W)
            else:
                row[name] = (measure("euler", precision, n, method, 0, steps, reps, flags=flags) / steps * 1e6, None)
        emit(json.dumps({"kind": "forms", "precision": precision, "n": n, "steps": steps,
                         **{k: {"us_per_step": v[0], "W": v[1]} for k, v in row.items()}}))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--scheme", choices=("heat", "euler"), default="heat")
    ap.add_argument("--precision", choices=tuple(PREC), default="fp64")
    ap.add_argument("--exps", type=int, nargs=2, default=(14, 24), help="log2 N range, inclusive")
    ap.add_argument("--step", type=int, default=1, help="log2 N stride")
    ap.add_argument("--widths", type=int, nargs="+", default=(32, 64, 128, 256, 512, 1024))
    ap.add_argument("--target", type=float, default=None, help="cell-steps per measurement")
    ap.add_argument("--cap", type=int, default=20000, help="most time steps per measurement")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--fit-exps", type=int, nargs=2, default=None,
                    help="log2 N range of the power-law fit (default: all measured)")
    ap.add_argument("--work-factors", type=int, nargs="+", default=[0],
                    help="GPU work factors (Eq. 1) to map; 0 = the GPU alone")
    ap.add_argument("--threads", type=int, default=None, help="host threads of the hybrid runs (default: all cores)")
    ap.add_argument("--forms", action="store_true",
                    help="Euler: time the lengthened and flattened forms, swept and per step (Section 4.3)")
    a = ap.parse_args(argv)
    import torch
    from . import build
    build.build()
    torch.cuda.set_device(0)
    target = a.target if a.target is not None else (2.0 ** 32 if a.scheme == "heat" else 2.0 ** 28)
    if a.forms:
        run_forms(PREC[a.precision], range(a.exps[0], a.exps[1] + 1, a.step), a.widths,
                  a.target if a.target is not None else 2.0 ** 28, a.cap, a.reps)
        return
    import os
    threads = a.threads or (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    run_map(a.scheme, PREC[a.precision], range(a.exps[0], a.exps[1] + 1, a.step), a.widths, target, a.cap, a.reps,
            fit_exps=a.fit_exps, work_factors=a.work_factors, threads=threads)


if __name__ == "__main__":
    main()
