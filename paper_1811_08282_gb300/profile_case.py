"""Run one configured case through the C ABI (for profilers and quick timing).

    python -m paper_1811_08282_gb300.profile_case --scheme heat --precision fp64 \
        --method swept --n 16777216 --steps 2048 --width 1024 [--repeat 1] [--generic]
    python -m paper_1811_08282_gb300.profile_case --scheme heat2d --precision fp64 \
        --nx 4096 --ny 4096 --steps 256 --width 64
    python -m paper_1811_08282_gb300.profile_case --scheme batch --count 1024 --steps 200

Inputs are the seeded synthetic states of ``inputs`` (heat: 32 sine modes;
Euler: Sod, or 64 random Riemann segments with --init riemann). Prints the
CUDA-event time of the last repeat and the cell-update rate.
"""
from __future__ import annotations

import argparse
import json

from . import inputs as I
from . import swept as S

PREC = {"fp64": S.SW_FP64, "fp32": S.SW_FP32, "fp32_comp": S.SW_FP32_COMP}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scheme", choices=("heat", "euler", "heat2d", "batch"), default="heat")
    ap.add_argument("--count", type=int, default=1024, help="batch: problems (the batched workload's first ones)")
    ap.add_argument("--nx", type=int, default=4096, help="heat2d: grid width")
    ap.add_argument("--ny", type=int, default=4096, help="heat2d: grid height")
    ap.add_argument("--precision", choices=tuple(PREC), default="fp64")
    ap.add_argument("--method", choices=("swept", "perstep"), default="swept")
    ap.add_argument("--boundary", choices=("periodic", "transmissive"), default=None)
    ap.add_argument("--init", choices=("sod", "riemann"), default="sod")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--steps", type=int, default=2048)
    ap.add_argument("--width", type=int, default=1024)
    ap.add_argument("--r", type=float, default=None,
                    help="heat: r (default 0.3); heat2d: rx = ry (default 0.2, stable: rx + ry <= 1/2)")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--threads", type=int, default=0, help="heat2d swept: threads per CTA (0: the default)")
    ap.add_argument("--bridge-threads", type=int, default=0, help="heat2d swept: threads per bridges CTA")
    ap.add_argument("--generic", action="store_true", help="force the generic phase kernel (SW_FLAG_GENERIC)")
    ap.add_argument("--flags", type=int, default=0, help="further SW_FLAG_* bits (e.g. 8: flattened Euler)")
    a = ap.parse_args(argv)

    import torch
    from . import build
    build.build()
    if a.scheme == "heat2d":
        return run2d(a)
    if a.scheme == "batch":
        return run_batch(a)
    heat = a.scheme == "heat"
    if a.r is None:
        a.r = 0.3
    bc = a.boundary or ("periodic" if heat else "transmissive")
    p = S.Problem(scheme=S.SW_HEAT if heat else S.SW_EULER, precision=PREC[a.precision],
                  boundary=S.SW_PERIODIC if bc == "periodic" else S.SW_TRANSMISSIVE,
                  method=S.SW_SWEPT if a.method == "swept" else S.SW_PERSTEP, n=a.n, r=a.r,
                  dt_dx=(I.sod_lambda() if a.init == "sod" else I.riemann_lambda()), gamma=I.GAMMA,
                  tile_width=a.width if a.method == "swept" else 0,
                  flags=(S.SW_FLAG_GENERIC if a.generic else 0) | a.flags)
    if heat:
        x = I.heat_initial(I.heat_modes(a.n, 32, seed=1))
    elif a.init == "sod":
        x = I.sod(a.n)
    else:
        x = I.riemann_initial(I.riemann_segments(a.n, 64, 1))
    st = S.to_state(p, torch.as_tensor(x.reshape(-1), device="cuda"))
    fresh = st.clone()
    t = None
    with S.Handle(p) as h:
        for _ in range(a.repeat):
            st.copy_(fresh)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.sw_run(st, a.steps)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
        launches = h.sw_last_launch_count()
        rc = h.sw_sync_status()
    print(json.dumps({"scheme": a.scheme, "precision": a.precision, "method": a.method, "n": a.n,
                      "steps": a.steps, "width": a.width, "generic": a.generic, "flags": a.flags, "launches": launches, "seconds": t,
                      "gcell_updates_per_s": a.n * a.steps / t / 1e9, "status": rc}))
    return 0 if rc == 0 else 1


def run_batch(a) -> int:
    """The batched workload's first `count` problems (FP32 hi/lo unless --precision says
    otherwise) at the widths the tuner usually picks (heat 1024, Euler flattened 256), one
    persistent launch from its CUDA graph after one untimed run."""
    import torch
    from . import batched
    items = batched.default_items(4096, seed=7)[: a.count]
    widths = {"heat": (1024, 0), "euler": (256, S.SW_FLAG_FLATTENED)}
    prec = PREC[a.precision] if a.precision != "fp64" else S.SW_FP32_COMP
    bt = batched.build(items, a.steps, precision=prec, widths=widths)
    bt.batch.sw_batch_run()
    rc = bt.batch.sw_batch_status()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    bt.batch.sw_batch_run()
    e1.record()
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    rc = rc or bt.batch.sw_batch_status()
    print(json.dumps({"scheme": "batch", "problems": len(items), "cells": bt.cells, "steps": a.steps,
                      "items": bt.batch.sw_batch_items(), "seconds": t,
                      "gcell_steps_per_s": bt.cells * a.steps / t / 1e9, "status": rc}))
    bt.batch.close()
    return 0 if rc == 0 else 1


def run2d(a) -> int:
    """The 2D heat case: 16 seeded separable modes, r = a.r in both directions."""
    import torch
    if a.r is None:
        a.r = 0.2
    p = S.Heat2D(precision=PREC[a.precision], method=S.SW_SWEPT if a.method == "swept" else S.SW_PERSTEP,
                 tile_width=a.width if a.method == "swept" else 0, nx=a.nx, ny=a.ny, rx=a.r, ry=a.r)
    x = I.heat2d_initial(I.heat2d_modes(a.nx, a.ny, 16, seed=1, kmax=16))
    dt = torch.float64 if p.precision == S.SW_FP64 else torch.float32
    fresh = torch.as_tensor(x.reshape(-1), device="cuda").to(dt)
    st = fresh.clone()
    t = None
    with S.Handle2D(p) as h:
        if a.method == "swept":
            h.sw2d_set_threads(a.threads, a.bridge_threads)
        for _ in range(a.repeat):
            st.copy_(fresh)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            h.sw2d_run(st, a.steps)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1) / 1e3
        launches = h.sw2d_last_launch_count()
    print(json.dumps({"scheme": "heat2d", "precision": a.precision, "method": a.method, "nx": a.nx, "ny": a.ny,
                      "steps": a.steps, "width": a.width, "threads": a.threads,
                      "bridge_threads": a.bridge_threads, "launches": launches, "seconds": t,
                      "gcell_updates_per_s": a.nx * a.ny * a.steps / t / 1e9}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
