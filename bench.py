#!/usr/bin/env python
"""Benchmark: Gcell-updates/s of the swept FP64 heat path on one GB300.

Workload (one bench step): the FTCS heat equation, FP64, periodic grid of
N = 2^24 cells, r drawn U[0.1, 0.45] (seeded), initial state a sum of 32 seeded
sine modes, advanced 50,000 time steps by the swept rule (Up Triangle, Diamonds,
Down Triangle; Section 4.1) with the tile base width chosen by a short timed
sweep over W in {32, ..., 1024} (the paper's advice in Section 6: tune over a
limited number of steps). One cell-update = one cell advanced one time step.

Printed (rank 0, one JSON line): the swept value, the per-step ("Classic")
kernel and the FP32 / FP32-compensated forms on the same grid with their errors
against the FP64 oracle's closed form, a roofline entry for the dominant kernel
(the Diamond phase) and the oracle timed on the host cores.

``--impl reference`` times the FP64 CPU oracle itself (the only reference this
paper has: no code was published with it) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 24
STEPS = 50_000
MODES = 32
SEED = 2024
WIDTHS = (32, 64, 128, 256, 512, 1024)
TUNE_STEPS = 4096
METRIC = "Gcell-updates/s, swept vs per-step kernel, FP32/FP64 at stated err; % roofline"
UNIT = "Gcell-updates/s"
WORKLOAD = "heat FTCS FP64 periodic N=2^24, r~U[0.1,0.45] seed 2024, 32 sine modes, 50000 steps, swept"
FLOPS_PER_UPDATE = 5  # a + b, fma(-2, u, .), fma(r, ., u): 1 add + 2 FMA
# FP64 peak: 152 SMs x 2 FP64 FMA / clock / SM x 2 flop x 2.07 GHz (the GB300
# part's 1.25 TFLOP/s dense FP64 at its maximum SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# The FP64 heat kernels run half their cells on the integer pipes (the same bits), so
# their ceiling is set by two pipes: the FP64 pipe (2 instructions / clock / SM) and
# the integer ALU pipe (64 lanes / clock / SM), each divided by the instructions per
# update it carries (counted by ncu, recorded with the kernel's source hash).
FP64_INST_PER_S = 152 * 2 * 2.07e9
ALU_LANE_INST_PER_S = 152 * 64 * 2.07e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the headline, time the other paper-shaped workloads (one JSON line each)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), \
        int(os.environ.get("WORLD_SIZE", "1"))


def I_mod():
    from paper_1811_08282_gb300 import inputs
    return inputs


def initial_state():
    from paper_1811_08282_gb300 import inputs as I
    modes = I.heat_modes(N, MODES, seed=SEED)
    r = I.heat_r(SEED)
    return modes, r, I.heat_initial(modes)


# sources that define each timed kernel (a recorded traffic figure is void once they change)
KERNEL_SOURCES = {
    "k_heat_fold": ("common.cuh", "heat.cuh", "flanks.cuh", "fp64_soft.cuh", "fold_heat.cuh"),
    "k_swept_phase": ("common.cuh", "heat.cuh", "heat_policy.cuh", "flanks.cuh", "swept_phase.cuh"),
}


def kernel_source_sha(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1811_08282_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded(kernel: str, key: str, field: str = "bytes_per_launch"):
    """A figure from the committed ncu summaries (DRAM bytes per launch, instructions
    per update), if the kernel is unchanged since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split("=", 1)
        vals[k.strip()] = v.strip()
    if vals.get(f"{kernel}.source_sha") != kernel_source_sha(kernel) or f"{key}.{field}" not in vals:
        return None
    return float(vals[f"{key}.{field}"])


def recorded_traffic(kernel: str, key: str):
    return recorded(kernel, key, "bytes_per_launch")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.path = None
        self.uuid = uuid

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for rec in csv.reader(io.StringIO(open(self.path).read())):
            if len(rec) < 9:
                continue
            try:
                rows.append(dict(sm=float(rec[1]), smax=float(rec[2]), power=float(rec[3]),
                                 hw=rec[5].strip(), hwt=rec[6].strip(), swt=rec[7].strip(), pcap=rec[8].strip()))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(t_local: float, world: int, device=None) -> float:
    """Slowest rank's time (every rank gets it); the identity on one rank."""
    if world <= 1:
        return float(t_local)
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(units_per_rank: float, t_max: float, world: int) -> float:
    """Whole-job Gcell-updates/s: every rank (an independent replica) advances the same
    units; the job takes as long as its slowest rank."""
    return world * units_per_rank / t_max / 1e9


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import numpy as np
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_1811_08282_gb300 import build
    build.build()
    from paper_1811_08282_gb300 import swept as S

    modes, r, u0 = initial_state()
    stream = torch.cuda.current_stream()
    u0_dev = torch.as_tensor(u0, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def problem(prec, method, W):
        return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=method, n=N, r=r,
                         tile_width=W if method == S.SW_SWEPT else 0)

    def timed_run(h, state, steps, reset_from=None):
        if reset_from is not None:
            state.copy_(reset_from)
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h.sw_run(state, steps, stream)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    # 1) tile width: short timed sweep (Section 6: tune over a limited number of steps)
    sweep = {}
    for W in WIDTHS:
        p = problem(S.SW_FP64, S.SW_SWEPT, W)
        st = S.to_state(p, u0_dev)
        with S.Handle(p) as h:
            timed_run(h, st, 64, u0_dev)
            t = timed_run(h, st, TUNE_STEPS, u0_dev)
        sweep[W] = N * TUNE_STEPS / t / 1e9
        del st
    best_w = max(sweep, key=sweep.get)

    # 2) warm-up and K timed steps of the full workload at the chosen width
    p = problem(S.SW_FP64, S.SW_SWEPT, best_w)
    state = S.to_state(p, u0_dev)
    h = S.Handle(p)
    for _ in range(args.warmup):
        timed_run(h, state, STEPS, u0_dev)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    times = []
    launches = 0
    barrier()
    sampler.start()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed launches
    wall0 = time.perf_counter()
    for k in range(args.steps):
        if k == args.steps - 1:
            h.sw_set_timing(STEPS // (best_w // 2) + 2)
        times.append(timed_run(h, state, STEPS, u0_dev))
        launches += h.sw_last_launch_count()
    barrier()
    wall = time.perf_counter() - wall0
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    traced = h.sw_launch_times()
    h.sw_set_timing(0)
    final = S.to_fp64(p, state)[0]
    t_total = max_over_ranks(sum(times), world, dev)
    value = whole_job_rate(N * STEPS * args.steps, t_total, world)
    ms_per_step = t_total / args.steps * 1e3

    # roofline of the dominant kernel (Diamond phases), from the traced launches
    diamonds = [ms for ms, kind in traced if kind == 1]
    H = best_w // 2
    flops_per_launch = N * H * FLOPS_PER_UPDATE
    achieved = flops_per_launch / (statistics.mean(diamonds) / 1e3) / 1e12 if diamonds else None
    # periodic heat at W = 32K runs its Diamonds on the register-resident kernel; the DRAM
    # traffic of one Diamond launch is the flanks in and out (W-independent: 4 N values)
    fold = best_w in (128, 256, 512, 1024)
    kname = "k_heat_fold" if fold else "k_swept_phase"
    traffic = recorded_traffic(kname, f"{kname}.heat_fp64.n2^24")
    # the register-resident kernel at W = 128 / 256 puts every other cell on the integer
    # pipes: its ceiling is the busier of the FP64 and ALU pipes for its instruction mix
    peak, peak_source = FP64_PEAK_TFLOPS, \
        "FP64 1.25 TFLOP/s class: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz (nominal, recipe)"
    fp64_ipu = recorded(kname, f"{kname}.heat_fp64.w{best_w}", "fp64_inst_per_update") if fold else None
    alu_ipu = recorded(kname, f"{kname}.heat_fp64.w{best_w}", "alu_inst_per_update") if fold else None
    if fp64_ipu and alu_ipu:
        ceiling = min(FP64_INST_PER_S / fp64_ipu, ALU_LANE_INST_PER_S / alu_ipu)  # updates/s
        peak = ceiling * FLOPS_PER_UPDATE / 1e12
        peak_source = (f"pipe ceiling of the FP64 + integer-pipe kernel, in FP64-equivalent flops (5 per update): "
                       f"min(FP64 pipe 152 SM x 2/clk x 2.07 GHz / {fp64_ipu:.3f} FP64 instr per update, "
                       f"ALU pipe 152 SM x 64 lanes/clk x 2.07 GHz / {alu_ipu:.2f} ALU instr per update) "
                       f"= {ceiling / 1e9:.1f} G updates/s (instruction counts: ncu, profiles/traffic.txt)")
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "fp64_pipe_peak": FP64_PEAK_TFLOPS,
                "frac_of_fp64_pipe_peak": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "kernel": (f"k_heat_fold<{best_w // 32}, FoldF64> (Diamond phases)" if fold
                           else "k_swept_phase<HeatPolicy<FP64>> (Diamond phases)"),
                "launches_traced": len(diamonds),
                "avg_launch_ms": statistics.mean(diamonds) if diamonds else None,
                "flops_per_launch": flops_per_launch,
                "peak_source": peak_source}

    # 3) end to end through the C ABI with host buffers (H2D + run + D2H inside the region)
    host_in = torch.empty(N, dtype=torch.float64, pin_memory=True)
    host_in.copy_(torch.as_tensor(u0))
    host_out = torch.empty_like(host_in)
    e2e_times = []
    for k in range(max(1, min(args.steps, 2)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.sw_run_host(host_in.data_ptr(), host_out.data_ptr(), STEPS, stream)
        t1 = time.perf_counter()
        if k > 0:
            e2e_times.append(t1 - t0)
    e2e = {"value": N * STEPS / statistics.mean(e2e_times) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8,
           "api": "sw_run_host (pinned host buffers)"}
    h.close()

    # 4) comparisons on the same grid: per-step kernel and the FP32 forms
    compare = {}
    outputs = {("fp64", "swept", STEPS): final.cpu()}
    for name, prec in (("fp64", S.SW_FP64), ("fp32", S.SW_FP32), ("fp32_comp", S.SW_FP32_COMP)):
        if name == "fp64":
            w_prec = best_w
        else:  # the same short timed sweep as for FP64
            rates = {}
            for W in WIDTHS[2:]:
                pw = problem(prec, S.SW_SWEPT, W)
                st = S.to_state(pw, u0_dev)
                fresh = st.clone()
                with S.Handle(pw) as hw:
                    timed_run(hw, st, 64, fresh)
                    rates[W] = TUNE_STEPS / timed_run(hw, st, TUNE_STEPS, fresh)
                del st, fresh
            w_prec = max(rates, key=rates.get)
        for method in ("swept", "perstep"):
            if name == "fp64" and method == "swept":
                compare["fp64_swept"] = {"value": value / world, "steps": STEPS, "W": best_w}
                continue
            steps = STEPS if method == "swept" else 5000
            W = w_prec
            pp = problem(prec, S.SW_SWEPT if method == "swept" else S.SW_PERSTEP, W)
            st = S.to_state(pp, u0_dev)
            fresh = st.clone()
            with S.Handle(pp) as hh:
                timed_run(hh, st, min(steps, 256), fresh)  # warm-up
                t = timed_run(hh, st, steps, fresh)
            compare[f"{name}_{method}"] = {"value": N * steps / t / 1e9, "steps": steps,
                                           "W": W if method == "swept" else None}
            outputs[(name, method, steps)] = S.to_fp64(pp, st)[0].cpu()
            del st, fresh
    # small grid: the launch-latency-bound workload (N = 16384, r = 1/4, 8 modes, 1000 steps, W = 64)
    small = {}
    n_s, steps_s = 16384, 1000
    u_s = torch.as_tensor(I_mod().heat_initial(I_mod().heat_modes(n_s, 8, seed=0)), device=dev)
    # "_graph": the run captured once into a CUDA graph and replayed (SW_FLAG_GRAPH)
    for key, prec, method, W, flags in (("fp64_swept_w64", S.SW_FP64, S.SW_SWEPT, 64, 0),
                                        ("fp64_perstep", S.SW_FP64, S.SW_PERSTEP, 0, 0),
                                        ("fp32_swept_w128", S.SW_FP32, S.SW_SWEPT, 128, 0),
                                        ("fp32_perstep", S.SW_FP32, S.SW_PERSTEP, 0, 0),
                                        ("fp64_swept_w64_graph", S.SW_FP64, S.SW_SWEPT, 64, S.SW_FLAG_GRAPH),
                                        ("fp64_perstep_graph", S.SW_FP64, S.SW_PERSTEP, 0, S.SW_FLAG_GRAPH),
                                        ("fp32_swept_w128_graph", S.SW_FP32, S.SW_SWEPT, 128, S.SW_FLAG_GRAPH),
                                        ("fp32_perstep_graph", S.SW_FP32, S.SW_PERSTEP, 0, S.SW_FLAG_GRAPH)):
        ps = S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=method, n=n_s,
                       r=0.25, tile_width=W, flags=flags)
        st = S.to_state(ps, u_s)
        fresh = st.clone()
        with S.Handle(ps) as hs:
            timed_run(hs, st, steps_s, fresh)
            t = min(timed_run(hs, st, steps_s, fresh) for _ in range(5))
            small[key] = {"ms": t * 1e3, "value": n_s * steps_s / t / 1e9, "launches": hs.sw_last_launch_count()}
    small["speedup_fp64"] = small["fp64_perstep"]["ms"] / small["fp64_swept_w64"]["ms"]
    small["speedup_fp32"] = small["fp32_perstep"]["ms"] / small["fp32_swept_w128"]["ms"]
    small["speedup_fp64_graphs"] = small["fp64_perstep_graph"]["ms"] / small["fp64_swept_w64_graph"]["ms"]
    small["speedup_fp32_graphs"] = small["fp32_perstep_graph"]["ms"] / small["fp32_swept_w128_graph"]["ms"]
    compare["small_grid_n16384_1000_steps"] = small

    # batched: 4096 independent problems (half heat, half Euler, lengths 2^10..2^18), FP32 hi/lo,
    # autotuned widths, one persistent launch from a CUDA graph; a 200-step run
    from paper_1811_08282_gb300 import batched
    items = batched.default_items(4096, seed=7)
    bt = batched.build(items, 200)
    bt.batch.sw_batch_run()
    bt.batch.sw_batch_status()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    bt.batch.sw_batch_run(stream)
    b.record(stream)
    b.synchronize()
    tb = a.elapsed_time(b) / 1e3
    compare["batched_4096"] = {"value": bt.cells * 200 / tb / 1e9, "unit": "Gcell-steps/s", "cells": bt.cells,
                               "steps": 200, "ms": tb * 1e3, "items": bt.batch.sw_batch_items(),
                               "status": bt.batch.sw_batch_status(), "precision": "fp32_comp"}
    bt.batch.close()

    # FP64 conservation sums (fixed-order tree) over the N = 2^24 state: the whole call,
    # two reduction launches and the 8-byte read-back, timed on the stream (L2 flushed)
    pc = problem(S.SW_FP64, S.SW_SWEPT, best_w)
    stc = S.to_state(pc, u0_dev)
    with S.Handle(pc) as hc:
        hc.sw_conservation(stc, stream)
        tcs = []
        for _ in range(5):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            hc.sw_conservation(stc, stream)
            b.record(stream)
            b.synchronize()
            tcs.append(a.elapsed_time(b) / 1e3)
    tc = min(tcs)
    compare["conservation_fp64_n2^24"] = {"us": tc * 1e6, "hbm_gbs": N * 8 / tc / 1e9,
                                          "note": "sw_conservation call incl. read-back of the sum"}
    del stc

    # hybrid CPU/GPU split (Section 4.2, Eq. 1): the host cores take 1 / (1 + WF / threads) of
    # the tiles; short sweep of the work factor, then the best against the GPU alone (same steps)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ph = problem(S.SW_FP64, S.SW_SWEPT, best_w)
    sth = S.to_state(ph, u0_dev)
    hy_steps = 2048
    with S.Handle(ph) as hh:
        def hyb(wf, steps):
            sth.copy_(u0_dev)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hh.sw_run_hybrid(sth, steps, wf, threads, stream)
            return time.perf_counter() - t0
        wf_rates = {}
        for wf in (16, 32, 48, 64, 96, 128, 192, 256):
            try:
                hyb(wf, 64)
                wf_rates[wf] = N * hy_steps / hyb(wf, hy_steps) / 1e9
            except S.SweptError:
                pass
        best_wf = max(wf_rates, key=wf_rates.get)
        t_h = min(hyb(best_wf, 4 * hy_steps) for _ in range(2))
        hyb_state = sth.clone()
        sth.copy_(u0_dev)
        hh.sw_run(sth, 4 * hy_steps, stream)
        torch.cuda.synchronize()
        t_g = timed_run(hh, sth, 4 * hy_steps, u0_dev)
        same = bool(torch.equal(hyb_state, sth))
    gt, per_thread = S.sw_hybrid_split(N // best_w, best_wf, threads)
    compare["hybrid_fp64"] = {"value": N * 4 * hy_steps / t_h / 1e9, "gpu_only": N * 4 * hy_steps / t_g / 1e9,
                              "speedup": t_g / t_h, "steps": 4 * hy_steps, "W": best_w, "threads": threads,
                              "work_factor": best_wf, "gpu_tiles": gt, "host_tiles": per_thread * threads,
                              "wf_sweep": wf_rates, "bitwise_equal_to_gpu_only": same}
    del sth, hyb_state

    perstep_bytes = 16  # FP64 per-step: read + write one value per update
    compare["fp64_perstep"]["hbm_gbs"] = compare["fp64_perstep"]["value"] * perstep_bytes
    compare["speedup_swept_over_perstep_fp64"] = compare["fp64_swept"]["value"] / compare["fp64_perstep"]["value"]
    compare["speedup_swept_over_perstep_fp32"] = compare["fp32_swept"]["value"] / compare["fp32_perstep"]["value"]
    compare["speedup_swept_over_perstep_fp32_comp"] = (compare["fp32_comp_swept"]["value"]
                                                        / compare["fp32_comp_perstep"]["value"])

    # 5) CPU baseline (rank 0 only): the FP64 oracle on the host cores, bounded
    #    sample; also states each result's error against the oracle's closed form.
    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline_leg(modes, r, u0, outputs, compare)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "time_steps": STEPS, "tile_width": best_w,
                   "r": r, "modes": MODES, "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) before every timed step; state reset from a device copy"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "wall_s_timed_region": wall, "tile_sweep_gcups": sweep, "compare": compare,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_leg(modes, r, u0, outputs, compare):
    import numpy as np

    import oracle
    # error of every GPU result against the closed form (sampled cells)
    idx = np.linspace(0, N - 1, 4096).astype(np.int64)
    for (name, method, steps), out in outputs.items():
        want = oracle.heat_modes(N, r, steps, modes.amps, modes.ks, idx)
        got = out.numpy()[idx]
        err = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
        compare.setdefault(f"{name}_{method}", {})["err_vs_oracle"] = err
    # timing: oracle FTCS stepping on the full grid, a bounded number of steps
    t0 = time.perf_counter()
    oracle.heat_run(u0, r, 2)
    per_step = (time.perf_counter() - t0) / 2
    steps = max(2, min(200, int(15.0 / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    oracle.heat_run(u0, r, steps)
    t = time.perf_counter() - t0
    return {"value": N * steps / t / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"N=2^24, first {steps} of {STEPS} steps (naive FP64 stepping, OpenMP over cells)",
            "cpu": _cpu_model()}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle
    modes, r, u0 = initial_state()
    oracle.build()
    t0 = time.perf_counter()
    oracle.heat_run(u0, r, 1)
    per_step = time.perf_counter() - t0
    # each bench step: a bounded sample of the workload (~5 s of CPU work)
    steps = max(1, min(100, int(5.0 / max(per_step, 1e-6))))
    for _ in range(args.warmup):
        oracle.heat_run(u0, r, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.heat_run(u0, r, steps)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = N * steps * args.steps / t / 1e9
    cpu = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"N=2^24, {steps} of {STEPS} steps per bench step (naive FP64 stepping)",
           "cpu": _cpu_model()}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "n": N, "time_steps": STEPS},
        "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                     "d2h_bytes_per_step": 0},
    }))


def run_configs(args):
    """Rates of the paper-shaped workloads besides the headline, each swept and per-step
    at FP64, FP32 and FP32 hi/lo, with the FP32 forms' error against the FP64 result
    (the FP64 path is bitwise equal to the oracle for Euler and within 1e-12 of the
    oracle's closed form for heat; the full-size parity tests check that on these
    workloads, Euler on the window the waves reach or on a shorter run). One untimed
    short run per handle first; single timed run per form (long runs)."""
    import numpy as np
    import torch
    from paper_1811_08282_gb300 import build, batched
    build.build()
    from paper_1811_08282_gb300 import swept as S, inputs as I
    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local_rank)
    precs = {"fp64": S.SW_FP64, "fp32": S.SW_FP32, "fp32_comp": S.SW_FP32_COMP}

    def timed(p, x0, steps, warm=8):
        st = S.to_state(p, torch.as_tensor(x0.reshape(-1), device="cuda"))
        fresh = st.clone()
        with S.Handle(p) as h:
            h.sw_run(st, warm)
            st.copy_(fresh)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            h.sw_run(st, steps)
            b.record()
            b.synchronize()
            rc = h.sw_sync_status()
            launches = h.sw_last_launch_count()
        if rc < 0:
            raise S.SweptError(rc, "configs")
        return a.elapsed_time(b) / 1e3, S.to_fp64(p, st).cpu().numpy().reshape(p.nv, p.n), launches

    def errors(got, ref):
        out = {}
        for v in range(ref.shape[0]):
            d = np.abs(got[v] - ref[v])
            out[f"v{v}"] = {"max_rel": float(d.max() / np.abs(ref[v]).max()),
                            "l2_rel": float(np.linalg.norm(d) / np.linalg.norm(ref[v]))}
        return out

    def best_width(make, x0, steps, widths=(64, 128, 256, 512, 1024)):
        n = x0.shape[-1]
        rates = {}
        for W in widths:
            if n % W or n < 2 * W:
                continue
            t, _, _ = timed(make(W), x0, steps)
            rates[W] = t
        return min(rates, key=rates.get)

    def compare(name, make, x0, steps, tune_steps, extra, flat=False):
        res = {"config": name, "n": x0.shape[-1], "steps": steps, **extra, "forms": {}}
        ref = None
        for pn, pv in precs.items():
            W = best_width(lambda W: make(pv, S.SW_SWEPT, W), x0, tune_steps)
            ts, xs, ls = timed(make(pv, S.SW_SWEPT, W), x0, steps)
            tp, xp, lp = timed(make(pv, S.SW_PERSTEP, 0), x0, steps)
            form = {"W": W, "swept": x0.shape[-1] * steps / ts / 1e9, "perstep": x0.shape[-1] * steps / tp / 1e9,
                    "speedup": tp / ts, "launches_swept": ls, "launches_perstep": lp,
                    "swept_equals_perstep": bool(np.array_equal(xs, xp))}
            if flat:  # Euler: the swept run in the flattened form of Section 4.3 (same bits)
                Wf = best_width(lambda W: make(pv, S.SW_SWEPT, W, S.SW_FLAG_FLATTENED), x0, tune_steps)
                tf, xf, _ = timed(make(pv, S.SW_SWEPT, Wf, S.SW_FLAG_FLATTENED), x0, steps)
                form.update({"W_flattened": Wf, "swept_flattened": x0.shape[-1] * steps / tf / 1e9,
                             "flattened_equals_lengthened": bool(np.array_equal(xf, xs))})
            if pn == "fp64":
                ref = xs
            else:
                form["err_vs_fp64"] = errors(xs, ref)
            res["forms"][pn] = form
            print(f"# {name} {pn} done", file=sys.stderr, flush=True)
        res["unit"] = "Gcell-steps/s"
        print(json.dumps(res), flush=True)

    # small grid: heat N = 16384, r = 0.25, 8 modes, seeds 0-4, 1000 steps, W = 64 vs per-step
    n, steps = 16384, 1000
    rows = []
    for seed in range(5):
        x0 = I.heat_initial(I.heat_modes(n, 8, seed=seed))[None]
        row = {}
        for pn in ("fp64", "fp32"):
            mk = lambda m, W: S.Problem(scheme=S.SW_HEAT, precision=precs[pn], boundary=S.SW_PERIODIC, method=m,
                                        n=n, r=0.25, tile_width=W)
            ts, xs, _ = timed(mk(S.SW_SWEPT, 64), x0, steps)
            tp, xp, _ = timed(mk(S.SW_PERSTEP, 0), x0, steps)
            row[pn] = {"swept_ms": ts * 1e3, "perstep_ms": tp * 1e3, "speedup": tp / ts,
                       "swept_equals_perstep": bool(np.array_equal(xs, xp))}
        rows.append(row)
    print(json.dumps({"config": "heat N=16384 r=0.25 8 modes seeds 0-4, 1000 steps, W=64", "seeds": rows,
                      "mean_speedup_fp64": statistics.mean(r["fp64"]["speedup"] for r in rows),
                      "mean_speedup_fp32": statistics.mean(r["fp32"]["speedup"] for r in rows)}), flush=True)

    # Euler Sod, N = 2^20, 20,000 steps, transmissive
    def euler(lam):
        return lambda pv, m, W, flags=0: S.Problem(
            scheme=S.SW_EULER, precision=pv, boundary=S.SW_TRANSMISSIVE, method=m,
            n=1 << 20 if lam == "sod" else 1 << 22, dt_dx=I.sod_lambda() if lam == "sod" else I.riemann_lambda(),
            gamma=I.GAMMA, tile_width=W, flags=flags)
    compare("Euler Sod N=2^20, 20000 steps, transmissive", euler("sod"), I.sod(1 << 20), 20_000, 512,
            {"dt_dx": I.sod_lambda()}, flat=True)

    # precision config: heat N = 2^22, r = 0.4, 100,000 steps; Euler N = 2^22, 64 random Riemann segments
    n = 1 << 22
    heat = lambda pv, m, W: S.Problem(scheme=S.SW_HEAT, precision=pv, boundary=S.SW_PERIODIC, method=m, n=n,
                                      r=0.4, tile_width=W)
    compare("heat N=2^22 r=0.4, 100000 steps, 32 modes", heat, I.heat_initial(I.heat_modes(n, 32, seed=1))[None],
            100_000, 4096, {"r": 0.4})
    compare("Euler N=2^22, 64 random Riemann segments, 20000 steps, transmissive", euler("riemann"),
            I.riemann_initial(I.riemann_segments(n, 64, 1)), 20_000, 512, {"dt_dx": I.riemann_lambda()}, flat=True)

    # batched: 4096 problems, FP32 hi/lo, tuned widths, 10,000 steps in one persistent launch
    items = batched.default_items(4096, seed=7)
    t0 = time.perf_counter()
    widths = batched.tune_widths(items)
    tune_s = time.perf_counter() - t0
    bt = batched.build(items, 10_000, widths=widths)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    bt.batch.sw_batch_run()
    b.record()
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    print(json.dumps({"config": "batched 4096 problems, lengths log-uniform 2^10..2^18, half heat / half Euler, "
                      "FP32 hi/lo, 10000 steps", "cells": bt.cells, "widths": widths, "tune_s": tune_s,
                      "seconds": t, "value": bt.cells * 10_000 / t / 1e9, "unit": "Gcell-steps/s",
                      "items": bt.batch.sw_batch_items(), "status": bt.batch.sw_batch_status()}), flush=True)
    bt.batch.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.configs:
        run_configs(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
