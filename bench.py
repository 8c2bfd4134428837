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
    "k2d": ("common.cuh", "heat.cuh", "fp64_soft.cuh", "fp64_soft2d.cuh", "heat2d.cu"),
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
    # pipes: its ceiling is the busier of the FP64 and ALU pipes for its instruction mix.
    # `peak` takes the pipes' nominal issue rates (ncu's "% busy" is relative to them); the
    # rates measured now by the chain probes (paper_1811_08282_gb300/peaks.py) give a second
    # ceiling beside it, and the algorithmic best split a third.
    try:
        from paper_1811_08282_gb300 import peaks
        pipes = peaks.measure()
    except Exception:
        pipes = None
    fp64_rate = pipes["fp64_fma"] if pipes else FP64_INST_PER_S
    alu_rate = pipes["int_alu"] if pipes else ALU_LANE_INST_PER_S
    peak, peak_source = FP64_PEAK_TFLOPS, \
        "FP64 1.25 TFLOP/s class: 152 SM x 2 DFMA/clk x 2 x 2.07 GHz (nominal, recipe)"
    fp64_ipu = recorded(kname, f"{kname}.heat_fp64.w{best_w}", "fp64_inst_per_update") if fold else None
    alu_ipu = recorded(kname, f"{kname}.heat_fp64.w{best_w}", "alu_inst_per_update") if fold else None
    best_split = peak_measured = None
    if fp64_ipu and alu_ipu:
        ceiling = min(FP64_INST_PER_S / fp64_ipu, ALU_LANE_INST_PER_S / alu_ipu)  # updates/s
        peak = ceiling * FLOPS_PER_UPDATE / 1e12
        peak_source = (f"pipe ceiling of the FP64 + integer-pipe kernel, in FP64-equivalent flops (5 per update): "
                       f"min(FP64 pipe 152 SM x 2/clk x 2.07 GHz / {fp64_ipu:.3f} FP64 instr per update, "
                       f"ALU pipe 152 SM x 64 lanes/clk x 2.07 GHz / {alu_ipu:.2f} ALU instr per update) "
                       f"= {ceiling / 1e9:.1f} G updates/s (nominal issue rates; instruction counts: ncu, "
                       f"profiles/traffic.txt)")
        if pipes:
            peak_measured = min(pipes["fp64_fma"] / fp64_ipu, pipes["int_alu"] / alu_ipu) * FLOPS_PER_UPDATE / 1e12
        # algorithmic best split: every FP64-pipe update at its 3 instructions plus every
        # integer-path update at its cost (2 x the per-update average at the half split), both
        # pipes busy all the time, at the nominal rates
        best_split = (FP64_INST_PER_S / 3 + ALU_LANE_INST_PER_S / (2 * alu_ipu)) * FLOPS_PER_UPDATE / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "fp64_pipe_peak": FP64_PEAK_TFLOPS,
                "frac_of_fp64_pipe_peak": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "pipe_rates_measured": {k: v / 1e9 for k, v in pipes.items()} if pipes else None,
                "pipe_rates_unit": "G thread operations/s",
                "peak_at_measured_rates": peak_measured,
                "frac_at_measured_rates": (achieved / peak_measured) if (achieved and peak_measured) else None,
                "best_split_peak": best_split,
                "frac_of_best_split": (achieved / best_split) if (achieved and best_split) else None,
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

    # 4) comparisons (one rank only: the replicas of a multi-GPU run time the headline alone):
    #    on the same grid, the per-step kernel and the FP32 forms, every form run for the same
    #    number of steps so that the errors compare like for like; then the other configured
    #    workloads
    compare = {}
    if world == 1:
        compare_legs(args, S, problem, timed_run, u0_dev, best_w, value, final, flush, stream, dev, compare,
                     modes, r, u0, fp64_rate, alu_rate)
    cpu = compare.pop("_cpu_baseline", None)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "time_steps": STEPS, "tile_width": best_w,
                   "r": r, "modes": MODES, "parallelism": f"replicas x{world}",
                   "l2": "flushed (256 MB write) before every timed step; state reset from a device copy"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks, "wall_s_timed_region": wall, "tile_sweep_gcups": sweep, "compare": compare or None,
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def compare_legs(args, S, problem, timed_run, u0_dev, best_w, value, final, flush, stream, dev, compare,
                 modes, r, u0, fp64_rate, alu_rate):
    """Every comparison of the JSON line besides the headline (single-GPU runs)."""
    import torch
    world = 1
    outputs = {("fp64", "swept", STEPS): final.cpu()}
    for name, prec in (("fp64", S.SW_FP64), ("fp32", S.SW_FP32), ("fp32_comp", S.SW_FP32_COMP)):
        if name == "fp64":
            w_prec = best_w
        else:  # the same short timed sweep as for FP64
            w_prec = tune_heat_width(S, problem, prec, u0_dev, timed_run, WIDTHS[2:], TUNE_STEPS)
        for method in ("swept", "perstep"):
            if name == "fp64" and method == "swept":
                compare["fp64_swept"] = {"value": value / world, "steps": STEPS, "W": best_w}
                continue
            pp = problem(prec, S.SW_SWEPT if method == "swept" else S.SW_PERSTEP, w_prec)
            st = S.to_state(pp, u0_dev)
            fresh = st.clone()
            with S.Handle(pp) as hh:
                timed_run(hh, st, 256, fresh)  # warm-up
                t = timed_run(hh, st, STEPS, fresh)
            compare[f"{name}_{method}"] = {"value": N * STEPS / t / 1e9, "steps": STEPS,
                                           "W": w_prec if method == "swept" else None}
            outputs[(name, method, STEPS)] = S.to_fp64(pp, st)[0].cpu()
            del st, fresh

    # the oracle's share of the configured workloads below, computed from the seeded
    # inputs alone in spawned processes while the GPU legs run (joined before any leg
    # that uses the host cores)
    side = OracleSide(True)

    # heat precision workload: N = 2^22, r = 0.4, 100,000 steps, three precisions
    compare["heat_precision_n2^22"] = heat_precision_leg(S, timed_run)
    # Euler workloads: Sod N = 2^20, 20,000 steps; 64 random Riemann segments, N = 2^22
    sod_out = euler_leg(S, timed_run, "sod")
    rie_out = euler_leg(S, timed_run, "riemann")
    # the swept rule in two dimensions (heat, 8192 x 8192)
    compare["heat2d_8192^2"] = heat2d_leg(S, flush, stream, fp64_rate, alu_rate)
    # batched: 4096 problems at the configured 10,000 steps
    batch_leg, batch_out = batched_leg(S, stream)
    compare["batched_4096"] = batch_leg

    side.join()  # the host cores are needed by the legs below
    finish_euler_leg(compare, "euler_sod_n2^20", sod_out, side.result("sod"))
    finish_euler_leg(compare, "euler_riemann_n2^22", rie_out, side.result("riemann"))
    finish_batched_leg(compare["batched_4096"], batch_out, side.result("batch"))

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

    # 5) CPU baseline: the FP64 oracle on the host cores, bounded sample; also states each
    #    result's error against the oracle's closed form.
    compare["_cpu_baseline"] = cpu_baseline_leg(modes, r, u0, outputs, compare)


# ------------------------------------------------------------------ configured workloads
HEAT4_N, HEAT4_STEPS, HEAT4_R, HEAT4_SEED = 1 << 22, 100_000, 0.4, 4
SOD_N, SOD_STEPS = 1 << 20, 20_000
RIE_N, RIE_SEGS, RIE_SEED, RIE_STEPS = 1 << 22, 64, 4, 4_000
RIE_WINDOWS, RIE_WINDOW_CELLS = 4, 2048
BATCH_COUNT, BATCH_SEED, BATCH_STEPS = 4096, 7, 10_000
BATCH_SUBSET, BATCH_SUBSET_MAX_N = 16, 1536  # per scheme: the first items of at most this length
EULER_WIDTHS = (256, 512, 1024)
PREC_NAMES = ("fp64", "fp32", "fp32_comp")


def tune_heat_width(S, problem, prec, x_dev, timed_run, widths, steps):
    """Fastest W on a short timed run of the real initial state (Section 6's advice)."""
    rates = {}
    for W in widths:
        pw = problem(prec, S.SW_SWEPT, W)
        st = S.to_state(pw, x_dev)
        fresh = st.clone()
        with S.Handle(pw) as hw:
            timed_run(hw, st, 64, fresh)
            rates[W] = steps / timed_run(hw, st, steps, fresh)
        del st, fresh
    return max(rates, key=rates.get)


def norm_errors(got, ref, names):
    """Norm-relative max and L2 error per variable (max|g - o| / max|o|, ||g - o|| / ||o||)."""
    import numpy as np
    out = {}
    for v, nm in enumerate(names):
        d = np.abs(got[v] - ref[v])
        out[nm] = {"max_rel": float(d.max() / max(np.abs(ref[v]).max(), 1e-300)),
                   "l2_rel": float(np.linalg.norm(d) / max(np.linalg.norm(ref[v]), 1e-300))}
    return out


def euler_quality(q, gamma=1.4):
    """Positivity and monotonicity of an Euler state (3, n): the smallest density and
    pressure, the total variation of both, and the number of local extrema of density
    whose two sides both exceed 1e-5 of its range (oscillations above rounding level)."""
    import numpy as np
    rho, m, E = q
    p = (gamma - 1.0) * (E - 0.5 * m * (m / rho))
    drho = np.diff(rho)
    tol = 1e-5 * max(float(rho.max() - rho.min()), 1e-300)
    a, b = drho[:-1], drho[1:]
    ext = int(np.count_nonzero((a * b < 0) & (np.minimum(np.abs(a), np.abs(b)) > tol)))
    return {"min_rho": float(rho.min()), "min_p": float(p.min()), "tv_rho": float(np.abs(drho).sum()),
            "tv_p": float(np.abs(np.diff(p)).sum()), "extrema_rho": ext,
            "finite": bool(np.isfinite(q).all())}


def heat_precision_leg(S, timed_run):
    """Heat, N = 2^22, r = 0.4, 100,000 steps (32 modes): swept and per-step in FP64, FP32
    and FP32 hi/lo, each with its error against the oracle's closed form (sampled cells)."""
    import numpy as np
    import torch

    import oracle
    from paper_1811_08282_gb300 import inputs as I
    n, steps = HEAT4_N, HEAT4_STEPS
    modes = I.heat_modes(n, 32, seed=HEAT4_SEED)
    x = torch.as_tensor(I.heat_initial(modes), device="cuda")
    idx = np.linspace(0, n - 1, 8192).astype(np.int64)
    want = oracle.heat_modes(n, HEAT4_R, steps, modes.amps, modes.ks, idx)

    def problem(prec, method, W):
        return S.Problem(scheme=S.SW_HEAT, precision=prec, boundary=S.SW_PERIODIC, method=method, n=n,
                         r=HEAT4_R, tile_width=W if method == S.SW_SWEPT else 0)
    res = {"n": n, "steps": steps, "r": HEAT4_R, "modes": 32, "unit": "Gcell-updates/s",
           "error": "norm-relative max over 8192 sampled cells vs the oracle's exact discrete solution"}
    for pn, prec in zip(PREC_NAMES, (S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP)):
        W = tune_heat_width(S, problem, prec, x, timed_run, (128, 256, 512, 1024), 2048)
        form = {"W": W}
        for method in ("swept", "perstep"):
            p = problem(prec, S.SW_SWEPT if method == "swept" else S.SW_PERSTEP, W)
            st = S.to_state(p, x)
            fresh = st.clone()
            with S.Handle(p) as h:
                timed_run(h, st, 256, fresh)
                t = timed_run(h, st, steps, fresh)
            got = S.to_fp64(p, st)[0].cpu().numpy()[idx]
            form[method] = n * steps / t / 1e9
            form[f"err_vs_oracle_{method}"] = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
            del st, fresh
        form["speedup"] = form["swept"] / form["perstep"]
        res[pn] = form
    return res


H2D_N, H2D_STEPS, H2D_R, H2D_SEED = 8192, 2048, 0.2, 6
H2D_FLOPS_PER_UPDATE = 10  # a + b, d + e, fma(-2, u, .) x 2, fma(ry, ., u), fma(rx, ., .)


def pipe_ceiling2d(key, fp64_rate, alu_rate):
    """Updates/s ceiling of an FP64 2D kernel that runs part of its cells on the integer
    pipes: the busier of the FP64 and ALU pipes at their measured rates for the kernel's
    instruction mix (ncu counts in profiles/traffic.txt), with the counts used; None when
    the kernel changed since they were taken."""
    f = recorded("k2d", key, "fp64_inst_per_update")
    a = recorded("k2d", key, "alu_inst_per_update")
    if not (f and a):
        return None, None, None
    return min(fp64_rate / f, alu_rate / a), f, a


def heat2d_leg(S, flush, stream, fp64_rate, alu_rate):
    """Heat in two dimensions (the 5-point extension of Section 6's future work): periodic
    8192 x 8192, rx = ry = 0.2, 16 separable modes, 2048 steps; per precision the swept run
    (W tuned on short runs) against the per-step kernel, the error against the oracle's
    exact mode solution at sampled cells (relative to the initial maximum), and for FP64 the
    roofline of one swept phase (a bridges and an octahedra launch) from traced launches."""
    import numpy as np
    import torch

    import oracle
    from paper_1811_08282_gb300 import inputs as I
    n, steps = H2D_N, H2D_STEPS
    m = I.heat2d_modes(n, n, 16, seed=H2D_SEED, kmax=16)
    u0 = I.heat2d_initial(m)
    rng = np.random.default_rng(1)
    ii, jj = rng.integers(0, n, 4096), rng.integers(0, n, 4096)
    want = oracle.heat2d_modes(n, n, H2D_R, H2D_R, steps, m.amps, m.kx, m.ky, m.fx, m.fy, ii, jj)
    umax = float(np.abs(u0).max())
    x64 = torch.as_tensor(u0.reshape(-1), device="cuda")

    def run(p, nsteps, trace=0):
        st = x64.to(torch.float64 if p.precision == S.SW_FP64 else torch.float32).clone()
        fresh = st.clone()
        with S.Handle2D(p) as h:
            h.sw2d_run(st, min(nsteps, 64))
            st.copy_(fresh)
            if trace:
                h.sw2d_set_timing(trace)
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.sw2d_run(st, nsteps, stream)
            b.record(stream)
            b.synchronize()
            launches = h.sw2d_last_launch_count()
            traced = h.sw2d_launch_times() if trace else []
        return a.elapsed_time(b) / 1e3, st, launches, traced

    res = {"workload": f"heat 2D FTCS periodic {n}x{n}, rx=ry={H2D_R}, 16 modes, {steps} steps", "unit":
           "Gcell-updates/s", "error": "max |got - exact| / max |initial| over 4096 sampled cells"}
    for pn, prec, widths in (("fp64", S.SW_FP64, (32, 64)), ("fp32", S.SW_FP32, (32, 64, 128))):
        rates = {W: 128 / run(S.Heat2D(precision=prec, method=S.SW_SWEPT, tile_width=W, nx=n, ny=n, rx=H2D_R,
                                       ry=H2D_R), 128)[0] for W in widths}
        W = max(rates, key=rates.get)
        ps = S.Heat2D(precision=prec, method=S.SW_SWEPT, tile_width=W, nx=n, ny=n, rx=H2D_R, ry=H2D_R)
        ts, st, ls, traced = run(ps, steps, trace=2 * steps // (W // 2) + W)
        got = st.double().cpu().numpy().reshape(n, n)[jj, ii]
        tp, stp, lp, _ = run(S.Heat2D(precision=prec, method=S.SW_PERSTEP, nx=n, ny=n, rx=H2D_R, ry=H2D_R), steps)
        form = {"W": W, "swept": n * n * steps / ts / 1e9, "perstep": n * n * steps / tp / 1e9, "speedup": tp / ts,
                "launches_swept": ls, "launches_perstep": lp, "swept_equals_perstep": bool(torch.equal(st, stp)),
                "err_vs_oracle": float(np.abs(got - want).max() / umax),
                "tile_sweep": {str(k): n * n * 128 / (128 / v) / 1e9 for k, v in rates.items()}}
        # one swept phase: a bridges launch (kind 1) and an octahedra launch (kind 2)
        br = [ms for ms, k in traced if k == 1]
        oc = [ms for ms, k in traced if k == 2]
        if br and oc:
            phase_s = (statistics.mean(br) + statistics.mean(oc)) / 1e3
            updates = n * n * (W // 2)
            form["phase_ms"] = phase_s * 1e3
            form["octahedra_share_of_phase"] = statistics.mean(oc) / (statistics.mean(br) + statistics.mean(oc))
            if prec == S.SW_FP64:
                achieved = updates * H2D_FLOPS_PER_UPDATE / phase_s / 1e12
                ceil, fi, ai = pipe_ceiling2d(f"k2d.phase_fp64.w{W}", fp64_rate, alu_rate)
                bpu = recorded("k2d", f"k2d.phase_fp64.w{W}", "bytes_per_update")
                peak = ceil * H2D_FLOPS_PER_UPDATE / 1e12 if ceil else None
                res["roofline"] = {
                    "bound": "fp64+alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": (achieved / peak) if peak else None,
                    "traffic": bpu * updates if bpu else None,
                    "kernel": f"k2d_bridges<double> + k2d_octa<double> (one swept phase, W = {W})",
                    "flops_per_update": H2D_FLOPS_PER_UPDATE,
                    "fp64_pipe_nominal": FP64_PEAK_TFLOPS,
                    "peak_source": (f"half the cells on the integer pipes: min(FP64 pipe {fp64_rate / 1e9:.0f} G/s / "
                                    f"{fi} FP64 instr per update, ALU pipe {alu_rate / 1e12:.1f} T/s / {ai} ALU instr "
                                    f"per update), measured rates (chain probes), ncu counts of the phase "
                                    f"(profiles/traffic.txt), in flops at 10 per update") if peak else
                                   "instruction counts not current for this kernel"}
        if prec == S.SW_FP64:
            ceil, fi, ai = pipe_ceiling2d("k2d.step_fp64", fp64_rate, alu_rate)
            if ceil:
                form["perstep_ceiling_gups"] = ceil / 1e9
                form["perstep_frac_of_ceiling"] = form["perstep"] / (ceil / 1e9)
        res[pn] = form
    return res


def _euler_case(kind):
    from paper_1811_08282_gb300 import inputs as I
    if kind == "sod":
        return dict(n=SOD_N, steps=SOD_STEPS, q0=I.sod(SOD_N), lam=I.sod_lambda(), periodic=False,
                    workload="Euler Sod N=2^20, 20000 steps, transmissive, CFL 0.4")
    n = RIE_N
    return dict(n=n, steps=RIE_STEPS, q0=I.riemann_initial(I.riemann_segments(n, RIE_SEGS, RIE_SEED)),
                lam=I.riemann_lambda(), periodic=True,
                workload=f"Euler N=2^22, {RIE_SEGS} random Riemann segments (rho, p log-U[0.1,1], u U[-0.5,0.5]), "
                         f"{RIE_STEPS} steps, periodic, CFL 0.4")


def euler_leg(S, timed_run, kind):
    """One Euler workload: per precision, swept (default form, W tuned on short runs of the
    real state) against per-step, the same steps; returns rates and the final states."""
    import numpy as np
    import torch
    from paper_1811_08282_gb300 import inputs as I
    c = _euler_case(kind)
    n, steps = c["n"], c["steps"]
    x = torch.as_tensor(c["q0"].reshape(-1), device="cuda")
    bc = S.SW_PERIODIC if c["periodic"] else S.SW_TRANSMISSIVE

    def problem(prec, method, W, flags=0):
        return S.Problem(scheme=S.SW_EULER, precision=prec, boundary=bc, method=method, n=n, dt_dx=c["lam"],
                         gamma=I.GAMMA, tile_width=W if method == S.SW_SWEPT else 0, flags=flags)

    def run(p, nsteps, warm=8):
        st = S.to_state(p, x)
        fresh = st.clone()
        with S.Handle(p) as h:
            timed_run(h, st, warm, fresh)
            t = timed_run(h, st, nsteps, fresh)
            rc = h.sw_sync_status()
            launches = h.sw_last_launch_count()
        if rc < 0:
            raise S.SweptError(rc, f"euler {kind}")
        return t, S.to_fp64(p, st).cpu().numpy().reshape(3, n), launches

    out = {"case": c, "forms": {}, "states": {}}
    for pn, prec in zip(PREC_NAMES, (S.SW_FP64, S.SW_FP32, S.SW_FP32_COMP)):
        probe = max(16, min(256, int(2e9 / n / (40 if prec == S.SW_FP64 else 1))))  # ~0.1 s per probe run
        rates = {W: probe / run(problem(prec, S.SW_SWEPT, W), probe, warm=4)[0] for W in EULER_WIDTHS}
        W = max(rates, key=rates.get)
        ts, xs, ls = run(problem(prec, S.SW_SWEPT, W), steps)
        tp, xp, lp = run(problem(prec, S.SW_PERSTEP, 0), steps)
        form = {"W": W, "form": "flattened" if W % 4 == 0 else "lengthened",
                "swept": n * steps / ts / 1e9, "perstep": n * steps / tp / 1e9, "speedup": tp / ts,
                "launches_swept": ls, "launches_perstep": lp, "swept_equals_perstep": bool(np.array_equal(xs, xp))}
        if prec != S.SW_FP64:
            # the lengthened swept form at the same width, for the Section 4.3 comparison (same bits)
            tl, xl, _ = run(problem(prec, S.SW_SWEPT, W, S.SW_FLAG_LENGTHENED), steps)
            form["swept_lengthened"] = n * steps / tl / 1e9
            form["lengthened_equals_flattened"] = bool(np.array_equal(xl, xs))
        out["forms"][pn] = form
        out["states"][pn] = xs
        print(f"# euler {kind} {pn} done", file=sys.stderr, flush=True)
    return out


def finish_euler_leg(compare, key, out, oracle_res):
    """Errors against the oracle, positivity / monotonicity, and the FP64 parity flags."""
    import numpy as np
    c = out["case"]
    n, steps = c["n"], c["steps"]
    names = ("rho", "m", "E")
    res = {"workload": c["workload"], "n": n, "steps": steps, "dt_dx": c["lam"], "unit": "Gcell-steps/s",
           "error": "norm-relative max / L2 per variable"}
    f64 = out["states"]["fp64"]
    if not c["periodic"]:
        # Sod: the oracle on the interface's numerical domain of dependence (4 cells per step
        # each side; constant beyond it), embedded in the untouched far field: the full field
        lo, hi = oracle_res["lo"], oracle_res["hi"]
        ref = c["q0"].copy()
        ref[:, lo:hi] = oracle_res["q"]
        res["oracle_cells"] = [int(lo), int(hi)]
        res["fp64_equals_oracle"] = bool(np.array_equal(f64, ref))
        q_ref = euler_quality(ref)
    else:
        # random Riemann problems: the oracle on sampled windows (each run on its window plus
        # its domain of dependence); the FP32 forms' full-field error is against the FP64 run
        wins = oracle_res["windows"]
        res["oracle_windows"] = [[int(a), int(b)] for a, b, _ in wins]
        res["fp64_equals_oracle"] = all(np.array_equal(f64[:, a:b], q) for a, b, q in wins)
        ref = f64
        q_ref = euler_quality(ref)
    res["quality_fp64"] = q_ref
    for pn, form in out["forms"].items():
        got = out["states"][pn]
        if pn != "fp64":
            form["err_vs_oracle" if not c["periodic"] else "err_vs_fp64"] = norm_errors(got, ref, names)
            if c["periodic"]:
                g = np.concatenate([got[:, a:b] for a, b, _ in oracle_res["windows"]], axis=1)
                o = np.concatenate([q for _, _, q in oracle_res["windows"]], axis=1)
                form["err_vs_oracle_windows"] = norm_errors(g, o, names)
            q = euler_quality(got)
            form["quality"] = q
            form["positive"] = bool(q["finite"] and q["min_rho"] > 0 and q["min_p"] > 0)
            form["tv_rho_ratio"] = q["tv_rho"] / q_ref["tv_rho"]
            form["tv_p_ratio"] = q["tv_p"] / q_ref["tv_p"]
            form["extrema_rho_vs_fp64"] = [q["extrema_rho"], q_ref["extrema_rho"]]
        else:
            form["err_vs_oracle"] = "bitwise equal" if res["fp64_equals_oracle"] else "DIFFERS"
        res[pn] = form
    compare[key] = res


def batched_leg(S, stream):
    """4096 problems, half heat / half Euler, FP32 hi/lo, lengths log-uniform 2^10..2^18, the
    configured 10,000 steps in one persistent graph-launched kernel. Widths (and the Euler
    form) from the tuner: one cap per scheme and one per size class (octave of length), each
    timed on the batch kernel, the faster table on a 1000-step run of the whole batch kept."""
    import torch
    from paper_1811_08282_gb300 import batched
    items = batched.default_items(BATCH_COUNT, seed=BATCH_SEED)
    t0 = time.perf_counter()
    widths, threads, tune_report = batched.tune(items)
    tune_s = time.perf_counter() - t0
    bt = batched.build(items, BATCH_STEPS, widths=widths, threads=threads)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    bt.batch.sw_batch_run(stream)
    b.record(stream)
    b.synchronize()
    t = a.elapsed_time(b) / 1e3
    status = bt.batch.sw_batch_status(stream)
    subset = batch_subset()
    finals = {i: (items[i].scheme, S.to_fp64(bt.problems[i], bt.states[i]).cpu().numpy().reshape(bt.problems[i].nv, -1))
              for i in subset}
    leg = {"value": bt.cells * BATCH_STEPS / t / 1e9, "unit": "Gcell-steps/s", "cells": bt.cells,
           "problems": len(items), "steps": BATCH_STEPS, "seconds": t, "items": bt.batch.sw_batch_items(),
           "status": status, "precision": "fp32_comp", "tune_s": tune_s, "tuner": tune_report}
    bt.batch.close()
    return leg, finals


def batch_subset():
    """The seeded subset the oracle checks: the first BATCH_SUBSET heat (even index) and Euler
    (odd index) problems of at most BATCH_SUBSET_MAX_N cells, in the batch's own order."""
    from paper_1811_08282_gb300 import inputs as I
    ns = I.batch_lengths(BATCH_COUNT, BATCH_SEED)
    out = []
    for parity in (0, 1):
        out += [i for i in range(parity, BATCH_COUNT, 2) if ns[i] <= BATCH_SUBSET_MAX_N][:BATCH_SUBSET]
    return out


def finish_batched_leg(leg, finals, oracle_res):
    """Each subset problem's error against the oracle: heat relative to the initial state's
    largest magnitude (10,000 steps decay the short problems' modes by up to ~1e-8, so the
    final state's own size says nothing about rounding); Euler norm-relative max and L2 per
    variable (the worst variable)."""
    import numpy as np
    from paper_1811_08282_gb300 import inputs as I
    idx = sorted(finals)
    init = {i: it.planes for i, it in zip(idx, I.batch_problems(BATCH_COUNT, BATCH_SEED, indices=idx))}
    errs = {"heat": [], "euler": []}
    l2s = []
    for i, (scheme, got) in finals.items():
        want = oracle_res[i]
        if scheme == "heat":
            errs[scheme].append(float(np.abs(got - want).max() / np.abs(init[i]).max()))
        else:
            errs[scheme].append(float((np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)).max()))
            l2s.append(float((np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)).max()))
    leg["subset_vs_oracle"] = {
        "heat": {"problems": len(errs["heat"]), "max_abs_over_initial_max": max(errs["heat"]),
                 "median": float(np.median(errs["heat"]))},
        "euler": {"problems": len(errs["euler"]), "max_rel_max": max(errs["euler"]),
                  "max_rel_median": float(np.median(errs["euler"])), "l2_rel_max": max(l2s),
                  "l2_rel_median": float(np.median(l2s))}}
    leg["subset_rule"] = (f"first {BATCH_SUBSET} heat and {BATCH_SUBSET} Euler problems of at most "
                          f"{BATCH_SUBSET_MAX_N} cells in batch order, 10,000 steps, against the oracle")


# ------------------------------------------------------------------ oracle side jobs
def _oracle_sod(threads):
    import numpy as np

    import oracle
    oracle.set_threads(threads)
    c = _euler_case("sod")
    reach = 4 * c["steps"] + 2
    mid = c["n"] // 2
    lo, hi = mid - reach - 8, mid + reach + 8
    q = oracle.euler_run(np.ascontiguousarray(c["q0"][:, lo:hi]), c["lam"], 1.4, c["steps"], oracle.TRANSMISSIVE)
    return {"lo": lo, "hi": hi, "q": q}


def _oracle_riemann(threads):
    import numpy as np

    import oracle
    from paper_1811_08282_gb300 import inputs as I
    oracle.set_threads(threads)
    c = _euler_case("riemann")
    n, steps = c["n"], c["steps"]
    reach = 4 * steps + 8
    # windows centred on seeded segment interfaces, where the waves are
    seg = n // RIE_SEGS
    ifaces = I.randint(99, RIE_WINDOWS, 1, RIE_SEGS - 1, stream=5)
    starts = ifaces * seg - RIE_WINDOW_CELLS // 2
    wins = []
    for a in starts:
        a = int(a)
        b = a + RIE_WINDOW_CELLS
        sub = np.ascontiguousarray(np.take(c["q0"], np.arange(a - reach, b + reach), axis=1, mode="wrap"))
        q = oracle.euler_run(sub, c["lam"], 1.4, steps, oracle.TRANSMISSIVE)
        wins.append((a, b, q[:, reach:reach + RIE_WINDOW_CELLS].copy()))
    return {"windows": wins}


def _oracle_batch(indices):
    import oracle
    from paper_1811_08282_gb300 import inputs as I
    oracle.set_threads(1)
    out = {}
    for i, it in zip(indices, I.batch_problems(BATCH_COUNT, BATCH_SEED, indices=indices)):
        if it.scheme == "heat":
            out[i] = oracle.heat_run(it.planes[0], it.r, BATCH_STEPS, oracle.PERIODIC)[None]
        else:
            out[i] = oracle.euler_run(it.planes, I.riemann_lambda(), I.GAMMA, BATCH_STEPS, oracle.TRANSMISSIVE)
    return out


class OracleSide:
    """The oracle results the configured workloads need, computed from the seeded inputs in
    spawned worker processes (no CUDA there) while the GPU legs run; `join` waits for all."""

    def __init__(self, enabled: bool):
        self.futs = {}
        self.res = {}
        self.ex = None
        if not enabled:
            return
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        self.ex = ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn"))
        subset = batch_subset()
        half = len(subset) // 2
        # leave two host cores to the process driving the GPU
        self.futs["sod"] = [self.ex.submit(_oracle_sod, max(1, ncpu - 6))]
        self.futs["riemann"] = [self.ex.submit(_oracle_riemann, 2)]
        self.futs["batch"] = [self.ex.submit(_oracle_batch, subset[:half]), self.ex.submit(_oracle_batch, subset[half:])]

    def join(self):
        if not self.ex:
            return
        for k, fs in self.futs.items():
            parts = [f.result() for f in fs]
            if k == "batch":
                merged = {}
                for part in parts:
                    merged.update(part)
                self.res[k] = merged
            else:
                self.res[k] = parts[0]
        self.ex.shutdown()
        self.ex = None

    def result(self, key):
        return self.res.get(key)


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
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    oracle.heat_run(u0, r, 2)
    per_step = (time.perf_counter() - t0) / 2
    steps = max(2, min(200, int(15.0 / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    oracle.heat_run(u0, r, steps)
    t = time.perf_counter() - t0
    # the same on one core (a shorter sample)
    oracle.set_threads(1)
    t1 = time.perf_counter()
    oracle.heat_run(u0, r, 2)
    per_step1 = (time.perf_counter() - t1) / 2
    steps1 = max(2, min(50, int(5.0 / max(per_step1, 1e-6))))
    t1 = time.perf_counter()
    oracle.heat_run(u0, r, steps1)
    t1 = time.perf_counter() - t1
    oracle.set_threads(cores)
    return {"value": N * steps / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"N=2^24, first {steps} of {STEPS} steps (naive FP64 stepping, OpenMP over cells)",
            "value_1core": N * steps1 / t1 / 1e9,
            "sample_1core": f"N=2^24, first {steps1} of {STEPS} steps on one thread",
            "cpu": _cpu_model()}


ARM_PARTS = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd49": "Arm Neoverse-N2",
             "0xd0c": "Arm Neoverse-N1", "0xd8f": "Arm Neoverse-V3"}


def _cpu_model():
    """The host CPU's model name (lscpu's "Model name"; on Arm hosts /proc/cpuinfo gives only
    the part id, named here for the Neoverse cores)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                v = line.split(":", 1)[1].strip()
                return f"{ARM_PARTS[v]} (part {v})" if v in ARM_PARTS else v
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


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
