"""Build an autotuned batch of independent problems (one persistent launch per run).

    from paper_1811_08282_gb300 import batched
    bt = batched.build(batched.default_items(4096, seed=7), nsteps=10_000)
    bt.batch.sw_batch_run(); bt.batch.sw_batch_status()

Tile widths are tuned by timing the batch kernel itself on short runs (Section 6's
advice: tune on a few short runs), either as one cap per scheme (`tune_widths`) or
per size class, one octave of problem length per class (`tune_classes`), and then
fitted to each problem's length (largest width <= the cap that divides it and
leaves at least two tiles). For Euler the tuner also picks the staging form of
Section 4.3, lengthened or flattened (same results). `tune` runs both and keeps
the one that times faster on a short run of the whole batch. Heat problems are
periodic, Euler problems transmissive Riemann problems.
"""
from __future__ import annotations

import math
import time

from dataclasses import dataclass, field

from . import inputs as I
from . import swept as S


@dataclass
class BuiltBatch:
    batch: "S.Batch"
    problems: list
    states: list
    items: list
    # scheme -> (width cap, flags), or (scheme, size class) -> (width cap, flags)
    widths: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return sum(p.n for p in self.problems)


def default_items(count: int, seed: int):
    """The batched workload's problems: lengths log-uniform in [2^10, 2^18]."""
    return I.batch_problems(count, seed, lo_exp=10.0, hi_exp=18.0, multiple=256)


def _problem(item, precision, W, flags=0):
    if item.scheme == "heat":
        return S.Problem(scheme=S.SW_HEAT, precision=precision, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                         n=item.n, r=item.r, tile_width=W, flags=0)
    return S.Problem(scheme=S.SW_EULER, precision=precision, boundary=S.SW_TRANSMISSIVE, method=S.SW_SWEPT,
                     n=item.n, dt_dx=I.riemann_lambda(), gamma=I.GAMMA, tile_width=W, flags=flags)


def tune_widths(items, precision=S.SW_FP32_COMP, candidates=(256, 512, 1024), sample_cells: int = 1 << 24):
    """One tile-width cap (and, for Euler, staging form) per scheme, chosen by timing
    the batch kernel itself on short runs (Section 6: tune W on a few short runs).

    For each scheme, a prefix of that scheme's items totalling about `sample_cells`
    cells (all of them when there are fewer) runs as its own batch once per
    candidate cap, each problem at the largest width <= the cap that fits it. The
    items are already in random order, so the prefix keeps the length mix; it is
    large enough to give every SM several work items per phase, as the whole batch
    does, so queue and occupancy effects are part of what is timed (a few small
    probe problems would leave most SMs idle and favour narrow tiles). Each timed
    run covers two phases of the widest candidate, after one untimed run of the
    same length. Returns {scheme: (width cap, flags)}: flags 0 for heat; for Euler
    SW_FLAG_LENGTHENED or SW_FLAG_FLATTENED, the form (Section 4.3) that timed faster."""
    import torch
    widths = {}
    for scheme in sorted({it.scheme for it in items}):
        sample, cells = [], 0
        for it in items:
            if it.scheme == scheme and cells < sample_cells:
                sample.append(it)
                cells += it.n
        levels = max(candidates)
        steps = levels if scheme == "heat" else levels // 4
        best = None
        forms = (S.SW_FLAG_LENGTHENED, S.SW_FLAG_FLATTENED) if scheme == "euler" else (0,)
        for cap, flags in [(c, f) for c in candidates for f in forms]:
            probs = [_problem(it, precision, fit_width(it.n, cap, flags), flags) for it in sample]
            states = [S.to_state(p, torch.as_tensor(it.planes.reshape(-1), device="cuda"))
                      for p, it in zip(probs, sample)]
            with S.Batch(probs, states, steps) as b:
                b.sw_batch_run()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                b.sw_batch_run()
                e1.record()
                e1.synchronize()
                t = e0.elapsed_time(e1)
                if b.sw_batch_status() != S.SW_OK:
                    continue
            if best is None or t < best[0]:
                best = (t, (cap, flags))
        widths[scheme] = best[1] if best else (256, 0)
    return widths


def fit_width(n: int, tuned: int, flags: int = 0) -> int:
    """Largest W <= tuned (halving) that divides n with at least two tiles; the
    flattened form needs W >= 8."""
    floor = 8 if flags & S.SW_FLAG_FLATTENED else 4
    W = tuned
    while W > floor and (n % W or n < 2 * W):
        W //= 2
    return W


def build(items, nsteps: int, precision=S.SW_FP32_COMP, widths=None, threads: int = 128) -> BuiltBatch:
    import torch
    widths = widths if widths is not None else tune_widths(items, precision)
    problems, states = [], []
    for it in items:
        cap, flags = choice(widths, it)
        W = fit_width(it.n, cap, flags)
        p = _problem(it, precision, W, flags)
        problems.append(p)
        states.append(S.to_state(p, torch.as_tensor(it.planes.reshape(-1), device="cuda")))
    batch = S.Batch(problems, states, nsteps)
    if threads != 128:
        batch.sw_batch_set_threads(threads)
    return BuiltBatch(batch, problems, states, items, widths)


def size_class(n: int) -> int:
    """The octave of a problem length: floor(log2 n)."""
    return int(math.floor(math.log2(n)))


def choice(widths: dict, item):
    """(width cap, flags) for an item from a per-scheme or a per-size-class table."""
    key = (item.scheme, size_class(item.n))
    v = widths.get(key, widths.get(item.scheme))
    if v is None:
        raise KeyError(f"no width for {key}")
    return v if isinstance(v, tuple) else (v, 0)


def _time_batch(items, table, precision, steps, threads=128):
    """Seconds of one run (after an untimed one) of a batch of `items` under `table`, with
    `threads` per CTA, or None when the run did not finish cleanly."""
    import torch
    probs, states = [], []
    for it in items:
        cap, flags = choice(table, it)
        p = _problem(it, precision, fit_width(it.n, cap, flags), flags)
        probs.append(p)
        states.append(S.to_state(p, torch.as_tensor(it.planes.reshape(-1), device="cuda")))
    with S.Batch(probs, states, steps) as b:
        if threads != 128:
            b.sw_batch_set_threads(threads)
        b.sw_batch_run()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.sw_batch_run()
        e1.record()
        e1.synchronize()
        if b.sw_batch_status() != S.SW_OK:
            return None
        return e0.elapsed_time(e1) / 1e3


def tune_classes(items, precision=S.SW_FP32_COMP, candidates=(128, 256, 512, 1024), sample_cells: int = 1 << 23,
                 max_problems: int = 2048):
    """Width cap (and, for Euler, staging form) per (scheme, size class), each chosen by the
    cell-steps per second of the batch kernel on a short run of that class alone.

    A class's sample is its items in batch order, repeated (as independent problems) until
    it holds about `sample_cells` cells (at most `max_problems` problems), so that every class is timed GPU-filling: the small
    classes then measure the throughput they get inside the whole batch, where their few
    phases overlap the long problems', not the latency of running them alone. Each timed run
    covers two phases of the widest candidate (heat: 1024 steps; Euler: 256 steps), after an
    untimed run. Returns {(scheme, class): (cap, flags)}."""
    table = {}
    classes = sorted({(it.scheme, size_class(it.n)) for it in items})
    for scheme, cls in classes:
        members = [it for it in items if it.scheme == scheme and size_class(it.n) == cls]
        sample, cells = [], 0
        while cells < sample_cells and len(sample) < max_problems:
            it = members[len(sample) % len(members)]
            sample.append(it)
            cells += it.n
        steps = max(candidates) if scheme == "heat" else max(candidates) // 4
        forms = (S.SW_FLAG_LENGTHENED, S.SW_FLAG_FLATTENED) if scheme == "euler" else (0,)
        best = None
        for cap in candidates:
            if cap > max(it.n for it in members) // 2 and cap != min(candidates):
                continue  # no problem of the class is long enough for it
            for flags in forms:
                t = _time_batch(sample, {scheme: (cap, flags)}, precision, steps)
                if t is None:
                    continue
                rate = cells * steps / t
                if best is None or rate > best[0]:
                    best = (rate, (cap, flags))
        table[(scheme, cls)] = best[1] if best else ((256, 0) if scheme == "heat" else (256, S.SW_FLAG_LENGTHENED))
    return table


def tune(items, precision=S.SW_FP32_COMP, check_steps: int = 500, threads=(64, 128, 256)):
    """Per-scheme caps and the per-size-class table, each timed on `check_steps` steps of the
    whole batch, then the threads per CTA of the persistent kernel for the winning table;
    returns (winning table, threads, report)."""
    t0 = time.perf_counter()
    per_scheme = tune_widths(items, precision)
    t1 = time.perf_counter()
    per_class = tune_classes(items, precision)
    t2 = time.perf_counter()
    cells = sum(it.n for it in items)
    rate_scheme = cells * check_steps / _time_batch(items, per_scheme, precision, check_steps) / 1e9
    rate_class = cells * check_steps / _time_batch(items, per_class, precision, check_steps) / 1e9
    winner = per_class if rate_class > rate_scheme else per_scheme
    rates_nt = {}
    for nt in threads:
        t = rate_scheme if (nt == 128 and winner is per_scheme) else \
            (rate_class if nt == 128 else None)
        if t is None:
            sec = _time_batch(items, winner, precision, check_steps, nt)
            t = cells * check_steps / sec / 1e9 if sec else 0.0
        rates_nt[nt] = t
    best_nt = max(rates_nt, key=rates_nt.get)
    report = {"per_scheme": {k: {"cap": v[0], "flags": v[1]} for k, v in per_scheme.items()},
              "per_class": {f"{k[0]} 2^{k[1]}": {"cap": v[0], "flags": v[1]} for k, v in sorted(per_class.items())},
              "check_steps": check_steps, "rate_per_scheme": rate_scheme, "rate_per_class": rate_class,
              "chosen": "per_class" if winner is per_class else "per_scheme",
              "rate_by_threads_per_cta": rates_nt, "threads_per_cta": best_nt,
              "tune_s_per_scheme": t1 - t0, "tune_s_per_class": t2 - t1, "tune_s": time.perf_counter() - t0}
    return winner, best_nt, report
