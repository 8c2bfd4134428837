"""Build an autotuned batch of independent problems (one persistent launch per run).

    from paper_1811_08282_gb300 import batched
    bt = batched.build(batched.default_items(4096, seed=7), nsteps=10_000)
    bt.batch.sw_batch_run(); bt.batch.sw_batch_status()

Tile widths are tuned as one cap per scheme by timing the batch kernel itself on
short runs of a GPU-filling sample of the items (Section 6's advice: tune on a few
short runs), then fitted to each problem's length (largest width <= the cap that
divides it and leaves at least two tiles). For Euler the tuner also picks the
staging form of Section 4.3, lengthened or flattened (same results). Heat problems
are periodic, Euler problems transmissive Riemann problems.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import inputs as I
from . import swept as S


@dataclass
class BuiltBatch:
    batch: "S.Batch"
    problems: list
    states: list
    items: list
    widths: dict = field(default_factory=dict)  # scheme -> (tuned width cap, flags)

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


def build(items, nsteps: int, precision=S.SW_FP32_COMP, widths=None) -> BuiltBatch:
    import torch
    widths = widths if widths is not None else tune_widths(items, precision)
    problems, states = [], []
    for it in items:
        cap, flags = widths[it.scheme] if isinstance(widths[it.scheme], tuple) else (widths[it.scheme], 0)
        W = fit_width(it.n, cap, flags)
        p = _problem(it, precision, W, flags)
        problems.append(p)
        states.append(S.to_state(p, torch.as_tensor(it.planes.reshape(-1), device="cuda")))
    return BuiltBatch(S.Batch(problems, states, nsteps), problems, states, items, widths)
