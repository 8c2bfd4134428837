"""Build an autotuned batch of independent problems (one persistent launch per run).

    from paper_1811_08282_gb300 import batched
    bt = batched.build(batched.default_items(4096, seed=7), nsteps=10_000)
    bt.batch.sw_batch_run(); bt.batch.sw_batch_status()

Tile widths come from the library's autotuner (sw_autotune: short timed runs per
width, Section 6's advice) applied once per (scheme, power-of-two size class) and
then fitted to each problem's length (largest tuned-or-smaller width that divides
it). Heat problems are periodic, Euler problems transmissive Riemann problems.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import inputs as I
from . import swept as S


@dataclass
class BuiltBatch:
    batch: "S.Batch"
    problems: list
    states: list
    items: list
    widths: dict = field(default_factory=dict)  # (scheme, size class) -> tuned width

    @property
    def cells(self) -> int:
        return sum(p.n for p in self.problems)


def default_items(count: int, seed: int):
    """The batched workload's problems: lengths log-uniform in [2^10, 2^18]."""
    return I.batch_problems(count, seed, lo_exp=10.0, hi_exp=18.0, multiple=256)


def _problem(item, precision, W, flags=0):
    if item.scheme == "heat":
        return S.Problem(scheme=S.SW_HEAT, precision=precision, boundary=S.SW_PERIODIC, method=S.SW_SWEPT,
                         n=item.n, r=item.r, tile_width=W, flags=flags)
    return S.Problem(scheme=S.SW_EULER, precision=precision, boundary=S.SW_TRANSMISSIVE, method=S.SW_SWEPT,
                     n=item.n, dt_dx=I.riemann_lambda(), gamma=I.GAMMA, tile_width=W, flags=flags)


def tune_widths(items, precision=S.SW_FP32_COMP, probe_steps: int = 256):
    """Tuned width per (scheme, size class 2^k), measured on a length-2^k problem."""
    widths = {}
    for it in items:
        k = int(round(math.log2(it.n)))
        key = (it.scheme, k)
        if key in widths:
            continue
        probe = _problem(I.BatchItem(it.scheme, 1 << k, 0.3, None), precision, 0, flags=S.SW_FLAG_GENERIC)
        widths[key] = S.sw_autotune(probe, probe_steps)
    return widths


def fit_width(n: int, tuned: int) -> int:
    W = tuned
    while W > 4 and (n % W or n < 2 * W):
        W //= 2
    return W


def build(items, nsteps: int, precision=S.SW_FP32_COMP, widths=None) -> BuiltBatch:
    import torch
    widths = widths if widths is not None else tune_widths(items, precision)
    problems, states = [], []
    for it in items:
        k = int(round(math.log2(it.n)))
        W = fit_width(it.n, widths[(it.scheme, k)])
        p = _problem(it, precision, W)
        problems.append(p)
        states.append(S.to_state(p, torch.as_tensor(it.planes.reshape(-1), device="cuda")))
    return BuiltBatch(S.Batch(problems, states, nsteps), problems, states, items, widths)
