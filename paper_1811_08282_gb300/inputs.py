"""Seeded synthetic inputs shaped like the paper's test problems.

This module is shared by the tests, the benchmark and the smoke check. It holds
no arithmetic of either numerical scheme: it only draws initial states and
parameters (SplitMix64, a counter-based generator) and converts primitive gas
states (rho, u, p) to the conservative variables the solvers take as input.

Problem shapes follow Section 4.2 of the paper (1D heat equation and 1D Euler
equations, grids of powers of two): sums of seeded sine modes for heat; the Sod
shock tube and seeded random Riemann problems for Euler; batches of both with
log-uniform lengths.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, stream: int = 0) -> np.ndarray:
    """SplitMix64 outputs for counters 1..count of (seed, stream), as uint64.

    Counter-based: output i is mix(seed' + (i+1) * golden), seed' = seed mixed
    with the stream id, so any sub-range can be regenerated independently.
    """
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream & 0xFFFFFFFF) * _M2)
        x = base + (np.arange(1, count + 1, dtype=np.uint64) * _GOLDEN)
        z = x
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0, stream: int = 0) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, count, stream) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def randint(seed: int, count: int, lo: int, hi: int, stream: int = 0) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by scaling a uniform double."""
    u = uniform(seed, count, 0.0, 1.0, stream)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# --------------------------------------------------------------------------- heat
@dataclass(frozen=True)
class HeatModes:
    """Initial state u_j = sum_m amps[m] * sin(2 pi ks[m] j / n)."""
    n: int
    amps: np.ndarray
    ks: np.ndarray


def heat_modes(n: int, n_modes: int, seed: int, kmax: int = 64) -> HeatModes:
    """Seeded amplitudes U[-1,1] and integer wavenumbers U{1..kmax}."""
    kmax = int(min(kmax, max(1, n // 2)))
    amps = uniform(seed, n_modes, -1.0, 1.0, stream=1)
    ks = randint(seed, n_modes, 1, kmax, stream=2)
    return HeatModes(n=n, amps=amps, ks=ks)


def heat_initial(modes: HeatModes) -> np.ndarray:
    """Evaluate the sine-mode sum on the n cells (angles reduced exactly mod n)."""
    n = modes.n
    j = np.arange(n, dtype=np.int64)
    u = np.zeros(n, dtype=np.float64)
    for a, k in zip(modes.amps, modes.ks):
        kj = (int(k) * j) % n
        u += a * np.sin((2.0 * np.pi / n) * kj.astype(np.float64))
    return u


def heat_r(seed: int, lo: float = 0.1, hi: float = 0.45) -> float:
    """Seeded diffusion number r = alpha dt / dx^2 drawn U[lo, hi]."""
    return float(uniform(seed, 1, lo, hi, stream=3)[0])


@dataclass(frozen=True)
class HeatModes2D:
    """Initial state u_ij = sum_m amps[m] f_m(2 pi kx[m] i / nx) g_m(2 pi ky[m] j / ny),
    f, g = sin when fx / fy is 0, cos when 1; array layout (ny, nx), x fastest."""
    nx: int
    ny: int
    amps: np.ndarray
    kx: np.ndarray
    ky: np.ndarray
    fx: np.ndarray
    fy: np.ndarray


def heat2d_modes(nx: int, ny: int, n_modes: int, seed: int, kmax: int = 32) -> HeatModes2D:
    """Seeded amplitudes U[-1,1], integer wavenumbers U{1..kmax} per direction, sin or cos."""
    amps = uniform(seed, n_modes, -1.0, 1.0, stream=31)
    kx = randint(seed, n_modes, 1, int(min(kmax, max(1, nx // 2))), stream=32)
    ky = randint(seed, n_modes, 1, int(min(kmax, max(1, ny // 2))), stream=33)
    fx = randint(seed, n_modes, 0, 1, stream=34).astype(np.int32)
    fy = randint(seed, n_modes, 0, 1, stream=35).astype(np.int32)
    return HeatModes2D(nx=nx, ny=ny, amps=amps, kx=kx, ky=ky, fx=fx, fy=fy)


def heat2d_initial(modes: HeatModes2D) -> np.ndarray:
    """Evaluate the separable mode sum on the (ny, nx) grid (angles reduced exactly)."""
    nx, ny = modes.nx, modes.ny
    i = np.arange(nx, dtype=np.int64)
    j = np.arange(ny, dtype=np.int64)
    u = np.zeros((ny, nx), dtype=np.float64)
    for a, kx, ky, fx, fy in zip(modes.amps, modes.kx, modes.ky, modes.fx, modes.fy):
        ax = (2.0 * np.pi / nx) * ((int(kx) * i) % nx).astype(np.float64)
        ay = (2.0 * np.pi / ny) * ((int(ky) * j) % ny).astype(np.float64)
        f = np.cos(ax) if fx else np.sin(ax)
        g = np.cos(ay) if fy else np.sin(ay)
        u += a * np.outer(g, f)
    return u


# -------------------------------------------------------------------------- euler
GAMMA = 1.4


def primitive_to_conservative(rho, u, p, gamma: float = GAMMA) -> np.ndarray:
    """(rho, u, p) -> (rho, rho u, E) with E = p/(gamma-1) + rho u^2 / 2; shape (3, n)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    return np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])


SOD_LEFT = (1.0, 0.0, 1.0)
SOD_RIGHT = (0.125, 0.0, 0.1)
# Upper bound on the fastest signal speed |u| + c of the Sod solution (the
# right star state: u* + c*_R ~= 2.1909); the tests check it against the
# exact Riemann solution.
SOD_MAX_SPEED = 2.2


def sod(n: int, gamma: float = GAMMA) -> np.ndarray:
    """Sod shock tube on [0,1], interface at x = 1/2 (cells j < n/2 are left)."""
    left = np.arange(n) < n // 2
    rho = np.where(left, SOD_LEFT[0], SOD_RIGHT[0])
    u = np.where(left, SOD_LEFT[1], SOD_RIGHT[1])
    p = np.where(left, SOD_LEFT[2], SOD_RIGHT[2])
    return primitive_to_conservative(rho, u, p, gamma)


def sod_lambda(cfl: float = 0.4) -> float:
    """dt/dx for the Sod problem at the given Courant number."""
    return cfl / SOD_MAX_SPEED


@dataclass(frozen=True)
class RiemannSegments:
    """Piecewise-constant primitive states: segment s covers cells [s*n/nseg, (s+1)*n/nseg)."""
    n: int
    rho: np.ndarray
    u: np.ndarray
    p: np.ndarray


def riemann_segments(n: int, nseg: int, seed: int) -> RiemannSegments:
    """Seeded states: rho, p log-uniform in [0.1, 1], u uniform in [-0.5, 0.5]."""
    rho = 10.0 ** uniform(seed, nseg, -1.0, 0.0, stream=11)
    p = 10.0 ** uniform(seed, nseg, -1.0, 0.0, stream=12)
    u = uniform(seed, nseg, -0.5, 0.5, stream=13)
    return RiemannSegments(n=n, rho=rho, u=u, p=p)


def riemann_initial(seg: RiemannSegments, gamma: float = GAMMA) -> np.ndarray:
    nseg = seg.rho.size
    which = (np.arange(seg.n, dtype=np.int64) * nseg) // seg.n
    return primitive_to_conservative(seg.rho[which], seg.u[which], seg.p[which], gamma)


# Upper bound on |u| + c for the random Riemann states above, including their
# star regions (checked against the exact Riemann solutions by the tests):
# max c = sqrt(1.4 * 1 / 0.1) ~= 3.74, |u| <= 0.5, star states stay below 5.
RIEMANN_MAX_SPEED = 5.0


def riemann_lambda(cfl: float = 0.4) -> float:
    return cfl / RIEMANN_MAX_SPEED


# ------------------------------------------------------------------------ batches
@dataclass(frozen=True)
class BatchItem:
    """One problem of a batch: heat (periodic, r) or Euler (transmissive Riemann problem)."""
    scheme: str        # "heat" or "euler"
    n: int
    r: float           # heat only
    planes: np.ndarray  # FP64 initial state, shape (nv, n)


def batch_lengths(count: int, seed: int, lo_exp: float = 10.0, hi_exp: float = 18.0,
                  multiple: int = 256) -> np.ndarray:
    """Problem lengths of a batch: log-uniform in [2^lo_exp, 2^hi_exp], rounded to a
    multiple of `multiple` (at least `multiple`)."""
    e = uniform(seed, count, lo_exp, hi_exp, stream=21)
    return np.maximum(multiple, np.round(2.0 ** e / multiple).astype(np.int64) * multiple)


def batch_item(i: int, n: int, r: float, seed: int) -> BatchItem:
    """Problem i of a batch of length n: even i heat (r, 8 sine modes, k <= min(64, n/8)),
    odd i Euler (one Riemann problem, interface at the middle, states as in
    riemann_segments)."""
    if i % 2 == 0:
        modes = heat_modes(n, 8, seed=seed * 100003 + i, kmax=min(64, max(1, n // 8)))
        return BatchItem("heat", n, float(r), heat_initial(modes)[None])
    seg = riemann_segments(n, 2, seed * 100003 + i)
    return BatchItem("euler", n, 0.0, riemann_initial(seg))


def batch_problems(count: int, seed: int, lo_exp: float = 10.0, hi_exp: float = 18.0,
                   multiple: int = 256, indices=None):
    """Lengths log-uniform in [2^lo_exp, 2^hi_exp] rounded to a multiple of `multiple`;
    even indices heat (r ~ U[0.1, 0.45], 8 sine modes, k <= min(64, n/8)), odd indices
    Euler (one Riemann problem per domain, interface at the middle, states as in
    riemann_segments). `indices`: only those problems of the batch (same draws)."""
    ns = batch_lengths(count, seed, lo_exp, hi_exp, multiple)
    rs = uniform(seed, count, 0.1, 0.45, stream=22)
    which = range(count) if indices is None else indices
    return [batch_item(i, int(ns[i]), float(rs[i]), seed) for i in which]
