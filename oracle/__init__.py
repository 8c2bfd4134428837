"""FP64 CPU oracle for the 1D swept stencil path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package. The product path (the C-ABI
library and its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
this module compiles it on first use with the host ``gcc`` and wraps the entry
points with numpy arrays.  Each wrapper names the scheme reading it follows;
the readings themselves are written out in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC = 0
TRANSMISSIVE = 1


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        pd = ctypes.POINTER(ctypes.c_double)
        pl = ctypes.POINTER(ctypes.c_int64)
        lib.orc_num_threads.restype = i32
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_set_threads.restype = None
        lib.orc_heat_run.argtypes = [i64, f64, i32, i64, pd]
        lib.orc_heat_run.restype = i32
        lib.orc_heat_modes.argtypes = [i64, f64, i64, i32, pd, pl, pl, i64, pd]
        lib.orc_heat_modes.restype = i32
        pi32 = ctypes.POINTER(ctypes.c_int32)
        lib.orc_heat2d_run.argtypes = [i64, i64, f64, f64, i32, i64, pd]
        lib.orc_heat2d_run.restype = i32
        lib.orc_heat2d_modes.argtypes = [i64, i64, f64, f64, i64, i32, pd, pl, pl, pi32, pi32, pl, pl, i64, pd]
        lib.orc_heat2d_modes.restype = i32
        lib.orc_euler_run.argtypes = [i64, f64, f64, i32, i64, pd, pd, pd]
        lib.orc_euler_run.restype = i32
        lib.orc_riemann_star.argtypes = [f64] * 7 + [pd]
        lib.orc_riemann_star.restype = i32
        lib.orc_riemann_sample.argtypes = [f64] * 7 + [pd, i64, pd, pd, pd, pd]
        lib.orc_riemann_sample.restype = i32
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lptr(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def num_threads() -> int:
    """Threads the oracle's parallel cell loops use (OpenMP)."""
    return int(_load().orc_num_threads())


def set_threads(n: int) -> None:
    """Use `n` threads in the parallel cell loops from now on (results are unchanged)."""
    _load().orc_set_threads(int(n))


def heat_run(u0, r: float, nsteps: int, boundary: int = PERIODIC) -> np.ndarray:
    """FTCS heat equation, naive stepping (Section 4.2). Returns a new array."""
    u = np.array(u0, dtype=np.float64, copy=True, order="C")
    rc = _load().orc_heat_run(u.size, float(r), int(boundary), int(nsteps), _dptr(u))
    if rc != 0:
        raise RuntimeError(f"orc_heat_run failed: {rc}")
    return u


def heat_modes(n: int, r: float, nsteps: int, amps, ks, idx=None) -> np.ndarray:
    """Exact discrete FTCS solution of a periodic sum of sine modes (long double)."""
    amps = np.ascontiguousarray(amps, dtype=np.float64)
    ks = np.ascontiguousarray(ks, dtype=np.int64)
    idx = np.arange(n, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.size, dtype=np.float64)
    rc = _load().orc_heat_modes(int(n), float(r), int(nsteps), int(amps.size),
                                _dptr(amps), _lptr(ks), _lptr(idx), idx.size, _dptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_heat_modes failed: {rc}")
    return out


def heat2d_run(u0, rx: float, ry: float, nsteps: int, boundary: int = PERIODIC) -> np.ndarray:
    """2D FTCS heat equation (5-point stencil), naive stepping. ``u0`` has shape (ny, nx)
    (x fastest). Returns a new array."""
    u = np.array(u0, dtype=np.float64, copy=True, order="C")
    assert u.ndim == 2
    rc = _load().orc_heat2d_run(u.shape[1], u.shape[0], float(rx), float(ry), int(boundary), int(nsteps), _dptr(u))
    if rc != 0:
        raise RuntimeError(f"orc_heat2d_run failed: {rc}")
    return u


def heat2d_modes(nx: int, ny: int, rx: float, ry: float, nsteps: int, amps, kx, ky, fx, fy, ii, jj) -> np.ndarray:
    """Exact discrete 2D FTCS solution of a periodic sum of separable sin/cos modes, at
    cells (ii[q], jj[q]) (long double)."""
    amps = np.ascontiguousarray(amps, dtype=np.float64)
    kx = np.ascontiguousarray(kx, dtype=np.int64)
    ky = np.ascontiguousarray(ky, dtype=np.int64)
    fx = np.ascontiguousarray(fx, dtype=np.int32)
    fy = np.ascontiguousarray(fy, dtype=np.int32)
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.empty(ii.size, dtype=np.float64)
    p32 = ctypes.POINTER(ctypes.c_int32)
    rc = _load().orc_heat2d_modes(int(nx), int(ny), float(rx), float(ry), int(nsteps), int(amps.size), _dptr(amps),
                                  _lptr(kx), _lptr(ky), fx.ctypes.data_as(p32), fy.ctypes.data_as(p32), _lptr(ii),
                                  _lptr(jj), ii.size, _dptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_heat2d_modes failed: {rc}")
    return out


def euler_run(q0, lam: float, gamma: float, nsteps: int,
              boundary: int = TRANSMISSIVE) -> np.ndarray:
    """Second-order FV Euler scheme, naive two-stage stepping (Sections 4.2-4.3).

    ``q0`` has shape (3, n): density, momentum, total energy. Returns a new array.
    """
    q = np.array(q0, dtype=np.float64, copy=True, order="C")
    assert q.ndim == 2 and q.shape[0] == 3
    rc = _load().orc_euler_run(q.shape[1], float(lam), float(gamma), int(boundary),
                               int(nsteps), _dptr(q[0]), _dptr(q[1]), _dptr(q[2]))
    if rc != 0:
        raise RuntimeError(f"orc_euler_run failed: {rc}")
    return q


def riemann_star(left, right, gamma: float = 1.4):
    """Exact Riemann star state: (p*, u*, rho*_L, rho*_R) for primitive (rho, u, p)."""
    out = np.empty(4, dtype=np.float64)
    rc = _load().orc_riemann_star(*map(float, left), *map(float, right), float(gamma), _dptr(out))
    if rc != 0:
        raise ValueError("Riemann data generate vacuum")
    return out


def riemann_sample(left, right, xi, gamma: float = 1.4):
    """Exact Riemann solution at x/t = xi. Returns (rho, u, p, wave_speeds[5])."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    waves = np.empty(5, dtype=np.float64)
    rc = _load().orc_riemann_sample(*map(float, left), *map(float, right), float(gamma),
                                    _dptr(xi), xi.size, _dptr(rho), _dptr(u), _dptr(p),
                                    _dptr(waves))
    if rc != 0:
        raise ValueError("Riemann data generate vacuum")
    return rho, u, p, waves
