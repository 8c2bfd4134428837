"""Thin ctypes binding of libswept.so (include/swept.h), same names as the C ABI.

Argument marshalling only: every step of the swept and per-step paths runs in
the CUDA kernels of the library. torch tensors are accepted where the C ABI
takes device pointers (their ``data_ptr()``), and streams default to
``torch.cuda.current_stream()``. There is no CPU fallback: if the library is
missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libswept.so")

ABI_VERSION = 5  # SW_ABI_VERSION of include/swept.h
SW_HEAT, SW_EULER = 0, 1
SW_FP64, SW_FP32, SW_FP32_COMP = 0, 1, 2
SW_PERIODIC, SW_TRANSMISSIVE = 0, 1
SW_SWEPT, SW_PERSTEP = 0, 1
SW_OK, SW_WARN_UNSTABLE = 0, 1
SW_ERR_BAD_ARG, SW_ERR_CUDA, SW_ERR_OOM = -1, -2, -3
SW_ERR_TIMEOUT, SW_ERR_NONPHYSICAL, SW_ERR_UNSUPPORTED = -4, -5, -6
SW_ERR_TOO_LARGE = -7
SW_ERR_CORRUPT = -8
SW_NOALLOC_SCRATCH_BYTES = 16 << 20
SW_MIN_TILE, SW_MAX_TILE = 4, 1024
SW_FLAG_GENERIC = 1
SW_FLAG_EULER_FOLD = 2
SW_FLAG_LENGTHENED = 4
SW_FLAG_FLATTENED = 8
SW_FLAG_GRAPH = 16

# every symbol declared in include/swept.h
EXPORTS = (
    "sw_create", "sw_destroy", "sw_state_planes", "sw_state_bytes", "sw_run", "sw_run_host",
    "sw_pack_fp64", "sw_unpack_fp64", "sw_conservation", "sw_check_physical", "sw_sync_status",
    "sw_last_launch_count", "sw_tile_width", "sw_status_string", "sw_abi_version",
    "sw_set_timing", "sw_launch_times", "sw_run_noalloc",
    "sw_batch_create", "sw_batch_run", "sw_batch_status", "sw_batch_items", "sw_batch_debug",
    "sw_batch_destroy", "sw_batch_set_threads", "sw_autotune", "sw_hybrid_split", "sw_run_hybrid", "sw_debug_corrupt_guard",
    "sw2d_create", "sw2d_destroy", "sw2d_run", "sw2d_last_launch_count", "sw2d_tile_width", "sw2d_set_timing",
    "sw2d_launch_times", "sw2d_set_threads", "sw2d_threads",
)


class sw_problem(ctypes.Structure):
    _fields_ = [
        ("scheme", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("r", ctypes.c_double),
        ("dt_dx", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("tile_width", ctypes.c_int32),
        ("flags", ctypes.c_int32),
    ]


class sw_heat2d(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("method", ctypes.c_int32),
        ("tile_width", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("rx", ctypes.c_double),
        ("ry", ctypes.c_double),
    ]


class SweptError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_string(code)} ({code})")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libswept.so and declare its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libswept.so not found at {path}; build it with "
                           "`python -m paper_1811_08282_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER(sw_problem)
    sig = {
        "sw_create": ([P, ctypes.POINTER(vp)], ctypes.c_int),
        "sw_destroy": ([vp], None),
        "sw_state_planes": ([P], ctypes.c_int),
        "sw_state_bytes": ([P], i64),
        "sw_run": ([vp, vp, i64, vp], ctypes.c_int),
        "sw_run_host": ([vp, vp, vp, i64, vp], ctypes.c_int),
        "sw_hybrid_split": ([i64, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "sw_run_hybrid": ([vp, vp, i64, i32, i32, vp], ctypes.c_int),
        "sw_debug_corrupt_guard": ([vp, i32], ctypes.c_int),
        "sw_pack_fp64": ([P, vp, vp, vp], ctypes.c_int),
        "sw_unpack_fp64": ([P, vp, vp, vp], ctypes.c_int),
        "sw_conservation": ([vp, vp, ctypes.POINTER(dbl), vp], ctypes.c_int),
        "sw_check_physical": ([vp, vp, ctypes.POINTER(i64), vp], ctypes.c_int),
        "sw_sync_status": ([vp, vp], ctypes.c_int),
        "sw_last_launch_count": ([vp], i64),
        "sw_tile_width": ([vp], i32),
        "sw_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "sw_abi_version": ([], ctypes.c_int),
        "sw_set_timing": ([vp, i64], ctypes.c_int),
        "sw_launch_times": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32), i64], i64),
        "sw_run_noalloc": ([P, vp, i64, vp], ctypes.c_int),
        "sw_batch_create": ([P, ctypes.POINTER(vp), i32, i64, ctypes.POINTER(vp)], ctypes.c_int),
        "sw_batch_run": ([vp, vp], ctypes.c_int),
        "sw_batch_status": ([vp, vp], ctypes.c_int),
        "sw_batch_items": ([vp], i64),
        "sw_batch_debug": ([vp, i64, i32], ctypes.c_int),
        "sw_batch_destroy": ([vp], None),
        "sw_batch_set_threads": ([vp, i32], ctypes.c_int),
        "sw_autotune": ([P, i64, vp], ctypes.c_int),
        "sw2d_create": ([ctypes.POINTER(sw_heat2d), ctypes.POINTER(vp)], ctypes.c_int),
        "sw2d_destroy": ([vp], None),
        "sw2d_run": ([vp, vp, i64, vp], ctypes.c_int),
        "sw2d_last_launch_count": ([vp], i64),
        "sw2d_tile_width": ([vp], i32),
        "sw2d_set_threads": ([vp, i32, i32], ctypes.c_int),
        "sw2d_threads": ([vp, i32], i32),
        "sw2d_set_timing": ([vp, i64], ctypes.c_int),
        "sw2d_launch_times": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32), i64], i64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if lib.sw_abi_version() != ABI_VERSION:
        raise RuntimeError(f"libswept.so at {path} has ABI version {lib.sw_abi_version()}, this binding "
                           f"expects {ABI_VERSION}: rebuild it with `python -m paper_1811_08282_gb300.build`")
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().sw_status_string(int(code)).decode()


def _ptr(x) -> int:
    """Device (or host) address of a torch tensor, or an int passed through."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise SweptError(rc, where)
    return rc


@dataclass
class Problem:
    """Python view of ``sw_problem`` (Section 4.2's problem statement)."""
    scheme: int = SW_HEAT
    precision: int = SW_FP64
    boundary: int = SW_PERIODIC
    method: int = SW_SWEPT
    n: int = 1024
    r: float = 0.25
    dt_dx: float = 0.0
    gamma: float = 1.4
    tile_width: int = 0
    flags: int = 0

    def c(self) -> sw_problem:
        return sw_problem(int(self.scheme), int(self.precision), int(self.boundary), int(self.method),
                          int(self.n), float(self.r), float(self.dt_dx), float(self.gamma),
                          int(self.tile_width), int(self.flags))

    @property
    def nv(self) -> int:
        return 1 if self.scheme == SW_HEAT else 3


def sw_state_planes(p: Problem) -> int:
    return _check(load().sw_state_planes(ctypes.byref(p.c())), "sw_state_planes")


def sw_state_bytes(p: Problem) -> int:
    return _check(load().sw_state_bytes(ctypes.byref(p.c())), "sw_state_bytes")


def sw_abi_version() -> int:
    return load().sw_abi_version()


def sw_status_string(code: int) -> str:
    return status_string(code)


def sw_pack_fp64(p: Problem, src_fp64, dst_state, stream=None) -> None:
    _check(load().sw_pack_fp64(ctypes.byref(p.c()), _ptr(src_fp64), _ptr(dst_state), _stream(stream)),
           "sw_pack_fp64")


def sw_unpack_fp64(p: Problem, src_state, dst_fp64, stream=None) -> None:
    _check(load().sw_unpack_fp64(ctypes.byref(p.c()), _ptr(src_state), _ptr(dst_fp64), _stream(stream)),
           "sw_unpack_fp64")


def sw_run_noalloc(p: Problem, state, nsteps: int, stream=None) -> int:
    """Swept run with no device allocation (flank scratch in the library's static
    16 MiB device array); for callers that cannot call cudaMalloc. Calls share the
    array: do not overlap them on the GPU. Returns SW_OK or SW_WARN_UNSTABLE."""
    cp = p.c()
    return _check(load().sw_run_noalloc(ctypes.byref(cp), _ptr(state), int(nsteps), _stream(stream)),
                  "sw_run_noalloc")


class Handle:
    """Owner of an ``sw_handle`` (scratch on the current device)."""

    def __init__(self, problem: Problem):
        self.problem = problem
        self._cp = problem.c()
        h = ctypes.c_void_p()
        rc = load().sw_create(ctypes.byref(self._cp), ctypes.byref(h))
        _check(rc, "sw_create")
        self.warning = rc
        self._h = h

    @property
    def ptr(self) -> int:
        return self._h.value

    def close(self) -> None:
        if self._h and self._h.value:
            load().sw_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sw_run(self, state, nsteps: int, stream=None) -> None:
        _check(load().sw_run(self._h, _ptr(state), int(nsteps), _stream(stream)), "sw_run")

    def sw_run_host(self, state_in, state_out, nsteps: int, stream=None) -> None:
        _check(load().sw_run_host(self._h, _ptr(state_in), _ptr(state_out), int(nsteps), _stream(stream)),
               "sw_run_host")

    def sw_run_hybrid(self, state, nsteps: int, work_factor: int, cpu_threads: int, stream=None) -> None:
        """Swept run shared with `cpu_threads` host threads (GPU work factor `work_factor`)."""
        _check(load().sw_run_hybrid(self._h, _ptr(state), int(nsteps), int(work_factor), int(cpu_threads),
                                    _stream(stream)), "sw_run_hybrid")

    def sw_debug_corrupt_guard(self, which: int) -> None:
        """Test hook: overwrite a guard byte after scratch buffer `which` (0, 1 flanks; 2 per-step)."""
        _check(load().sw_debug_corrupt_guard(self._h, int(which)), "sw_debug_corrupt_guard")

    def sw_conservation(self, state, stream=None):
        sums = (ctypes.c_double * 3)()
        _check(load().sw_conservation(self._h, _ptr(state), sums, _stream(stream)), "sw_conservation")
        return [sums[i] for i in range(self.problem.nv)]

    def sw_check_physical(self, state, stream=None) -> int:
        """Returns -1 when every cell has rho > 0, p > 0 and finite values, else the first bad cell."""
        cell = ctypes.c_int64(-1)
        rc = load().sw_check_physical(self._h, _ptr(state), ctypes.byref(cell), _stream(stream))
        if rc not in (SW_OK, SW_ERR_NONPHYSICAL):
            _check(rc, "sw_check_physical")
        return int(cell.value)

    def sw_sync_status(self, stream=None) -> int:
        return load().sw_sync_status(self._h, _stream(stream))

    def sw_last_launch_count(self) -> int:
        return int(load().sw_last_launch_count(self._h))

    def sw_tile_width(self) -> int:
        return int(load().sw_tile_width(self._h))

    def sw_set_timing(self, capacity: int) -> None:
        _check(load().sw_set_timing(self._h, int(capacity)), "sw_set_timing")

    def sw_launch_times(self, cap: int = 1 << 16):
        """[(ms, kind)] of the last run's traced launches (kind 0 Up, 1 Diamond, 2 Down, 3 per-step)."""
        ms = (ctypes.c_float * cap)()
        kind = (ctypes.c_int32 * cap)()
        cnt = _check(int(load().sw_launch_times(self._h, ms, kind, int(cap))), "sw_launch_times")
        return [(float(ms[i]), int(kind[i])) for i in range(cnt)]


def sw_hybrid_split(tiles: int, work_factor: int, cpu_threads: int):
    """(gpu_tiles, tiles_per_thread) of the affinity split (Eq. 1's work factor)."""
    g, per = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().sw_hybrid_split(int(tiles), int(work_factor), int(cpu_threads), ctypes.byref(g), ctypes.byref(per)),
           "sw_hybrid_split")
    return g.value, per.value


def sw_create(problem: Problem) -> Handle:
    return Handle(problem)


class Batch:
    """Owner of an ``sw_batch``: problems[i] advanced on the device state states[i]."""

    def __init__(self, problems, states, nsteps: int):
        arr = (sw_problem * len(problems))(*[p.c() for p in problems])
        ptrs = (ctypes.c_void_p * len(states))(*[_ptr(s) for s in states])
        b = ctypes.c_void_p()
        _check(load().sw_batch_create(arr, ptrs, len(problems), int(nsteps), ctypes.byref(b)),
               "sw_batch_create")
        self._b = b
        self.problems = list(problems)
        self.states = list(states)  # keep the device buffers alive

    def close(self) -> None:
        if self._b and self._b.value:
            load().sw_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sw_batch_run(self, stream=None) -> None:
        _check(load().sw_batch_run(self._b, _stream(stream)), "sw_batch_run")

    def sw_batch_status(self, stream=None) -> int:
        return int(load().sw_batch_status(self._b, _stream(stream)))

    def sw_batch_items(self) -> int:
        return int(load().sw_batch_items(self._b))

    def sw_batch_set_threads(self, threads: int) -> None:
        """Threads per CTA of the persistent kernel (64, 128 or 256)."""
        _check(load().sw_batch_set_threads(self._b, int(threads)), "sw_batch_set_threads")

    def sw_batch_debug(self, wait_budget_cycles: int, drop_publish: bool) -> None:
        _check(load().sw_batch_debug(self._b, int(wait_budget_cycles), 1 if drop_publish else 0),
               "sw_batch_debug")


def sw_batch_create(problems, states, nsteps: int) -> Batch:
    return Batch(problems, states, nsteps)


def sw_autotune(p: Problem, probe_steps: int, stream=None) -> int:
    """Fastest tile width for ``p`` over short timed runs; also stored in ``p.tile_width``."""
    cp = p.c()
    _check(load().sw_autotune(ctypes.byref(cp), int(probe_steps), _stream(stream)), "sw_autotune")
    p.tile_width = int(cp.tile_width)
    return p.tile_width


@dataclass
class Heat2D:
    """Python view of ``sw_heat2d``: FTCS heat on an nx x ny grid (state (ny, nx), x fastest)."""
    precision: int = SW_FP64
    boundary: int = SW_PERIODIC
    method: int = SW_SWEPT
    tile_width: int = 0
    nx: int = 256
    ny: int = 256
    rx: float = 0.2
    ry: float = 0.2

    def c(self) -> sw_heat2d:
        return sw_heat2d(int(self.precision), int(self.boundary), int(self.method), int(self.tile_width),
                         int(self.nx), int(self.ny), float(self.rx), float(self.ry))


class Handle2D:
    """Owner of an ``sw_handle2d`` (strip buffers on the current device)."""

    def __init__(self, problem: Heat2D):
        self.problem = problem
        self._cp = problem.c()
        h = ctypes.c_void_p()
        rc = load().sw2d_create(ctypes.byref(self._cp), ctypes.byref(h))
        _check(rc, "sw2d_create")
        self.warning = rc
        self._h = h

    def close(self) -> None:
        if self._h and self._h.value:
            load().sw2d_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sw2d_run(self, state, nsteps: int, stream=None) -> None:
        _check(load().sw2d_run(self._h, _ptr(state), int(nsteps), _stream(stream)), "sw2d_run")

    def sw2d_last_launch_count(self) -> int:
        return int(load().sw2d_last_launch_count(self._h))

    def sw2d_tile_width(self) -> int:
        return int(load().sw2d_tile_width(self._h))

    def sw2d_set_threads(self, threads: int, bridge_threads: int = 0) -> None:
        _check(load().sw2d_set_threads(self._h, int(threads), int(bridge_threads)), "sw2d_set_threads")

    def sw2d_threads(self, bridges: bool = False) -> int:
        return int(load().sw2d_threads(self._h, int(bool(bridges))))

    def sw2d_set_timing(self, capacity: int) -> None:
        _check(load().sw2d_set_timing(self._h, int(capacity)), "sw2d_set_timing")

    def sw2d_launch_times(self, cap: int = 1 << 16):
        """[(ms, kind)] of the last run's traced launches (0 Up, 1 bridges, 2 octahedra,
        3 per-step, 4 last octahedra)."""
        ms = (ctypes.c_float * cap)()
        kind = (ctypes.c_int32 * cap)()
        cnt = _check(int(load().sw2d_launch_times(self._h, ms, kind, int(cap))), "sw2d_launch_times")
        return [(float(ms[i]), int(kind[i])) for i in range(cnt)]


def sw2d_create(problem: Heat2D) -> Handle2D:
    return Handle2D(problem)


# --------------------------------------------------------------- conveniences
def state_dtype(p: Problem):
    import torch
    return torch.float64 if p.precision == SW_FP64 else torch.float32


def to_state(p: Problem, fp64_planes, stream=None):
    """Device state in the working layout of ``p`` from FP64 planes (torch, cuda)."""
    import torch
    src = fp64_planes.to(device="cuda", dtype=torch.float64).contiguous()
    assert src.numel() == p.nv * p.n
    planes = sw_state_planes(p)
    dst = torch.empty(planes * p.n, dtype=state_dtype(p), device="cuda")
    sw_pack_fp64(p, src, dst, stream)
    return dst


def to_fp64(p: Problem, state, stream=None):
    """FP64 planes (nv, n) on the device from a state in the working layout."""
    import torch
    out = torch.empty(p.nv * p.n, dtype=torch.float64, device="cuda")
    sw_unpack_fp64(p, state, out, stream)
    return out.view(p.nv, p.n)


def run(p: Problem, fp64_planes, nsteps: int):
    """One-call form: FP64 planes in (numpy or torch), FP64 planes (torch, cuda) out."""
    import torch
    x = torch.as_tensor(fp64_planes, dtype=torch.float64)
    st = to_state(p, x.reshape(-1))
    with Handle(p) as h:
        h.sw_run(st, nsteps)
        out = to_fp64(p, st)
        rc = h.sw_sync_status()
        _check(rc, "sw_run (device status)")
    return out
