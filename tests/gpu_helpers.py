"""Shared helpers for the GPU tests: build/load the library, run through the C ABI."""
import numpy as np

from paper_1811_08282_gb300 import swept as S


def ensure_lib():
    from paper_1811_08282_gb300 import build
    build.build()
    return S.load()


def run_gpu(problem: S.Problem, planes_fp64, nsteps: int, sync=True) -> np.ndarray:
    """Advance FP64 planes (nv, n) with the library; returns FP64 planes on the host."""
    import torch
    x = torch.as_tensor(np.ascontiguousarray(planes_fp64, dtype=np.float64).reshape(-1), device="cuda")
    st = S.to_state(problem, x)
    with S.Handle(problem) as h:
        h.sw_run(st, nsteps)
        out = S.to_fp64(problem, st)
        rc = h.sw_sync_status()
        assert rc == 0, S.status_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(problem.nv, problem.n)


def norm_rel(got, want):
    """Norm-relative error max|g - o| / max|o| (per variable, max over variables)."""
    got = np.atleast_2d(got)
    want = np.atleast_2d(want)
    return max(float(np.max(np.abs(g - w)) / max(np.max(np.abs(w)), 1e-300)) for g, w in zip(got, want))
