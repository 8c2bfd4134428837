"""Host engine of the hybrid CPU/GPU split (csrc/cpu_phase.h), checked on the CPU alone:
a host-only harness runs every structure of every phase of a swept run through it
(as if the host threads took all tiles) and the result is compared with the oracle --
FP64 Euler bitwise, FP64 heat within 1e-12 (fused multiply-adds at fixed places), the
FP32 forms within the tolerances of their precision. The GPU tests check the same engine
against the GPU kernels bitwise (tests/test_gpu_hybrid.py)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1811_08282_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    oracle.build()
    out = str(tmp_path_factory.mktemp("host_engine") / "host_engine_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(ROOT, "paper_1811_08282_gb300", "csrc"), os.path.join(HERE, "host_engine_check.cu"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(harness, tmp_path, scheme, prec, x, W, periodic, steps, prm, gamma=1.4):
    fin, fout = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    np.ascontiguousarray(x, dtype=np.float64).tofile(fin)
    n = x.shape[-1]
    subprocess.run([harness, str(scheme), str(prec), str(n), str(W), str(int(periodic)), str(steps), repr(prm),
                    repr(gamma), fin, fout], check=True)
    return np.fromfile(fout).reshape(x.shape)


HEAT = [(256, 32, 37, True), (256, 32, 40, False), (1024, 128, 300, True), (1000, 40, 77, False), (96, 8, 23, False)]


@pytest.mark.parametrize("n,W,steps,periodic", HEAT)
def test_heat_fp64_matches_oracle(harness, tmp_path, n, W, steps, periodic):
    x = I.heat_initial(I.heat_modes(n, 8, seed=n))[None]
    got = _run(harness, tmp_path, 0, 0, x, W, periodic, steps, 0.3)
    want = oracle.heat_run(x[0], 0.3, steps, oracle.PERIODIC if periodic else oracle.TRANSMISSIVE)[None]
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (2, 1e-8)])  # hi/lo: increments are rounded in FP32
def test_heat_fp32_forms_within_precision(harness, tmp_path, prec, tol):
    n, W, steps = 1024, 64, 200
    x = I.heat_initial(I.heat_modes(n, 8, seed=3))[None]
    got = _run(harness, tmp_path, 0, prec, x, W, True, steps, 0.3)
    want = oracle.heat_run(x[0], 0.3, steps, oracle.PERIODIC)[None]
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol


EULER = [(256, 32, 9, False), (512, 64, 30, True), (1024, 128, 70, False), (960, 96, 33, True), (64, 8, 5, False)]


@pytest.mark.parametrize("n,W,steps,periodic", EULER)
def test_euler_fp64_equals_oracle_bitwise(harness, tmp_path, n, W, steps, periodic):
    x = I.riemann_initial(I.riemann_segments(n, max(2, n // 128), 3))
    got = _run(harness, tmp_path, 1, 0, x, W, periodic, steps, 0.08)
    want = oracle.euler_run(x, 0.08, 1.4, steps, oracle.PERIODIC if periodic else oracle.TRANSMISSIVE)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("prec", [1, 2])
def test_euler_fp32_forms_close_to_oracle(harness, tmp_path, prec):
    n, W, steps = 1024, 64, 50
    x = I.sod(n)
    got = _run(harness, tmp_path, 1, prec, x, W, False, steps, I.sod_lambda())
    want = oracle.euler_run(x, I.sod_lambda(), 1.4, steps, oracle.TRANSMISSIVE)
    assert np.all(np.isfinite(got)) and np.all(got[0] > 0)
    assert np.mean(np.abs(got - want)) < 1e-3
