"""The integer-pipe FP64 heat update (csrc/fp64_soft.cuh), checked on the CPU.

The FP64 swept and per-step heat kernels evaluate half their cells with integer
arithmetic that must reproduce fma(r, fma(-2, u, a + b), u) bit for bit (Section
4.2's update, each operation rounded to nearest even as IEEE 754 defines it). A
host-compiled harness (tests/fp64_soft_check.cu) runs the same source against the
host's own IEEE binary64 arithmetic over families of inputs chosen to reach every
branch: neighbours at all relative scales, the edges of the exponent window, exact
ties in the last rounding, results leaving u's binade, multipliers with few
significant bits, special values, and a whole heat run. Every accepted case must
match; the fallback share is bounded so that the fast path is actually exercised.
The GPU tests then check the kernels that use it bitwise against the FP64-only
per-step path and the oracle.

The 2D heat kernels' five-point update has its own integer-pipe form (two second
differences in u's frame, then two rounded corrections, the inner one kept inside
u's binade); tests/fp64_soft2d_check.cu checks it the same way against
fma(rx, fma(-2, u, a + b), fma(ry, fma(-2, u, d + e), u)), with ties placed in
either rounding and in the outer one after an exact inner correction of either
parity."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _build(tmp_path_factory, name):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp(name) / name)
    cmd = [nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
           "-I" + os.path.join(ROOT, "paper_1811_08282_gb300", "csrc"), os.path.join(HERE, name + ".cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    return _build(tmp_path_factory, "fp64_soft_check")


@pytest.fixture(scope="module")
def harness2d(tmp_path_factory):
    return _build(tmp_path_factory, "fp64_soft2d_check")


# family -> minimum share of cases on the integer path
MIN_FAST = {"smooth": 0.9, "window": 0.2, "ties": 0.9, "binade": 0.5, "r_bits": 0.8, "special": 0.01,
            "heat_run": 0.9}


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_path_matches_ieee_fp64(harness, seed):
    r = subprocess.run([harness, str(seed), "400000"], capture_output=True, text=True)
    rows = {}
    for line in r.stdout.splitlines():
        parts = line.split()
        if len(parts) == 4 and parts[0] in MIN_FAST:
            rows[parts[0]] = tuple(int(x) for x in parts[1:])
    assert r.returncode == 0, r.stdout
    assert set(rows) == set(MIN_FAST), r.stdout
    for name, (cases, fast, bad) in rows.items():
        assert bad == 0, (name, r.stdout)
        assert fast >= MIN_FAST[name] * cases, (name, cases, fast)


# 2D: family -> minimum share of cases on the integer path
MIN_FAST_2D = {"smooth": 0.8, "window": 0.15, "ties": 0.9, "binade": 0.4, "r_bits": 0.6, "special": 0.01,
               "heat_run": 0.99}


@pytest.mark.parametrize("seed", [1, 2])
def test_integer_path_2d_matches_ieee_fp64(harness2d, seed):
    r = subprocess.run([harness2d, str(seed), "400000"], capture_output=True, text=True)
    rows = {}
    for line in r.stdout.splitlines():
        parts = line.split()
        if len(parts) == 4 and parts[0] in MIN_FAST_2D:
            rows[parts[0]] = tuple(int(x) for x in parts[1:])
    assert r.returncode == 0, r.stdout
    assert set(rows) == set(MIN_FAST_2D), r.stdout
    for name, (cases, fast, bad) in rows.items():
        assert bad == 0, (name, r.stdout)
        assert fast >= MIN_FAST_2D[name] * cases, (name, cases, fast)
