"""Where the FP32 error of the Euler scheme comes from (CPU, no GPU): a small harness
(tests/euler_precision_probe.cpp, its own restatement of the scheme, sharing no code with
the library or the oracle) runs the Sod tube and periodic random Riemann problems with
single steps moved between FP32 and FP64 and compares each with the FP64 run:

- the scheme itself is sensitive: FP64 with one ulp added to every seventh energy value
  moves by ~1e-3 (max) -- the floor for any result that is not bitwise the FP64 one;
- FP32 and the FP32 hi/lo state (pressure, ratio and flux from the high parts, the
  library's FP32_COMP) err ~10x above that floor, and alike: an exact state update gains
  nothing when every step's pressure ratio and flux are evaluated in FP32;
- the hi/lo state with the flux in FP64 but the pressure ratio in FP32 still errs as FP32;
- the hi/lo state with every step in FP64 returns to the floor;
- density and pressure stay positive in every variant.
So the Euler error is set by the FP32 evaluation of the limiter's pressure differences and
of the fluxes, not by accumulation in the state; only FP64 evaluation of both removes it,
which costs what the FP64 form costs (the FP64 pipe binds either way).
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("probe") / "euler_precision_probe")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp",
                    os.path.join(HERE, "euler_precision_probe.cpp"), "-o", exe], check=True)
    return exe


def _run(exe, n, steps, kind):
    out = subprocess.run([exe, str(n), str(steps), str(kind)], check=True, capture_output=True, text=True).stdout
    rows = {}
    for line in out.strip().splitlines():
        name, mx, l2, minr, minp = line.split()
        rows[name] = (float(mx), float(l2), float(minr), float(minp))
    return rows


@pytest.mark.parametrize("n,steps,kind", [(4096, 2000, 0), (8192, 1500, 1)])
def test_error_is_set_by_fp32_evaluation_not_by_the_state(probe, n, steps, kind):
    r = _run(probe, n, steps, kind)
    floor = r["fp64_1ulp"][0]
    assert 1e-5 < floor < 5e-2                                        # the scheme amplifies one ulp
    assert r["fp32"][0] > 5 * floor and r["hilo"][0] > 5 * floor      # FP32 evaluation: far above
    assert 0.7 < r["hilo"][1] / r["fp32"][1] < 1.4                    # the exact state gains nothing
    assert 0.7 < r["hilo_flux64"][1] / r["hilo"][1] < 1.4             # nor does an FP64 flux alone
    assert r["hilo_all64"][0] < 3 * floor and r["hilo_all64"][1] < 3 * r["fp64_1ulp"][1]  # FP64 steps: the floor
    assert r["hilo_p64"][1] < r["hilo"][1]                            # an FP64 limiter alone: partway
    for name, (_, _, minr, minp) in r.items():
        assert minr > 0 and minp > 0, name
