"""The launch-condition map of Section 5 (Table 1's power-law fit) and the data-structure
experiment of Section 4.3 (Fig. 3), run on the GPU over a tiny range: every point, best
and fit row is emitted with sane values, and the fit's R^2 is defined."""
import json
import math

import pytest

from paper_1811_08282_gb300 import launch_map as LM
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("scheme,precision", [("heat", S.SW_FP64), ("euler", S.SW_FP32)])
def test_map_rows_and_fit(scheme, precision):
    rows = []
    best, (A, b, r2) = LM.run_map(scheme, precision, range(14, 17), (128, 256), target=2.0 ** 22, cap=2048,
                                  reps=1, emit=lambda s: rows.append(json.loads(s)))
    points = [r for r in rows if r["kind"] == "point"]
    bests = [r for r in rows if r["kind"] == "best"]
    fits = [r for r in rows if r["kind"] == "fit"]
    # three grids: two widths swept plus the per-step kernel each
    assert len(points) == 3 * 3 and len(bests) == 3 and len(fits) == 1
    assert {r["n"] for r in points} == {1 << 14, 1 << 15, 1 << 16}
    for r in points:
        assert r["us_per_step"] > 0 and math.isfinite(r["gcell_steps_per_s"])
    for r in bests:
        assert r["W"] in (128, 256) and r["speedup"] > 0
    f = fits[0]
    assert f["A_us"] > 0 and math.isfinite(f["b"]) and math.isfinite(f["r2"]) and f["r2"] <= 1.0
    assert f["n_range"] == [1 << 14, 1 << 16]
    assert (A, b, r2) == (f["A_us"], f["b"], f["r2"])
    assert [n for n, _ in best] == [1 << 14, 1 << 15, 1 << 16]


def test_forms_rows():
    rows = []
    LM.run_forms(S.SW_FP32, range(14, 16), (128, 256), target=2.0 ** 22, cap=1024, reps=1,
                 emit=lambda s: rows.append(json.loads(s)))
    assert len(rows) == 2
    for r in rows:
        assert r["kind"] == "forms"
        for k in ("swept_lengthened", "swept_flattened", "perstep_flattened", "perstep_lengthened"):
            assert r[k]["us_per_step"] > 0
        assert r["swept_flattened"]["W"] in (128, 256)
