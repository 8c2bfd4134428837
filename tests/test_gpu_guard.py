"""Guard words after the scratch buffers (out-of-bounds write detection): clean runs
leave them intact (every GPU test's sw_sync_status checks them), a byte changed from
the host through the test hook is reported once as SW_ERR_CORRUPT, then rewritten."""
import numpy as np
import pytest

from paper_1811_08282_gb300 import inputs as I
from paper_1811_08282_gb300 import swept as S
from tests.gpu_helpers import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("method,which", [(S.SW_SWEPT, 0), (S.SW_SWEPT, 1), (S.SW_PERSTEP, 2)])
def test_guard_damage_is_reported_once(method, which):
    import torch
    n = 4096
    p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=method, n=n, r=0.3,
                  tile_width=128 if method == S.SW_SWEPT else 0)
    st = S.to_state(p, torch.as_tensor(I.heat_initial(I.heat_modes(n, 4, seed=2)), device="cuda"))
    with S.Handle(p) as h:
        h.sw_run(st, 300)
        assert h.sw_sync_status() == S.SW_OK
        h.sw_debug_corrupt_guard(which)
        assert h.sw_sync_status() == S.SW_ERR_CORRUPT
        assert h.sw_sync_status() == S.SW_OK          # rewritten
        h.sw_run(st, 300)
        assert h.sw_sync_status() == S.SW_OK


def test_guard_hook_rejects_missing_buffers():
    import torch
    p = S.Problem(scheme=S.SW_HEAT, precision=S.SW_FP64, boundary=S.SW_PERIODIC, method=S.SW_PERSTEP, n=1024, r=0.3)
    with S.Handle(p) as h:
        with pytest.raises(S.SweptError):
            h.sw_debug_corrupt_guard(0)               # per-step handles have no flank buffers
        with pytest.raises(S.SweptError):
            h.sw_debug_corrupt_guard(3)
