"""Host arithmetic of the affinity split (Section 4.2, Eq. 1: WF = N_GPU / N_CPU in tiles)."""
import pytest

from paper_1811_08282_gb300 import swept as S


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from tests.gpu_helpers import ensure_lib
    ensure_lib()


@pytest.mark.parametrize("tiles,wf,threads", [(100, 10, 4), (131072, 60, 16), (2, 1, 1), (1000, 1, 999), (7, 3, 2)])
def test_split_follows_the_work_factor(tiles, wf, threads):
    g, per = S.sw_hybrid_split(tiles, wf, threads)
    assert per == tiles // (wf + threads) and per >= 1
    assert g + per * threads == tiles
    assert g >= wf * per                      # the GPU gets at least WF times a thread's share
    assert g - wf * per < wf + threads        # ... and the remainder of the division on top


@pytest.mark.parametrize("tiles,wf,threads", [(1, 1, 1), (10, 0, 2), (10, 2, 0), (10, 10, 1), (10, 1, 5000)])
def test_split_rejects(tiles, wf, threads):
    with pytest.raises(S.SweptError):
        S.sw_hybrid_split(tiles, wf, threads)
