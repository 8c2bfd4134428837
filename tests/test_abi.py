"""The C-ABI library builds, loads and exports every symbol include/swept.h declares.

Runs without a GPU: only host-side entry points are called (argument validation,
layout queries, status strings). No compute call is made here.
"""
import ctypes
import os
import re

import pytest

from paper_1811_08282_gb300 import build
from paper_1811_08282_gb300 import swept as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "swept.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SW_API[^;(]*?\b(sw(?:2d)?_\w+)\s*\(", text, flags=re.S)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return S.load()


def test_header_and_binding_agree():
    assert _declared() == sorted(S.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_abi_version_and_status_strings(lib):
    assert S.sw_abi_version() == S.ABI_VERSION == 5
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert S.status_string(code) and S.status_string(code) != "unknown status"
    assert S.status_string(12345) == "unknown status"


@pytest.mark.parametrize("scheme,prec,planes,esize", [
    (S.SW_HEAT, S.SW_FP64, 1, 8), (S.SW_HEAT, S.SW_FP32, 1, 4), (S.SW_HEAT, S.SW_FP32_COMP, 2, 4),
    (S.SW_EULER, S.SW_FP64, 3, 8), (S.SW_EULER, S.SW_FP32, 3, 4), (S.SW_EULER, S.SW_FP32_COMP, 6, 4),
])
def test_state_layout(lib, scheme, prec, planes, esize):
    p = S.Problem(scheme=scheme, precision=prec, n=4096, r=0.3, dt_dx=0.1, tile_width=64)
    assert S.sw_state_planes(p) == planes
    assert S.sw_state_bytes(p) == planes * 4096 * esize


@pytest.mark.parametrize("bad", [
    dict(n=1000, tile_width=64),             # W does not divide n
    dict(n=4096, tile_width=63),             # odd W
    dict(n=4096, tile_width=2),              # W below the minimum
    dict(n=4096, tile_width=2048),           # W above the maximum
    dict(n=64, tile_width=64),               # fewer than two tiles
    dict(n=4096, r=0.0),                     # non-positive r
    dict(n=4096, r=float("nan")),
    dict(n=4096, scheme=7),
    dict(n=4096, precision=3),
    dict(n=4096, boundary=2),
    dict(n=4096, method=5),
    dict(n=4096, flags=32),                  # unknown flag bit
    dict(n=2),
    dict(n=4096, scheme=S.SW_EULER, dt_dx=0.0),
    dict(n=4096, scheme=S.SW_EULER, dt_dx=0.1, gamma=1.0),
    dict(n=600, scheme=S.SW_EULER, dt_dx=0.1, tile_width=6, flags=S.SW_FLAG_FLATTENED),   # flattened: W % 4
    dict(n=64, scheme=S.SW_EULER, dt_dx=0.1, tile_width=4, flags=S.SW_FLAG_FLATTENED),    # flattened: W >= 8
])
def test_bad_problems_are_rejected_before_any_device_work(lib, bad):
    kw = dict(n=4096, r=0.3, tile_width=64)
    kw.update(bad)
    p = S.Problem(**kw)
    with pytest.raises(S.SweptError) as ei:
        S.Handle(p)
    assert ei.value.code == S.SW_ERR_BAD_ARG
    assert S.sw_state_planes.__name__  # binding intact


def test_null_arguments_are_rejected(lib):
    assert lib.sw_run(None, None, 1, None) == S.SW_ERR_BAD_ARG
    assert lib.sw_create(None, None) == S.SW_ERR_BAD_ARG
    assert lib.sw_sync_status(None, None) == S.SW_ERR_BAD_ARG
    assert lib.sw_last_launch_count(None) == 0
    lib.sw_destroy(None)
