"""Host-side checks of the C ABI: the library loads, exports every function that
include/rsim.h declares, and the ctypes structs match the C layouts.  No GPU needed;
no compute call is made."""
import ctypes
import os
import re

import pytest

from paper_2307_09226_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsim.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_abi.LIB_PATH):
        from paper_2307_09226_gb300 import build
        build.build()
    return _abi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsim_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
        assert n in _abi.SIGNATURES, f"binding misses {n}"
    assert set(_abi.SIGNATURES) == set(names)


def test_version_and_last_error_are_host_only(lib):
    assert "sm_103a" in _abi.rsim_version()
    assert isinstance(_abi.last_error(), str)


def test_struct_layouts_match_header():
    # rsim_radar_params: 4 int32 + 7 double + flags + reserved
    assert ctypes.sizeof(_abi.rsim_radar_params) == 16 + 7 * 8 + 8
    assert _abi.rsim_radar_params.flags.offset == 72
    assert _abi.rsim_radar_params.lambda_.offset == 16
    # rsim_pixels: int64 + 2 int32 + 6 pointers
    assert ctypes.sizeof(_abi.rsim_pixels) == 16 + 6 * 8
    assert _abi.rsim_pixels.range.offset == 16
    assert ctypes.sizeof(_abi.rsim_plan) == 32
    assert ctypes.sizeof(_abi.rsim_profile) == 8 + 5 * 8
    assert ctypes.sizeof(_abi.rsim_primitive) == 8 + 6 * 24 + 8
    assert _abi.PRIM_DTYPE.itemsize == ctypes.sizeof(_abi.rsim_primitive)
    for name, _ in _abi.rsim_primitive._fields_:
        assert _abi.PRIM_DTYPE.fields[name][1] == getattr(_abi.rsim_primitive, name).offset
    assert ctypes.sizeof(_abi.rsim_camera) == 8 + 4 * 8 + 8
    assert ctypes.sizeof(_abi.rsim_pixel_out) == ctypes.sizeof(_abi.rsim_pixels)
    assert ctypes.sizeof(_abi.rsim_server_opts) == 32
    assert ctypes.sizeof(_abi.rsim_request) == 80 + 64 + 8 + 8
    assert ctypes.sizeof(_abi.rsim_server_stats) == 4 * 8 + 6 * 8 + 8 + 8 + 3 * 8


def test_null_context_is_rejected_without_touching_a_device(lib):
    assert lib.rsim_sync_status(None, None) == _abi.ERR_INVALID_ARG
    assert lib.rsim_selftest_wait_timeout(None, 1000000, None) == _abi.ERR_INVALID_ARG
    assert lib.rsim_synth_host(None, None, None, 0, None, 0, None) == _abi.ERR_INVALID_ARG
    assert lib.rsim_server_stats_reset(None) == _abi.ERR_INVALID_ARG
    assert lib.rsim_destroy(None) == _abi.OK
    out = ctypes.c_size_t()
    p = _abi.rsim_radar_params(2, 4, 64, 32, 3.9e-3, 0, 3e13, 1e7, 6e-5, 0, 0)
    assert lib.rsim_workspace_size(None, ctypes.byref(p), 100, 0, ctypes.byref(out)) == _abi.ERR_INVALID_ARG
    assert "NULL" in _abi.last_error()


def test_build_entry_compiles_for_sm103a():
    src = open(os.path.join(ROOT, "paper_2307_09226_gb300", "build.py")).read()
    assert "arch=compute_103a,code=sm_103a" in src


def test_plans_are_checked_on_the_host(lib):
    """rsim_set_plan checks the plan before it needs a context: a variant other than 0, a
    column tile that is not a multiple of 8 or wider than the cube, and an accumulation
    group beyond the split tiers' accuracy cap are refused."""
    p = _abi.rsim_radar_params(2, 4, 64, 32, 3.9e-3, 0, 3e13, 1e7, 6e-5, 0, 0)
    bad = [
        (_abi.TIER_SPLIT_FP16, _abi.rsim_plan(2, 32, 0, 2, 0, 0, 0, 0), "variant"),
        (_abi.TIER_SPLIT_FP16, _abi.rsim_plan(2, 32, 0, 0, 0, 12, 0, 0), "tile_n"),
        (_abi.TIER_SPLIT_FP16, _abi.rsim_plan(2, 32, 0, 0, 0, 40, 0, 0), "tile_n"),  # L = 32
        (_abi.TIER_SPLIT_BF16, _abi.rsim_plan(2, 32, 0, 0, 0, 0, 41, 0), "group_chunks"),
        (_abi.TIER_BF16, _abi.rsim_plan(2, 32, 0, 0, 0, 0, 385, 0), "group_chunks"),
        (_abi.TIER_FP32, _abi.rsim_plan(2, 32, 0, 0, 0, 96, 0, 0), "tile_n"),
        (_abi.TIER_FP32, _abi.rsim_plan(0, 32, 0, 0, 0, 0, 0, 0), "splits"),
    ]
    for tier, plan, word in bad:
        assert lib.rsim_set_plan(None, ctypes.byref(p), 2048, tier, ctypes.byref(plan)) == _abi.ERR_INVALID_ARG
        assert word in _abi.last_error(), (word, _abi.last_error())
    # a valid plan gets as far as the missing context
    ok = _abi.rsim_plan(2, 32, 0, 0, 0, 32, 40, 0)
    assert lib.rsim_set_plan(None, ctypes.byref(p), 2048, _abi.TIER_SPLIT_FP16, ctypes.byref(ok)) == _abi.ERR_INVALID_ARG
    assert "ctx" in _abi.last_error()


def test_no_cluster_multicast_load_in_the_library():
    """Every CTA loads its own operands: no bulk or tensor load with cluster multicast."""
    csrc = os.path.join(ROOT, "paper_2307_09226_gb300", "csrc")
    for name in os.listdir(csrc):
        text = open(os.path.join(csrc, name)).read()
        assert "multicast" not in text, name
