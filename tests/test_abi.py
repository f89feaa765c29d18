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
    assert ctypes.sizeof(_abi.rsim_server_opts) == 16
    assert ctypes.sizeof(_abi.rsim_request) == 80 + 64 + 8 + 8
    assert ctypes.sizeof(_abi.rsim_server_stats) == 4 * 8 + 6 * 8 + 8 + 8


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
