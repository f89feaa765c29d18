"""ctypes binding of librsim (include/rsim.h): same names, argument marshalling only.

Tensors are PyTorch device tensors; their data pointers and the current CUDA stream
are passed through unchanged.  Every function raises ``RsimError`` on a non-OK status.
There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t,
                    c_uint64, c_void_p)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "librsim.so")

OK, ERR_INVALID_ARG, ERR_NONFINITE, ERR_OVERFLOW, ERR_OOM, ERR_BUDGET, ERR_TIMEOUT, \
    ERR_CANCELLED, ERR_CUDA, ERR_UNSUPPORTED, ERR_NOT_FOUND = range(11)
STATUS_NAMES = ["OK", "INVALID_ARG", "NONFINITE", "OVERFLOW", "OOM", "BUDGET", "TIMEOUT",
                "CANCELLED", "CUDA", "UNSUPPORTED", "NOT_FOUND"]
TIER_FP32, TIER_BF16, TIER_SPLIT_BF16, TIER_SPLIT_FP16, TIER_FP16, TIER_NUFFT = range(6)
TIERS = {"fp32": TIER_FP32, "bf16": TIER_BF16, "split_bf16": TIER_SPLIT_BF16,
         "split_fp16": TIER_SPLIT_FP16, "fp16": TIER_FP16, "nufft": TIER_NUFFT}
F32, F64 = 0, 1
FLAG_TDM_MOTION = 1
C64, C128 = 0, 1


class RsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rsim status {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class rsim_radar_params(Structure):
    _fields_ = [("M", c_int32), ("N", c_int32), ("Ns", c_int32), ("L", c_int32),
                ("lambda_", c_double), ("d_rx", c_double), ("mu", c_double), ("fs", c_double),
                ("t_b", c_double), ("t_slow", c_double), ("c", c_double),
                ("flags", c_int32), ("reserved", c_int32)]


class rsim_pixels(Structure):
    _fields_ = [("P", c_int64), ("dtype", c_int32), ("reserved", c_int32),
                ("range", c_void_p), ("sigma_re", c_void_p), ("sigma_im", c_void_p),
                ("az", c_void_p), ("el", c_void_p), ("vel", c_void_p)]


class rsim_primitive(Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("a", c_double * 3), ("b", c_double * 3),
                ("c", c_double * 3), ("d", c_double * 3), ("vel", c_double * 3), ("omega", c_double * 3),
                ("rho", c_double)]


class rsim_camera(Structure):
    _fields_ = [("n_az", c_int32), ("n_el", c_int32), ("az_min", c_double), ("az_max", c_double),
                ("el_min", c_double), ("el_max", c_double), ("flags", c_int32), ("reserved", c_int32)]


class rsim_pixel_out(Structure):
    _fields_ = [("P", c_int64), ("dtype", c_int32), ("reserved", c_int32),
                ("range", c_void_p), ("sigma_re", c_void_p), ("sigma_im", c_void_p),
                ("az", c_void_p), ("el", c_void_p), ("vel", c_void_p)]


PRIM_KINDS = {"plane": 0, "capsule": 1, "ellipsoid": 2}


def _prim_dtype():
    import numpy as np
    return np.dtype([("kind", "<i4"), ("reserved", "<i4"), ("a", "<f8", (3,)), ("b", "<f8", (3,)),
                     ("c", "<f8", (3,)), ("d", "<f8", (3,)), ("vel", "<f8", (3,)), ("omega", "<f8", (3,)),
                     ("rho", "<f8")])


PRIM_DTYPE = _prim_dtype()
RC_NO_FALLOFF = 1


class rsim_plan(Structure):
    _fields_ = [("splits", c_int32), ("chunk_px", c_int32), ("grid", c_int32),
                ("variant", c_int32), ("tuned", c_int32), ("tile_n", c_int32),
                ("group_chunks", c_int32), ("reserved", c_int32)]

    def as_dict(self) -> dict:
        return {"splits": self.splits, "grid": self.grid, "tile_n": self.tile_n,
                "group_chunks": self.group_chunks, "tuned": bool(self.tuned)}


SERVE_FIRST_FIT, SERVE_SHORTEST_FIRST = 0, 1
SERVE_POLICIES = {"first_fit": SERVE_FIRST_FIT, "shortest_first": SERVE_SHORTEST_FIRST}


class rsim_server_opts(Structure):
    _fields_ = [("slots", c_int32), ("max_queue", c_int32), ("hbm_budget_bytes", c_size_t),
                ("policy", c_int32), ("age_limit_ms", c_int32), ("express_slots", c_int32),
                ("reserved", c_int32)]


class rsim_request(Structure):
    _fields_ = [("params", rsim_radar_params), ("pixels", rsim_pixels), ("tier", c_int32),
                ("out_dtype", c_int32), ("cube", c_void_p)]


class rsim_server_stats(Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("cancelled", c_uint64),
                ("failed", c_uint64), ("p50_ms", c_double), ("p99_ms", c_double),
                ("mean_ms", c_double), ("max_ms", c_double), ("busy_s", c_double),
                ("path_samples", c_double), ("peak_reserved_bytes", c_size_t),
                ("peak_in_flight", c_int32), ("reserved", c_int32), ("p99_queue_ms", c_double),
                ("max_queue_ms", c_double), ("overtakes", c_uint64)]


class rsim_profile(Structure):
    _fields_ = [("calls", c_int32), ("kernels", c_int32), ("prep_ms", c_double),
                ("contract_ms", c_double), ("reduce_ms", c_double), ("operand_ms", c_double),
                ("main_ms", c_double)]


# name -> (restype, argtypes); the full exported surface of include/rsim.h
SIGNATURES = {
    "rsim_version": (c_char_p, []),
    "rsim_last_error": (c_char_p, []),
    "rsim_create": (c_int, [POINTER(c_void_p), c_int, c_size_t]),
    "rsim_destroy": (c_int, [c_void_p]),
    "rsim_workspace_size": (c_int, [c_void_p, POINTER(rsim_radar_params), c_int64, c_int,
                                    POINTER(c_size_t)]),
    "rsim_synth": (c_int, [c_void_p, POINTER(rsim_radar_params), POINTER(rsim_pixels), c_int,
                           c_void_p, c_int32, c_void_p]),
    "rsim_synth_host": (c_int, [c_void_p, POINTER(rsim_radar_params), POINTER(rsim_pixels), c_int,
                           c_void_p, c_int32, c_void_p]),
    "rsim_synth_batch": (c_int, [c_void_p, POINTER(rsim_radar_params), POINTER(rsim_pixels),
                                 c_int32, POINTER(c_void_p), c_int, c_int32, c_void_p]),
    "rsim_synth_static": (c_int, [POINTER(rsim_radar_params), POINTER(rsim_pixels), c_int, c_void_p,
                                  c_int32, c_void_p, c_void_p]),
    "rsim_valid_indices": (c_int, [c_void_p, POINTER(rsim_pixels), c_void_p, c_void_p, c_void_p]),
    "rsim_path_phases": (c_int, [c_void_p, POINTER(rsim_radar_params), POINTER(rsim_pixels),
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "rsim_range_doppler": (c_int, [c_void_p, POINTER(rsim_radar_params), POINTER(c_void_p), c_int32,
                                   c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "rsim_sync_status": (c_int, [c_void_p, c_void_p]),
    "rsim_selftest_wait_timeout": (c_int, [c_void_p, c_uint64, c_void_p]),
    "rsim_measure_smem_atomics": (c_int, [c_void_p, POINTER(c_double), c_void_p]),
    "rsim_measure_mma_rate": (c_int, [c_void_p, POINTER(c_double), c_void_p]),
    "rsim_autotune": (c_int, [c_void_p, POINTER(rsim_radar_params), c_int64, c_int,
                              POINTER(rsim_plan), c_void_p]),
    "rsim_raycast": (c_int, [c_void_p, POINTER(rsim_camera), POINTER(rsim_primitive), c_int32,
                             POINTER(rsim_pixel_out), c_void_p]),
    "rsim_profile_enable": (c_int, [c_void_p, c_int32]),
    "rsim_profile_read": (c_int, [c_void_p, POINTER(rsim_profile)]),
    "rsim_set_plan": (c_int, [c_void_p, POINTER(rsim_radar_params), c_int64, c_int,
                              POINTER(rsim_plan)]),
    "rsim_get_plan": (c_int, [c_void_p, POINTER(rsim_radar_params), c_int64, c_int,
                              POINTER(rsim_plan)]),
    "rsim_server_create": (c_int, [c_void_p, POINTER(rsim_server_opts), POINTER(c_void_p)]),
    "rsim_server_submit": (c_int, [c_void_p, POINTER(rsim_request), POINTER(c_uint64)]),
    "rsim_server_wait": (c_int, [c_void_p, c_uint64, c_int32]),
    "rsim_server_cancel": (c_int, [c_void_p, c_uint64]),
    "rsim_server_stats_get": (c_int, [c_void_p, POINTER(rsim_server_stats)]),
    "rsim_server_stats_reset": (c_int, [c_void_p]),
    "rsim_server_destroy": (c_int, [c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librsim.so (built by ``build.build()``) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librsim.so is not built ({path}); run paper_2307_09226_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().rsim_last_error().decode()


def check(status: int):
    if status != OK:
        raise RsimError(status, last_error())
    return status


def radar_params(radar) -> rsim_radar_params:
    """Marshal a ``synth.Radar`` (or anything with the same attributes)."""
    flags = FLAG_TDM_MOTION if getattr(radar, "tdm_motion", False) else 0
    flags |= (int(getattr(radar, "nufft_width", 0)) & 0xF) << 8
    return rsim_radar_params(int(radar.M), int(radar.N), int(radar.Ns), int(radar.L),
                             float(radar.lam), float(radar.d_rx), float(radar.mu), float(radar.fs),
                             float(radar.t_b), float(radar.t_slow), float(radar.c), flags, 0)


def pixels_struct(t) -> rsim_pixels:
    """Marshal a dict/tuple of six equal-length contiguous device tensors
    (range, sigma_re, sigma_im, az, el, vel) of float32 or float64."""
    import torch
    arrs = [t[k] for k in ("range", "sigma_re", "sigma_im", "az", "el", "vel")] if isinstance(t, dict) else list(t)
    P = int(arrs[0].numel())
    dt = arrs[0].dtype
    for a in arrs:
        if a.dtype != dt or a.numel() != P or not a.is_contiguous():
            raise ValueError("pixel arrays must be contiguous and share dtype and length")
    if dt == torch.float32:
        code = F32
    elif dt == torch.float64:
        code = F64
    else:
        raise ValueError("pixel arrays must be float32 or float64")
    return rsim_pixels(P, code, 0, *[a.data_ptr() for a in arrs])


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _ptr(x):
    return None if x is None else c_void_p(x.data_ptr())


# ---------------------------------------------------------------------------------
# Thin wrappers with the C names.
# ---------------------------------------------------------------------------------

def rsim_version() -> str:
    return load().rsim_version().decode()


def rsim_create(device: int = 0, hbm_budget_bytes: int = 0) -> c_void_p:
    h = c_void_p()
    check(load().rsim_create(ctypes.byref(h), int(device), int(hbm_budget_bytes)))
    return h


def rsim_destroy(ctx):
    check(load().rsim_destroy(ctx))


def rsim_workspace_size(ctx, radar, P: int, tier: int) -> int:
    out = c_size_t()
    check(load().rsim_workspace_size(ctx, ctypes.byref(radar_params(radar)), int(P), int(tier),
                                     ctypes.byref(out)))
    return int(out.value)


def rsim_synth(ctx, radar, pixels, tier: int, cube, stream=None):
    """cube: complex64 or complex128 device tensor of shape [M*N, Ns, L]."""
    import torch
    od = C128 if cube.dtype == torch.complex128 else C64
    if cube.dtype not in (torch.complex64, torch.complex128) or not cube.is_contiguous():
        raise ValueError("cube must be a contiguous complex64/complex128 tensor")
    px = pixels if isinstance(pixels, rsim_pixels) else pixels_struct(pixels)
    check(load().rsim_synth(ctx, ctypes.byref(radar_params(radar)), ctypes.byref(px), int(tier),
                            _ptr(cube), od, _stream(stream)))


def rsim_synth_host(ctx, radar, pixels, tier: int, cube, stream=None):
    """pixels: six equal-length contiguous HOST tensors (page-locked for asynchronous
    copies); cube: contiguous complex64/complex128 HOST tensor [M*N, Ns, L]."""
    import torch
    if cube.device.type != "cpu" or any(pixels[k].device.type != "cpu" for k in pixels):
        raise ValueError("rsim_synth_host takes host tensors")
    od = C128 if cube.dtype == torch.complex128 else C64
    if cube.dtype not in (torch.complex64, torch.complex128) or not cube.is_contiguous():
        raise ValueError("cube must be a contiguous complex64/complex128 tensor")
    check(load().rsim_synth_host(ctx, ctypes.byref(radar_params(radar)), ctypes.byref(pixels_struct(pixels)),
                                 int(tier), _ptr(cube), od, _stream(stream)))


def rsim_synth_batch(ctx, radar, frames, tier: int, cubes, stream=None):
    import torch
    F = len(frames)
    arr = (rsim_pixels * F)(*[f if isinstance(f, rsim_pixels) else pixels_struct(f) for f in frames])
    ptrs = (c_void_p * F)(*[c.data_ptr() for c in cubes])
    od = C128 if cubes[0].dtype == torch.complex128 else C64
    check(load().rsim_synth_batch(ctx, ctypes.byref(radar_params(radar)), arr, F, ptrs, int(tier), od,
                                  _stream(stream)))


def rsim_synth_static(radar, pixels, tier: int, cube, device_status=None, stream=None):
    """Synthesis through the allocation-free entry point (scratch compiled into the
    library; no context).  Returns the raw status code (does not raise)."""
    import torch
    od = C128 if cube.dtype == torch.complex128 else C64
    px = pixels if isinstance(pixels, rsim_pixels) else pixels_struct(pixels)
    return int(load().rsim_synth_static(ctypes.byref(radar_params(radar)), ctypes.byref(px), int(tier),
                                        _ptr(cube), od, _ptr(device_status), _stream(stream)))


def rsim_valid_indices(ctx, pixels, idx, p_valid, stream=None):
    px = pixels if isinstance(pixels, rsim_pixels) else pixels_struct(pixels)
    check(load().rsim_valid_indices(ctx, ctypes.byref(px), _ptr(idx), _ptr(p_valid), _stream(stream)))


def rsim_path_phases(ctx, radar, pixels, a, cph, b, sigma, p_valid, stream=None):
    px = pixels if isinstance(pixels, rsim_pixels) else pixels_struct(pixels)
    check(load().rsim_path_phases(ctx, ctypes.byref(radar_params(radar)), ctypes.byref(px), _ptr(a),
                                  _ptr(cph), _ptr(b), _ptr(sigma), _ptr(p_valid), _stream(stream)))


RD_SKIP_STATIC = 1


def rsim_range_doppler(ctx, radar, cubes, power, v_est, peak=None, skip_static=False, stream=None):
    """cubes: list of complex64 device tensors [V, Ns, L]; power: float32 [F, Ns, L];
    v_est: float32 [F]; peak: int32 [F, 2] or None."""
    F = len(cubes)
    ptrs = (c_void_p * F)(*[c.data_ptr() for c in cubes])
    check(load().rsim_range_doppler(ctx, ctypes.byref(radar_params(radar)), ptrs, F, _ptr(power),
                                    _ptr(v_est), _ptr(peak), RD_SKIP_STATIC if skip_static else 0,
                                    _stream(stream)))


def rsim_sync_status(ctx, stream=None) -> int:
    """Returns the status code (does not raise) so callers can test for NONFINITE."""
    return int(load().rsim_sync_status(ctx, _stream(stream)))


def rsim_selftest_wait_timeout(ctx, limit_ns: int, stream=None) -> None:
    check(load().rsim_selftest_wait_timeout(ctx, int(limit_ns), _stream(stream)))


def rsim_autotune(ctx, radar, P: int, tier: int, stream=None) -> rsim_plan:
    plan = rsim_plan()
    check(load().rsim_autotune(ctx, ctypes.byref(radar_params(radar)), int(P), int(tier),
                               ctypes.byref(plan), _stream(stream)))
    return plan


def primitives_array(scene):
    """A scene (list of primitive dicts with kind, a, b, c, d, vel, omega, rho) as a numpy
    structured array laid out like rsim_primitive (an array passes through unchanged)."""
    import numpy as np
    if isinstance(scene, np.ndarray) and scene.dtype == PRIM_DTYPE:
        return np.ascontiguousarray(scene)
    arr = np.zeros(len(scene), dtype=PRIM_DTYPE)
    if len(scene):
        arr["kind"] = [PRIM_KINDS[p["kind"]] for p in scene]
        for f in ("a", "b", "c", "d", "vel", "omega"):
            arr[f] = [p[f] for p in scene]
        arr["rho"] = [p["rho"] for p in scene]
    return arr


def rsim_raycast(ctx, scene, n_az, n_el, fov, out, falloff=True, stream=None):
    """Render `scene` into the six device tensors of `out` (dict, float32 or float64,
    n_az * n_el elements each)."""
    (az0, az1), (el0, el1) = fov
    cam = rsim_camera(int(n_az), int(n_el), float(az0), float(az1), float(el0), float(el1),
                      0 if falloff else RC_NO_FALLOFF, 0)
    px = pixels_struct(out)
    po = rsim_pixel_out(px.P, px.dtype, 0, px.range, px.sigma_re, px.sigma_im, px.az, px.el, px.vel)
    arr = primitives_array(scene)
    ptr = arr.ctypes.data_as(POINTER(rsim_primitive)) if arr.size else None
    check(load().rsim_raycast(ctx, ctypes.byref(cam), ptr, int(arr.size), ctypes.byref(po), _stream(stream)))


def rsim_profile_enable(ctx, on: bool):
    check(load().rsim_profile_enable(ctx, 1 if on else 0))


def rsim_measure_smem_atomics(ctx, stream=None) -> float:
    """Measured shared-memory atomic rate of the device (lane operations per second)."""
    v = c_double()
    check(load().rsim_measure_smem_atomics(ctx, ctypes.byref(v), _stream(stream)))
    return v.value


def rsim_measure_mma_rate(ctx, stream=None) -> float:
    """Measured flop rate of the contraction's tensor-core instruction on the device."""
    v = c_double()
    check(load().rsim_measure_mma_rate(ctx, ctypes.byref(v), _stream(stream)))
    return v.value


def rsim_profile_read(ctx) -> rsim_profile:
    p = rsim_profile()
    check(load().rsim_profile_read(ctx, ctypes.byref(p)))
    return p


def rsim_set_plan(ctx, radar, P: int, tier: int, splits: int, grid: int = 0, tile_n: int = 0,
                  group_chunks: int = 0, variant: int = 0):
    plan = rsim_plan(int(splits), 32, int(grid), int(variant), 0, int(tile_n), int(group_chunks), 0)
    check(load().rsim_set_plan(ctx, ctypes.byref(radar_params(radar)), int(P), int(tier),
                               ctypes.byref(plan)))


def rsim_get_plan(ctx, radar, P: int, tier: int) -> rsim_plan:
    plan = rsim_plan()
    check(load().rsim_get_plan(ctx, ctypes.byref(radar_params(radar)), int(P), int(tier),
                               ctypes.byref(plan)))
    return plan


def rsim_server_create(ctx, slots=4, max_queue=4096, hbm_budget_bytes=0, policy="first_fit",
                       age_limit_ms=0, express_slots=0) -> c_void_p:
    h = c_void_p()
    opts = rsim_server_opts(int(slots), int(max_queue), int(hbm_budget_bytes), SERVE_POLICIES[policy],
                            int(age_limit_ms), int(express_slots), 0)
    check(load().rsim_server_create(ctx, ctypes.byref(opts), ctypes.byref(h)))
    return h


def make_request(radar, pixels, tier, cube) -> rsim_request:
    import torch
    px = pixels if isinstance(pixels, rsim_pixels) else pixels_struct(pixels)
    od = C128 if cube.dtype == torch.complex128 else C64
    return rsim_request(radar_params(radar), px, int(tier), od, c_void_p(cube.data_ptr()))


def rsim_server_submit(server, req: rsim_request) -> int:
    t = c_uint64()
    check(load().rsim_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


def rsim_server_wait(server, ticket: int, timeout_ms: int = -1) -> int:
    """Returns the request's status code (does not raise)."""
    return int(load().rsim_server_wait(server, c_uint64(ticket), int(timeout_ms)))


def rsim_server_cancel(server, ticket: int) -> int:
    return int(load().rsim_server_cancel(server, c_uint64(ticket)))


def rsim_server_stats_get(server) -> rsim_server_stats:
    s = rsim_server_stats()
    check(load().rsim_server_stats_get(server, ctypes.byref(s)))
    return s


def rsim_server_stats_reset(server):
    check(load().rsim_server_stats_reset(server))


def rsim_server_destroy(server):
    check(load().rsim_server_destroy(server))
