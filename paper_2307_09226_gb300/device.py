"""Device-side helpers: move seeded synthetic frames into HBM as PyTorch tensors and
call the library through the binding.  PyTorch provides device memory and streams
only; every step of the synthesis runs in librsim's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import _abi
from .synth import Frame

FIELDS = ("range", "sigma_re", "sigma_im", "az", "el", "vel")


def upload(frame_or_pixels, device="cuda", pin=False):
    """Pixel SoA -> dict of contiguous device tensors (dtype preserved)."""
    px = frame_or_pixels.pixels if isinstance(frame_or_pixels, Frame) else frame_or_pixels
    out = {}
    for name, arr in zip(FIELDS, px.arrays()):
        t = torch.from_numpy(np.ascontiguousarray(arr))
        if pin:
            t = t.pin_memory()
        out[name] = t.to(device, non_blocking=pin)
    return out


def cube_tensor(radar, out_dtype="complex64", device="cuda"):
    dt = torch.complex128 if out_dtype == "complex128" else torch.complex64
    return torch.empty((radar.V, radar.Ns, radar.L), dtype=dt, device=device)


class Context:
    """Owns an rsim_ctx on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.h = _abi.rsim_create(device, hbm_budget_bytes)

    def close(self):
        if self.h is not None:
            _abi.rsim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synth(self, radar, pixels, tier="fp32", cube=None, out_dtype="complex64", stream=None):
        t = _abi.TIERS[tier] if isinstance(tier, str) else int(tier)
        if cube is None:
            cube = cube_tensor(radar, out_dtype)
        _abi.rsim_synth(self.h, radar, pixels, t, cube, stream)
        return cube

    def synth_host(self, radar, pixels, tier="fp32", cube=None, out_dtype="complex64", stream=None):
        """synth on host tensors: the library copies the pixels in and the cube out on
        `stream`; the cube is complete after a synchronisation."""
        t = _abi.TIERS[tier] if isinstance(tier, str) else int(tier)
        if cube is None:
            cube = cube_tensor(radar, out_dtype, device="cpu").pin_memory()
        _abi.rsim_synth_host(self.h, radar, pixels, t, cube, stream)
        return cube

    def synth_batch(self, radar, frames, tier="fp32", cubes=None, out_dtype="complex64", stream=None):
        t = _abi.TIERS[tier] if isinstance(tier, str) else int(tier)
        if cubes is None:
            cubes = [cube_tensor(radar, out_dtype) for _ in frames]
        _abi.rsim_synth_batch(self.h, radar, frames, t, cubes, stream)
        return cubes

    def raycast(self, scene, n_az, n_el, fov, dtype=torch.float32, falloff=True, out=None, stream=None):
        """Render an analytic scene into per-pixel buffers (dict of six device tensors,
        the input of synth)."""
        P = int(n_az) * int(n_el)
        if out is None:
            out = {k: torch.empty(P, dtype=dtype, device="cuda") for k in FIELDS}
        _abi.rsim_raycast(self.h, scene, n_az, n_el, fov, out, falloff, stream)
        return out

    def valid_indices(self, pixels, stream=None):
        P = int(pixels["range"].numel())
        idx = torch.full((max(P, 1),), -1, dtype=torch.int32, device="cuda")
        pv = torch.zeros(1, dtype=torch.int64, device="cuda")
        _abi.rsim_valid_indices(self.h, pixels, idx, pv, stream)
        n = int(pv.item())
        return idx[:n]

    def path_phases(self, radar, pixels, stream=None):
        P = int(pixels["range"].numel())
        V = radar.V
        a = torch.zeros(max(V * P, 1), dtype=torch.int32, device="cuda")
        c = torch.zeros(max(V * P, 1), dtype=torch.int32, device="cuda")
        b = torch.zeros(max(P, 1), dtype=torch.int32, device="cuda")
        s = torch.zeros(max(2 * P, 2), dtype=torch.float32, device="cuda")
        pv = torch.zeros(1, dtype=torch.int64, device="cuda")
        _abi.rsim_path_phases(self.h, radar, pixels, a, c, b, s, pv, stream)
        n = int(pv.item())
        u32 = lambda t: t.cpu().numpy().view(np.uint32)
        return dict(P_valid=n, a=u32(a)[: V * P].reshape(V, P)[:, :n] if P else u32(a)[:0],
                    c=u32(c)[: V * P].reshape(V, P)[:, :n] if P else u32(c)[:0],
                    b=u32(b)[:n], sigma=s.cpu().numpy()[: 2 * n].reshape(n, 2))

    def sync_status(self, stream=None) -> int:
        return _abi.rsim_sync_status(self.h, stream)

    def selftest_wait_timeout(self, limit_ns: int, stream=None) -> None:
        """Run the library's bounded device wait on a barrier nothing completes; the
        next sync_status() reports the timeout."""
        _abi.rsim_selftest_wait_timeout(self.h, limit_ns, stream)
