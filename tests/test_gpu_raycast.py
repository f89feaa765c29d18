"""GPU parity of the analytic-scene ray-caster against the FP64 oracle, through the
C-ABI.  Pixels whose first hit is ambiguous (a silhouette or an occlusion edge within
the rounding of the pixel's ray) may differ; every such pixel must flip in the oracle
itself when its ray is turned by a tiny angle."""
import numpy as np
import pytest
import torch

import oracle.raycast as rc
from paper_2307_09226_gb300 import _abi, device, synth

pytestmark = pytest.mark.gpu

FOV = synth.CAMERA_FOV


@pytest.fixture(scope="module")
def ctx():
    c = device.Context(0)
    yield c
    c.close()


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def _ambiguous(scene, az, el, which, eps=2e-5):
    """Pixels whose oracle primitive changes when the ray turns by eps rad."""
    flip = np.zeros(az.size, dtype=bool)
    for da, de in ((eps, 0), (-eps, 0), (0, eps), (0, -eps)):
        o = rc.raycast_angles(scene, az + da, el + de)
        flip |= o["prim"] != which
    return flip


def _compare(scene, got, want, rtol_r, rtol_s, atol_v, max_ambiguous=0.01):
    R, Rw = got["range"].astype(np.float64), want["range"]
    hit_g, hit_w = np.isfinite(R), np.isfinite(Rw)
    both = hit_w & hit_g
    close_r = hit_g == hit_w  # a miss (inf) must be a miss on both sides ...
    close_r[both] = np.abs(R[both] - Rw[both]) <= rtol_r * Rw[both]  # ... and hits agree in range
    smax = max(want["sigma_re"].max(), 1e-30)
    close_s = np.abs(got["sigma_re"] - want["sigma_re"]) <= rtol_s * np.maximum(want["sigma_re"], 1e-3 * smax)
    close_v = np.abs(got["vel"] - want["vel"]) <= atol_v
    bad = ~(close_r & close_s & close_v)
    if bad.any():
        amb = _ambiguous(scene, want["az"][bad], want["el"][bad], want["prim"][bad])
        assert amb.all(), f"{int((~amb).sum())} non-ambiguous pixels differ"
    assert bad.mean() <= max_ambiguous
    assert np.all(got["sigma_im"] == 0)
    return bad


@pytest.mark.parametrize("dtype,rtol_r,rtol_s,atol_v", [
    (torch.float64, 1e-11, 1e-9, 1e-9),
    # FP32: a handful of roundings of O(1-10) quantities, with the root's sqrt(disc)
    # amplifying near (but not at) a silhouette: 2e-5 relative range error budget
    (torch.float32, 2e-5, 1e-3, 2e-4),
])
def test_random_scene_matches_oracle(ctx, dtype, rtol_r, rtol_s, atol_v):
    scene = synth.random_scene(seed=7, n_prims=12)
    n_az, n_el = 200, 96
    got = _host(ctx.raycast(scene, n_az, n_el, FOV, dtype=dtype))
    torch.cuda.synchronize()
    want = rc.raycast(scene, n_az, n_el, *FOV)
    assert np.isfinite(want["range"]).sum() > 2000
    # pixel angles: the grid formula in FP64, rounded to the buffer type
    np.testing.assert_array_equal(got["az"], want["az"].astype(got["az"].dtype))
    np.testing.assert_array_equal(got["el"], want["el"].astype(got["el"].dtype))
    _compare(scene, got, want, rtol_r, rtol_s, atol_v)


def test_no_falloff_and_many_primitives(ctx):
    # more primitives than one shared-memory tile (64), and the flag without 1/R^2
    scene = synth.random_scene(seed=11, n_prims=150)
    got = _host(ctx.raycast(scene, 96, 48, FOV, dtype=torch.float64, falloff=False))
    want = rc.raycast(scene, 96, 48, *FOV, falloff=False)
    _compare(scene, got, want, 1e-11, 1e-9, 1e-9, max_ambiguous=0.03)


def test_empty_scene_is_all_background(ctx):
    got = _host(ctx.raycast([], 33, 7, FOV))
    assert np.all(np.isinf(got["range"])) and np.all(got["sigma_re"] == 0) and np.all(got["vel"] == 0)


def test_invalid_scenes_are_rejected(ctx):
    good = synth.random_scene(seed=7, n_prims=3)
    bad_ell = [dict(good[2], c=np.asarray(good[2]["b"]) * 0.5 + np.asarray(good[2]["c"]))]
    bad_cap = [dict(good[1], c=np.array([0.0, 0, 0]))]
    bad_plane = [dict(good[0], c=np.asarray(good[0]["b"]) * 2.0)]
    for scene in (bad_ell, bad_cap, bad_plane):
        with pytest.raises(_abi.RsimError):
            ctx.raycast(scene, 8, 8, FOV)
    out = {k: torch.empty(63, dtype=torch.float32, device="cuda") for k in device.FIELDS}
    with pytest.raises(_abi.RsimError):
        ctx.raycast(good, 8, 8, FOV, out=out)  # P != n_az n_el


def test_rendered_walking_frame_synthesises_and_sees_the_walker(ctx):
    # render -> synthesise -> range-Doppler: the strongest moving return of the rendered
    # pedestrian lies within two Doppler bins of its torso's closing speed
    radar = synth.Radar(M=3, N=4, Ns=256, L=128)
    scene, truth = synth.walking_scene(frame=30)
    px = ctx.raycast(scene, 256, 128, FOV)
    cube = ctx.synth(radar, px, "fp32")
    power = torch.empty((1, radar.Ns, radar.L), dtype=torch.float32, device="cuda")
    v_est = torch.empty(1, dtype=torch.float32, device="cuda")
    _abi.rsim_range_doppler(ctx.h, radar, [cube], power, v_est, None, skip_static=True)
    torch.cuda.synchronize()
    r = radar.resolved()
    bin_v = r.lam / (2 * r.t_slow * r.L)
    assert abs(float(v_est.item()) - truth["closing_speed"]) <= 2 * bin_v + 0.35
