"""GPU range-Doppler maps and max-power velocities (rsim_range_doppler) against the
FP64 oracle of the same cube, plus the Doppler-time method of Section III on the
walking-pedestrian batch."""
import numpy as np
import pytest

import oracle
from paper_2307_09226_gb300 import synth
from paper_2307_09226_gb300.synth import Radar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2307_09226_gb300 import _abi, device
    ctx = device.Context(0)
    yield torch, _abi, device, ctx
    ctx.close()


def _rd(env, radar, cubes, skip_static=False):
    torch, _abi, device, ctx = env
    F = len(cubes)
    power = torch.empty((F, radar.Ns, radar.L), dtype=torch.float32, device="cuda")
    v = torch.empty(F, dtype=torch.float32, device="cuda")
    peak = torch.empty((F, 2), dtype=torch.int32, device="cuda")
    _abi.rsim_range_doppler(ctx.h, radar, cubes, power, v, peak, skip_static=skip_static)
    torch.cuda.synchronize()
    return power.cpu().numpy(), v.cpu().numpy(), peak.cpu().numpy()


@pytest.mark.parametrize("shape", [dict(M=2, N=4, Ns=64, L=32), dict(M=3, N=4, Ns=256, L=128),
                                   dict(M=1, N=2, Ns=512, L=256)])
def test_power_map_matches_oracle(env, shape):
    torch, _abi, device, ctx = env
    f = synth.parity_frame(seed=5, n_az=40, n_el=30, **shape)
    cube = ctx.synth(f.radar, device.upload(f), "fp32")
    pw, v, peak = _rd(env, f.radar, [cube])
    ref = oracle.range_doppler_power(cube.cpu().numpy())
    assert np.linalg.norm(pw[0] - ref) / np.linalg.norm(ref) < 1e-5
    # the chosen bin holds the maximum (to FP32 rounding), and its velocity follows
    k, d = peak[0]
    assert ref[k, d] >= ref.max() * (1 - 1e-5)
    L = f.radar.L
    r = f.radar.resolved()
    ds = d if d < L // 2 else d - L
    assert abs(v[0] - (-ds * r.lam / (2 * r.t_slow * L))) < 1e-6


def test_point_targets_give_their_velocity(env):
    torch, _abi, device, ctx = env
    radar = Radar(M=3, N=4, Ns=256, L=128)
    r = radar.resolved()
    cubes, truth = [], []
    for k_r, k_d, sign in [(20, 7, 1), (41, 3, -1), (100, 31, 1)]:
        R = k_r * r.c * r.fs / (2 * r.mu * r.Ns)
        vel = sign * k_d * r.lam / (2 * r.t_slow * r.L)
        px = synth.point_scatterer(radar, R, 1 + 1j, 0.2, 0.0, vel, dtype=np.float32)
        cubes.append(ctx.synth(radar, device.upload(px), "fp32"))
        truth.append((vel, (-sign * k_d) % r.L))
    pw, v, peak = _rd(env, radar, cubes)
    for i, (vel, d) in enumerate(truth):
        assert peak[i][1] == d
        assert abs(v[i] - vel) < 1e-4


def test_doppler_time_on_walking_scene(env):
    """Section III's method on the synthetic walk: max-power velocity per CPI with the
    zero-Doppler notch (the wall is static), against the torso velocity."""
    torch, _abi, device, ctx = env
    frames = synth.walking_batch(n_frames=16, n_az=128, n_el=128)
    radar = frames[0].radar
    cubes = ctx.synth_batch(radar, [device.upload(f) for f in frames], "split_fp16")
    pw, v, peak = _rd(env, radar, cubes, skip_static=True)
    for i in (0, 9):
        ref = oracle.range_doppler_power(cubes[i].cpu().numpy())
        ref_v, _ = oracle.max_power_velocity(radar, ref, skip_static=True)
        k, d = peak[i]
        refn = ref.copy()
        refn[:, 0] = -1
        assert refn[k, d] >= refn.max() * (1 - 1e-4)
    truth = np.array([f.meta["v_torso"] for f in frames])
    err = oracle.e_velo(v, truth)
    print(f"E_velo on the synthetic walk: {err:.3f} m/s")
    assert np.all(np.isfinite(v)) and err < 1.5  # limbs spread +-1.5 m/s around the torso


def test_non_power_of_two_is_unsupported(env):
    torch, _abi, device, ctx = env
    radar = Radar(M=1, N=1, Ns=48, L=32)
    cube = torch.zeros((1, 48, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(_abi.RsimError) as e:
        _rd(env, radar, [cube])
    assert e.value.status == _abi.ERR_UNSUPPORTED
