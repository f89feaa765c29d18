"""GPU NUFFT tier: agreement with the CPU NUFFT reference at the same kernel width
(implementation error only), repeat runs and batches bit-identical to single frames,
empty frames, crowded grids, and the size limits."""
import numpy as np
import pytest
import torch

import oracle
import oracle.nufft as nu
from paper_2307_09226_gb300 import _abi, device, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = device.Context(0)
    yield c
    c.close()


def test_gpu_matches_cpu_nufft_at_width_7(ctx):
    # both compute the same gridding approximation; the GPU adds FP32 rounding only
    f = synth.parity_frame(seed=41, M=2, N=2, Ns=128, L=64, n_az=90, n_el=60)
    got = ctx.synth(f.radar, device.upload(f), "nufft").cpu().numpy()
    cpu = nu.cube_nufft(f.radar, f.pixels, w=7)
    ref = oracle.cube_separable(f.radar, f.pixels)
    e_impl, e_cpu, e_gpu = oracle.rel_l2(got, cpu), oracle.rel_l2(cpu, ref), oracle.rel_l2(got, ref)
    print(f"gpu vs cpu nufft {e_impl:.2e}, cpu nufft vs exact {e_cpu:.2e}, gpu vs exact {e_gpu:.2e}")
    assert e_impl <= 5e-6
    assert e_gpu <= 2e-5


def test_kernel_widths(ctx):
    # every width against the CPU NUFFT at that width (implementation error only), and
    # against the exact sum: the error falls by orders of magnitude as the width grows
    from dataclasses import replace
    f = synth.parity_frame(seed=52, M=2, N=2, Ns=64, L=32, n_az=40, n_el=30)
    ref = oracle.cube_separable(f.radar, f.pixels)
    errs = {}
    for w in (4, 5, 6, 7, 8):
        radar = replace(f.radar, nufft_width=w)
        got = ctx.synth(radar, device.upload(f), "nufft").cpu().numpy()
        cpu = nu.cube_nufft(radar, f.pixels, w=w)
        assert oracle.rel_l2(got, cpu) <= 5e-6, w
        errs[w] = oracle.rel_l2(got, ref)
    print("gpu nufft vs exact by width", {w: f"{e:.1e}" for w, e in errs.items()})
    assert all(errs[w + 1] < 0.3 * errs[w] for w in (4, 5, 6))
    assert errs[7] <= 5e-6 and errs[4] > 1e-4
    for bad in (3, 9):
        with pytest.raises(_abi.RsimError) as e:
            ctx.synth(replace(f.radar, nufft_width=bad), device.upload(f), "nufft")
        assert e.value.status == _abi.ERR_INVALID_ARG


def test_crowded_grid_cell(ctx):
    # every pixel at nearly the same range and speed: all points land in one grid tile,
    # which the work items share among many CTAs
    r = synth.Radar(M=2, N=2, Ns=64, L=32)
    px = synth.random_frame(r, 100, 100, seed=8, r_lo=3.0, r_hi=3.001, v_max=0.001)
    got = ctx.synth(r, device.upload(px), "nufft").cpu().numpy()
    ref = oracle.cube_separable(r, px)
    assert oracle.rel_l2(got, ref) <= 2e-5


def test_batch_equals_alone_bitwise(ctx):
    frames = synth.walking_batch(n_frames=4, n_az=96, n_el=64)
    radar = frames[0].radar
    pxs = [device.upload(f) for f in frames]
    alone = [ctx.synth(radar, px, "nufft").cpu().numpy() for px in pxs]
    again = [ctx.synth(radar, px, "nufft").cpu().numpy() for px in pxs]
    batch = [c.cpu().numpy() for c in ctx.synth_batch(radar, pxs, "nufft")]
    for a, b, c in zip(alone, again, batch):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_batch_reusing_streams_and_scratch_bitwise(ctx):
    """More frames than the library's NUFFT streams (eight): later frames reuse a
    stream and its grid scratch after an earlier frame; every frame, including the
    empty one, still equals its single-frame result bit for bit."""
    frames = synth.walking_batch(n_frames=11, n_az=64, n_el=48)
    radar = frames[0].radar
    px0 = frames[3].pixels
    px0.sigma_re[:] = 0.0
    px0.sigma_im[:] = 0.0
    frames[3] = synth.Frame(radar, px0, frames[3].out_dtype)
    pxs = [device.upload(f) for f in frames]
    alone = [ctx.synth(radar, px, "nufft").cpu().numpy() for px in pxs]
    batch = [c.cpu().numpy() for c in ctx.synth_batch(radar, pxs, "nufft")]
    torch.cuda.synchronize()
    assert ctx.sync_status() == _abi.OK
    assert np.all(alone[3] == 0)
    for a, c in zip(alone, batch):
        assert np.array_equal(a, c)


def test_empty_frame_gives_zero(ctx):
    f = synth.config2()
    px = f.pixels.astype(np.float32)
    px.sigma_re[:] = 0.0
    px.sigma_im[:] = 0.0
    got = ctx.synth(f.radar, device.upload(px), "nufft").cpu().numpy()
    assert np.all(got == 0)


# Grid sides G = 2 N from 16 to 4096 take every FFT kernel shape: one radix-16 pass
# (G = 16), radix 16 then 2, 4, 8 or 16 (G = 32 .. 256), and two radix-16 passes then
# 2, 4, 8 or 16 (G = 512 .. 4096), on both axes; G = 4096 is the largest grid supported.
@pytest.mark.parametrize("Ns,L", [(8, 2048), (16, 1024), (32, 512), (64, 256), (128, 128), (256, 64),
                                  (512, 32), (1024, 16), (2048, 8)])
def test_every_fft_shape_against_exact_sum(ctx, Ns, L):
    f = synth.parity_frame(seed=Ns + L, M=1, N=2, Ns=Ns, L=L, n_az=13, n_el=11)
    got = ctx.synth(f.radar, device.upload(f), "nufft").cpu().numpy()
    ref = oracle.cube_separable(f.radar, f.pixels)
    assert oracle.rel_l2(got, ref) <= 2e-5


@pytest.mark.parametrize("Ns,L", [(4096, 4), (64, 2)])
def test_unsupported_axes(ctx, Ns, L):
    r = synth.Radar(M=1, N=1, Ns=Ns, L=L)
    px = synth.random_frame(r, 8, 8, seed=1)
    with pytest.raises(_abi.RsimError) as e:
        ctx.synth(r, device.upload(px), "nufft")
    assert e.value.status == _abi.ERR_UNSUPPORTED


def test_shared_atomic_rate_probe(ctx):
    """The measured shared-memory atomic rate (the spreading kernel's roofline denominator)
    is a plausible number for a GPU of this size: above 1e12 and at most the one
    32-lane-wavefront-per-clock figure at a 2.1 GHz clock on 152 SMs, with headroom."""
    rate = _abi.rsim_measure_smem_atomics(ctx.h)
    print(f"shared atomics: {rate / 1e12:.3f} T lane-op/s")
    assert 1e12 < rate < 1.2 * 152 * 32 * 2.1e9
