"""GPU parity of the CUDA path against the CPU FP64 oracle, through the C ABI.

Bars: index lists bit-exact; fixed-point phases within 1 unit of 2^-32 of the FP64
values; cubes within the normwise relative L2 tolerance of their tier
(FP32 direct and split precision 2e-5, plain 16-bit 1e-2).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2307_09226_gb300 import synth
from paper_2307_09226_gb300.synth import Pixels, Radar

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-5, "split_fp16": 2e-5, "split_bf16": 2e-5, "bf16": 1e-2, "fp16": 1e-2, "nufft": 2e-5}
TENSOR_TIERS = ("split_fp16", "split_bf16", "bf16", "fp16")
ALL_TIERS = ("fp32",) + TENSOR_TIERS + ("nufft",)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2307_09226_gb300 import device
    c = device.Context(0)
    yield c
    c.close()


def _dev():
    from paper_2307_09226_gb300 import device
    return device


def _run(ctx, frame, tier, out_dtype=None):
    from paper_2307_09226_gb300 import _abi
    dev = _dev()
    px = dev.upload(frame)
    cube = ctx.synth(frame.radar, px, tier, out_dtype=out_dtype or frame.out_dtype)
    assert ctx.sync_status() == _abi.OK
    return cube.cpu().numpy()


# ------------------------------------------------------------------ mask / compaction

@pytest.mark.parametrize("maker", [
    lambda: synth.config1().pixels,
    lambda: synth.config2().pixels,
    lambda: synth.parity_frame(seed=12, n_az=37, n_el=29, mask_frac=0.55).pixels,
    lambda: synth.random_frame(Radar(1, 1, 4, 4), 3000, 1, seed=9, mask_frac=1.0),
    lambda: synth.random_frame(Radar(1, 1, 4, 4), 1, 1, seed=9),
])
def test_valid_indices_bit_exact(ctx, maker):
    px = maker()
    idx = ctx.valid_indices(_dev().upload(px)).cpu().numpy().astype(np.int64)
    ref = oracle.valid_indices(px.sigma_re, px.sigma_im)
    assert np.array_equal(idx, ref)


def test_negative_zero_strength_is_masked(ctx):
    n = 2053
    rng = np.random.default_rng(2)
    sre = rng.normal(size=n).astype(np.float32)
    sim = rng.normal(size=n).astype(np.float32)
    sre[::3] = -0.0
    sim[::3] = 0.0
    sre[1::7] = 0.0  # imaginary part alone keeps the pixel
    px = Pixels(np.full(n, 2.0, np.float32), sre, sim, np.zeros(n, np.float32),
                np.zeros(n, np.float32), np.zeros(n, np.float32))
    idx = ctx.valid_indices(_dev().upload(px)).cpu().numpy()
    assert np.array_equal(idx.astype(np.int64), oracle.valid_indices(sre, sim))


# ------------------------------------------------------------------ FP64 pixel-to-path

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_path_phases_match_fp64(ctx, dtype):
    f = synth.parity_frame(seed=21, M=3, N=4, n_az=61, n_el=17, dtype=dtype)
    ph = ctx.path_phases(f.radar, _dev().upload(f))
    t = oracle.path_terms(f.radar, f.pixels)
    p = t["params"]
    assert ph["P_valid"] == t["idx"].size
    two32 = 2.0 ** 32

    def units(x):
        return np.mod(np.round(np.mod(x, 1.0) * two32), two32).astype(np.int64)

    def close(got, want):
        d = (got.astype(np.int64) - want) % (1 << 32)
        d = np.minimum(d, (1 << 32) - d)
        return int(d.max()) if d.size else 0

    a = 2 * p["mu"] * t["R_pv"] / (p["c"] * p["fs"])
    cph = t["k"] * p["d_rx"] * t["u"][None, :] / p["lam"]
    b = -t["fD"] * p["t_slow"]
    assert close(ph["a"], units(a)) <= 1
    assert close(ph["c"], units(cph)) <= 1
    assert close(ph["b"], units(b)) <= 1
    s = t["sigma"]
    np.testing.assert_array_equal(ph["sigma"][:, 0], s.real.astype(np.float32))
    np.testing.assert_array_equal(ph["sigma"][:, 1], s.imag.astype(np.float32))


# ------------------------------------------------------------------ cube parity

@pytest.mark.parametrize("tier", ALL_TIERS)
def test_config1_cube(ctx, tier):
    f = synth.config1()
    ref = oracle.cube_literal(f.radar, f.pixels)
    got = _run_or_skip(ctx, f, tier)
    assert got.dtype == np.complex128
    err = oracle.rel_l2(got, ref)
    print(f"config1 {tier}: {err:.3e}")
    assert err <= TOL[tier]


def _run_or_skip(ctx, f, tier, out_dtype=None):
    from paper_2307_09226_gb300 import _abi
    try:
        return _run(ctx, f, tier, out_dtype)
    except _abi.RsimError as e:
        if e.status == _abi.ERR_UNSUPPORTED:
            pytest.skip(f"{tier} not built")
        raise


@pytest.mark.parametrize("tier", ALL_TIERS)
@pytest.mark.parametrize("shape", [
    dict(M=2, N=3, Ns=96, L=48, n_az=71, n_el=70),      # ragged rows, columns and pixels
    dict(M=1, N=1, Ns=8, L=8, n_az=5, n_el=3),          # tiny: one partial tile
    dict(M=4, N=2, Ns=200, L=136, n_az=50, n_el=41),    # L > 128: two column tiles
    dict(M=1, N=3, Ns=33, L=12, n_az=100, n_el=1),      # odd everything
])
def test_ragged_cube(ctx, tier, shape):
    f = synth.parity_frame(seed=31, **shape)
    ref = oracle.cube_separable(f.radar, f.pixels)
    got = _run_or_skip(ctx, f, tier)
    err = oracle.rel_l2(got, ref)
    print(f"{shape} {tier}: {err:.3e}")
    assert err <= TOL[tier]


@pytest.mark.parametrize("tier", ALL_TIERS)
def test_config2_full_frame(ctx, tier):
    f = synth.config2()
    ref = oracle.cube_separable(f.radar, f.pixels)
    got = _run_or_skip(ctx, f, tier)
    err = oracle.rel_l2(got, ref)
    print(f"config2 {tier}: {err:.3e}")
    assert err <= TOL[tier]


LARGEST_CHANNELS = [0, 23, 47]
_largest_refs = {}


def _largest_frame(mask):
    """The largest request the server admits: 512 x 512 pixels, V = 48, N_s = 512, L = 256,
    with the serving mix's 30% background mask or none (262,144 valid pixels, the longest
    pixel sum)."""
    radar = Radar(M=4, N=12, Ns=512, L=256)
    px = synth.random_frame(radar, 512, 512, seed=77, mask_frac=mask)
    if mask not in _largest_refs:
        _largest_refs[mask] = oracle.cube_separable(radar, px, channels=LARGEST_CHANNELS)
    return synth.Frame(radar, px, "complex64"), _largest_refs[mask]


@pytest.mark.parametrize("mask", [0.3, 0.0])
@pytest.mark.parametrize("tier", ["fp32", "split_fp16", "split_bf16", "nufft"])
def test_largest_serving_shape_normwise(ctx, tier, mask):
    """Normwise error over whole channels (first, middle, last) of the largest serving
    request, at the tier's bar: the longest accumulations the library runs."""
    f, ref = _largest_frame(mask)
    got = _run(ctx, f, tier)[LARGEST_CHANNELS]
    err = oracle.rel_l2(got, ref)
    print(f"largest shape, mask {mask}, {tier}: {err:.3e}")
    assert err <= TOL[tier]


@pytest.mark.parametrize("tier", ALL_TIERS)
def test_empty_and_all_masked_frames_give_zero(ctx, tier):
    radar = Radar(M=2, N=2, Ns=16, L=8)
    px = synth.random_frame(radar, 40, 40, seed=1, mask_frac=1.0)
    got = _run_or_skip(ctx, synth.Frame(radar, px, "complex64"), tier)
    assert not np.any(got)
    from paper_2307_09226_gb300 import _abi
    import torch
    empty = {k: torch.zeros(0, dtype=torch.float32, device="cuda") for k in _dev().FIELDS}
    cube = torch.full((4, 16, 8), 7.0, dtype=torch.complex64, device="cuda")
    _abi.rsim_synth(ctx.h, radar, empty, _abi.TIERS[tier], cube)
    assert ctx.sync_status() == _abi.OK
    assert not torch.any(cube != 0)


def test_nonfinite_valid_pixel_is_reported(ctx):
    from paper_2307_09226_gb300 import _abi
    f = synth.parity_frame(seed=4, n_az=20, n_el=10, mask_frac=0.0)
    f.pixels.range[17] = np.nan
    px = _dev().upload(f)
    ctx.synth(f.radar, px, "fp32")
    assert ctx.sync_status() == _abi.ERR_NONFINITE
    # a masked pixel's fields are ignored
    f2 = synth.parity_frame(seed=4, n_az=20, n_el=10, mask_frac=0.0)
    f2.pixels.range[17] = np.nan
    f2.pixels.sigma_re[17] = 0.0
    f2.pixels.sigma_im[17] = 0.0
    ctx.synth(f2.radar, _dev().upload(f2), "fp32")
    assert ctx.sync_status() == _abi.OK


def test_invalid_arguments_are_rejected(ctx):
    from paper_2307_09226_gb300 import _abi
    import torch
    f = synth.parity_frame(seed=4, n_az=20, n_el=10)
    px = _dev().upload(f)
    cube = _dev().cube_tensor(f.radar)
    bad = Radar(M=0, N=4, Ns=8, L=8)
    with pytest.raises(_abi.RsimError) as e:
        _abi.rsim_synth(ctx.h, bad, px, 0, cube)
    assert e.value.status == _abi.ERR_INVALID_ARG
    with pytest.raises(_abi.RsimError) as e:
        _abi.rsim_synth(ctx.h, f.radar, px, 99, cube)
    assert e.value.status == _abi.ERR_INVALID_ARG
    huge = Radar(M=1024, N=1024, Ns=1 << 16, L=1 << 16)
    with pytest.raises(_abi.RsimError) as e:
        _abi.rsim_synth(ctx.h, huge, px, 0, cube)
    assert e.value.status == _abi.ERR_OVERFLOW


@pytest.mark.parametrize("tier", ALL_TIERS)
def test_repeat_runs_are_bit_identical(ctx, tier):
    f = synth.parity_frame(seed=8, M=3, N=4, Ns=128, L=64, n_az=90, n_el=80)
    a = _run_or_skip(ctx, f, tier)
    b = _run_or_skip(ctx, f, tier)
    assert np.array_equal(a, b)


def test_linearity_in_sigma_on_gpu(ctx):
    f = synth.parity_frame(seed=13, n_az=30, n_el=30, mask_frac=0.2)
    a = _run(ctx, f, "fp32")
    g = synth.parity_frame(seed=13, n_az=30, n_el=30, mask_frac=0.2)
    g.pixels.sigma_re *= 2.0
    g.pixels.sigma_im *= 2.0
    b = _run(ctx, g, "fp32")
    assert np.array_equal(b, 2 * a)  # power-of-two scaling is exact end to end


def test_point_target_fft_peaks_on_gpu(ctx):
    """The GPU cube of a point target peaks at the FMCW range bin and Doppler bin."""
    radar = Radar(M=3, N=4, Ns=256, L=128)
    r = radar.resolved()
    k_r, k_d = 37, 9
    R = k_r * r.c * r.fs / (2 * r.mu * r.Ns)
    vel = k_d * r.lam / (2 * r.t_slow * r.L)
    px = synth.point_scatterer(radar, R, 1.5 + 0.5j, 0.0, 0.0, vel, dtype=np.float32)
    cube = _run(ctx, synth.Frame(radar, px, "complex64"), "fp32")
    spec = np.abs(np.fft.fft2(cube[0]))
    kr, kd = np.unravel_index(np.argmax(spec), spec.shape)
    assert (kr, kd) == (k_r, (-k_d) % r.L)


@pytest.mark.parametrize("tier", ["fp32", "split_fp16", "split_bf16", "bf16", "nufft"])
def test_tdm_motion_flag(ctx, tier):
    """RSIM_FLAG_TDM_MOTION adds -f_D m T_b per Tx slot; parity with the oracle."""
    from dataclasses import replace
    f = synth.parity_frame(seed=17, M=3, N=4, Ns=64, L=32, n_az=60, n_el=40)
    radar = replace(f.radar, tdm_motion=True)
    g = synth.Frame(radar, f.pixels, "complex64")
    ref = oracle.cube_separable(radar, f.pixels)
    got = _run_or_skip(ctx, g, tier)
    assert oracle.rel_l2(got, ref) <= TOL[tier]
    plain = oracle.cube_separable(f.radar, f.pixels)
    assert oracle.rel_l2(got, plain) > 1e-3  # the term is really there


def test_tensor_core_rate_probe(ctx):
    """The measured flop rate of the contraction's MMA instruction (the ceiling of its
    executed rate) is plausible for this GPU: above 1 PFLOP/s and at most the rate of one
    M=128, N=256, K=16 MMA per 128 clocks per SM at a 2.1 GHz clock on 152 SMs, with
    headroom."""
    from paper_2307_09226_gb300 import _abi
    rate = _abi.rsim_measure_mma_rate(ctx.h)
    print(f"tensor-core MMA rate: {rate / 1e12:.1f} TFLOP/s")
    assert 1e15 < rate < 1.1 * 152 * (2 * 128 * 256 * 16 / 128) * 2.1e9


@pytest.mark.parametrize("tier", ["split_fp16", "fp32"])
def test_cuda_graph_capture_replays_the_call(ctx, tier):
    """rsim_synth and rsim_synth_host captured into a CUDA graph (after an uncaptured call
    sized the workspace) allocate nothing while captured, and every replay gives the same
    bits as the plain call."""
    torch = pytest.importorskip("torch")
    device = _dev()
    f = synth.parity_frame(seed=71, M=2, N=4, Ns=64, L=48, n_az=40, n_el=30)
    px = device.upload(f)
    plain = ctx.synth(f.radar, px, tier).cpu().numpy()
    host = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            for k, a in zip(device.FIELDS, f.pixels.arrays())}
    out_host = device.cube_tensor(f.radar, device="cpu").pin_memory()
    ctx.synth_host(f.radar, host, tier, cube=out_host)  # sizes the staging buffer
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    cube = device.cube_tensor(f.radar)
    g1, g2 = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(g1, stream=s):
        ctx.synth(f.radar, px, tier, cube=cube, stream=s)
    with torch.cuda.graph(g2, stream=s):
        ctx.synth_host(f.radar, host, tier, cube=out_host, stream=s)
    for _ in range(2):
        cube.zero_()
        out_host.zero_()
        g1.replay()
        g2.replay()
        torch.cuda.synchronize()
        assert np.array_equal(cube.cpu().numpy(), plain)
        assert np.array_equal(out_host.numpy(), plain)
