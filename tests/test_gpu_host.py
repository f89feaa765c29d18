"""rsim_synth_host: host pixel buffers in, host cube out, bit-identical to rsim_synth on
device copies of the same buffers, for pinned and pageable host memory, growing frames
and an empty frame."""
import numpy as np
import pytest
import torch

from paper_2307_09226_gb300 import _abi, device, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = device.Context(0)
    yield c
    c.close()


def _host(frame, pin):
    t = {k: torch.from_numpy(np.ascontiguousarray(a)) for k, a in zip(device.FIELDS, frame.pixels.arrays())}
    return {k: v.pin_memory() for k, v in t.items()} if pin else t


@pytest.mark.parametrize("tier", ["fp32", "split_bf16", "nufft"])
@pytest.mark.parametrize("pin", [True, False])
def test_host_call_equals_device_call(ctx, tier, pin):
    for n_az, n_el in ((31, 17), (64, 50)):  # the second frame grows the staging buffer
        f = synth.parity_frame(seed=n_az, n_az=n_az, n_el=n_el)
        want = ctx.synth(f.radar, device.upload(f), tier).cpu().numpy()
        got = ctx.synth_host(f.radar, _host(f, pin), tier)
        torch.cuda.synchronize()
        assert ctx.sync_status() == _abi.OK
        assert np.array_equal(got.numpy(), want)


def test_host_call_complex128_and_empty_frame(ctx):
    f = synth.config1()
    want = ctx.synth(f.radar, device.upload(f), "fp32", out_dtype="complex128").cpu().numpy()
    got = ctx.synth_host(f.radar, _host(f, True), "fp32", out_dtype="complex128")
    torch.cuda.synchronize()
    assert got.dtype == torch.complex128 and np.array_equal(got.numpy(), want)
    px = f.pixels
    px.sigma_re[:] = 0.0
    px.sigma_im[:] = 0.0
    got = ctx.synth_host(f.radar, _host(synth.Frame(f.radar, px, "complex128"), True), "split_bf16")
    torch.cuda.synchronize()
    assert np.all(got.numpy() == 0)


def test_device_tensors_are_rejected(ctx):
    f = synth.parity_frame(seed=3, n_az=8, n_el=8)
    with pytest.raises(ValueError):
        ctx.synth_host(f.radar, device.upload(f), "fp32")


@pytest.mark.parametrize("tier,out_dtype", [("fp32", "complex64"), ("split_fp16", "complex64"),
                                            ("split_bf16", "complex128")])
def test_host_call_row_ranges(ctx, tier, out_dtype):
    """A full-size frame whose pixels are split across several partial sums: the host
    call's cube equals the device call's bit for bit."""
    f = synth.config2()
    want = ctx.synth(f.radar, device.upload(f), tier, out_dtype=out_dtype).cpu().numpy()
    plan = _abi.rsim_get_plan(ctx.h, f.radar, f.pixels.P, _abi.TIERS[tier])
    assert plan.splits > 1  # the split reduction runs
    got = ctx.synth_host(f.radar, _host(f, True), tier, out_dtype=out_dtype)
    torch.cuda.synchronize()
    assert ctx.sync_status() == _abi.OK
    assert np.array_equal(got.numpy(), want)
