"""Failure detection on the GPU without a fault: the library's bounded device wait runs
out on a barrier phase that nothing completes, the timeout reaches the host through the
status word, and the same context then computes a correct cube."""
import time

import pytest
import torch

import oracle
from paper_2307_09226_gb300 import _abi, device, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = device.Context(0)
    yield c
    c.close()


def test_device_wait_runs_out_and_context_recovers(ctx):
    assert ctx.sync_status() == _abi.OK
    limit_ns = 20_000_000
    t0 = time.perf_counter()
    ctx.selftest_wait_timeout(limit_ns)
    assert ctx.sync_status() == _abi.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= limit_ns * 1e-9
    assert ctx.sync_status() == _abi.OK  # reported once, then cleared
    f = synth.parity_frame(seed=5, n_az=40, n_el=30)
    for tier in ("split_bf16", "nufft"):
        got = ctx.synth(f.radar, device.upload(f), tier).cpu().numpy()
        assert ctx.sync_status() == _abi.OK
        assert oracle.rel_l2(got, oracle.cube_separable(f.radar, f.pixels)) <= 2e-5


@pytest.mark.parametrize("limit_ns", [0, 999, 10_000_000_001])
def test_limit_out_of_range_is_rejected(ctx, limit_ns):
    with pytest.raises(_abi.RsimError) as e:
        ctx.selftest_wait_timeout(limit_ns)
    assert e.value.status == _abi.ERR_INVALID_ARG
