"""GPU tests of the batched path, the serving loop and the autotuner (through the C ABI).

* A batch of frames gives, frame by frame, the same bits as rsim_synth of each frame
  alone (equal pixel counts share a plan), and matches the FP64 oracle.
* The server's results equal the alone results, whatever mix of shapes and tiers runs
  concurrently; admission keeps the reserved workspace within the HBM budget; queued
  requests can be cancelled; a non-finite valid pixel is reported per request.
* The autotuner's choice is cached (in the context and in RSIM_TUNE_CACHE) and keeps
  results within tolerance.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2307_09226_gb300 import synth
from paper_2307_09226_gb300.synth import Radar

pytestmark = pytest.mark.gpu

TOL = {"fp32": 2e-5, "split_fp16": 2e-5, "split_bf16": 2e-5, "bf16": 1e-2, "fp16": 1e-2, "nufft": 2e-5}


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


@pytest.mark.parametrize("tier", ["split_fp16", "fp32", "split_bf16"])
def test_batch_equals_alone_bit_for_bit(env, tier):
    torch, _abi, device, ctx = env
    frames = synth.walking_batch(n_frames=8, n_az=128, n_el=128)
    radar = frames[0].radar
    pxs = [device.upload(f) for f in frames]
    cubes = ctx.synth_batch(radar, pxs, tier)
    assert ctx.sync_status() == _abi.OK
    for f, px, cb in zip(frames, pxs, cubes):
        alone = ctx.synth(radar, px, tier).cpu().numpy()
        assert np.array_equal(cb.cpu().numpy(), alone), f.meta["frame"]
    for i in (0, 5):
        ref = oracle.cube_separable(radar, frames[i].pixels)
        err = oracle.rel_l2(cubes[i].cpu().numpy(), ref)
        print(f"batch {tier} frame {i}: {err:.3e}")
        assert err <= TOL[tier]


def test_batch_with_uneven_pixel_counts(env):
    torch, _abi, device, ctx = env
    radar = Radar(M=2, N=4, Ns=128, L=64)
    frames = [synth.random_frame(radar, a, b, seed=s, mask_frac=m)
              for a, b, s, m in [(60, 50, 1, 0.1), (10, 7, 2, 0.5), (90, 80, 3, 0.3), (33, 3, 4, 0.0)]]
    pxs = [device.upload(p) for p in frames]
    for tier in ("split_fp16", "fp32"):
        cubes = ctx.synth_batch(radar, pxs, tier)
        assert ctx.sync_status() == _abi.OK
        for p, cb in zip(frames, cubes):
            err = oracle.rel_l2(cb.cpu().numpy(), oracle.cube_separable(radar, p))
            assert err <= TOL[tier], (tier, err)


@pytest.mark.parametrize("tier", ["split_fp16", "bf16", "nufft"])
def test_batch_of_fp64_frames(env, tier):
    """A batch of FP64 pixel buffers of one size with uneven valid counts (the tensor tiers'
    operand builder computes every frame's fast-time phases from the FP64 fields): each
    frame is bit-identical to its alone result (equal pixel counts share a plan) and within
    its tier's tolerance of the oracle."""
    torch, _abi, device, ctx = env
    radar = Radar(M=2, N=4, Ns=96, L=40)
    frames = [synth.random_frame(radar, 60, 45, seed=s, mask_frac=m, dtype=np.float64)
              for s, m in [(11, 0.2), (12, 0.9), (13, 0.0)]]
    pxs = [device.upload(p) for p in frames]
    cubes = ctx.synth_batch(radar, pxs, tier)
    assert ctx.sync_status() == _abi.OK
    for p, px, cb in zip(frames, pxs, cubes):
        got = cb.cpu().numpy()
        assert np.array_equal(got, ctx.synth(radar, px, tier).cpu().numpy())
        err = oracle.rel_l2(got, oracle.cube_separable(radar, p))
        assert err <= TOL[tier], (tier, err)


def _requests(n, seed=5):
    reqs = synth.serving_requests(n, seed=seed, grids=(32, 48, 64),
                                  tiers=("fp32", "split_bf16", "split_fp16", "nufft"))
    return reqs


@pytest.mark.parametrize("policy,slots,express", [("first_fit", 4, 0), ("shortest_first", 4, 0),
                                                   ("first_fit", 3, 5)])
def test_server_results_equal_alone(env, policy, slots, express):
    torch, _abi, device, ctx = env
    reqs = _requests(16)
    frames = [synth.request_frame(r) for r in reqs]
    pxs = [device.upload(f) for f in frames]
    cubes = [device.cube_tensor(f.radar) for f in frames]
    srv = _abi.rsim_server_create(ctx.h, slots=slots, policy=policy, express_slots=express)
    try:
        tickets = []
        for r, f, px, cb in zip(reqs, frames, pxs, cubes):
            tickets.append(_abi.rsim_server_submit(srv, _abi.make_request(f.radar, px, _abi.TIERS[r["tier"]], cb)))
        for t in tickets:
            assert _abi.rsim_server_wait(srv, t, 60000) == _abi.OK, _abi.last_error()
        st = _abi.rsim_server_stats_get(srv)
        # a new tally after a reset counts only the requests submitted after it
        _abi.rsim_server_stats_reset(srv)
        st0 = _abi.rsim_server_stats_get(srv)
        again = [_abi.rsim_server_submit(srv, _abi.make_request(f.radar, px, _abi.TIERS[r["tier"]], cb))
                 for r, f, px, cb in list(zip(reqs, frames, pxs, cubes))[:2]]
        for t in again:
            assert _abi.rsim_server_wait(srv, t, 60000) == _abi.OK, _abi.last_error()
        st2 = _abi.rsim_server_stats_get(srv)
    finally:
        _abi.rsim_server_destroy(srv)
    assert st0.submitted == 0 and st0.completed == 0 and st0.p50_ms == 0 and st0.busy_s == 0
    assert st2.submitted == 2 and st2.completed == 2 and st2.p50_ms > 0
    assert st.submitted == 16 and st.completed == 16 and st.failed == 0
    assert st.p50_ms > 0 and st.p99_ms >= st.p50_ms
    assert st.peak_in_flight >= 2  # requests ran concurrently
    for r, f, px, cb in zip(reqs, frames, pxs, cubes):
        alone = ctx.synth(f.radar, px, r["tier"]).cpu().numpy()
        got = cb.cpu().numpy()
        assert np.array_equal(got, alone), r
    # a quarter of the mix against the FP64 oracle as well
    for i in (0, 5, 10, 15):
        ref = oracle.cube_separable(frames[i].radar, frames[i].pixels)
        err = oracle.rel_l2(cubes[i].cpu().numpy(), ref)
        print(policy, i, reqs[i]["tier"], f"{err:.3e}")
        assert err <= TOL[reqs[i]["tier"]]


def test_server_config5_stream_sampled_against_oracle(env):
    """The serving workload's own request mix (all radar shapes up to 512 x 512 pixels,
    FP32 and split-BF16), submitted at seeded exponential intervals so that requests
    overlap on the device: every request completes, and a seeded 5% sample is checked
    against the FP64 oracle at 32 random cube entries each (each entry its own FP64 sum
    over the pixels), normwise over the sampled entries at the tier's tolerance."""
    import time
    torch, _abi, device, ctx = env
    reqs = synth.serving_requests(60, seed=5)
    frames = [synth.request_frame(r) for r in reqs]
    pxs = [device.upload(f) for f in frames]
    cubes = [device.cube_tensor(f.radar) for f in frames]
    rng = np.random.default_rng(55)
    gaps = rng.exponential(0.004, size=len(reqs))  # mean 4 ms between arrivals
    srv = _abi.rsim_server_create(ctx.h, slots=3, express_slots=5)
    try:
        tickets = []
        for r, f, px, cb, gap in zip(reqs, frames, pxs, cubes, gaps):
            tickets.append(_abi.rsim_server_submit(srv, _abi.make_request(f.radar, px, _abi.TIERS[r["tier"]], cb)))
            time.sleep(float(gap))
        for t in tickets:
            assert _abi.rsim_server_wait(srv, t, 120000) == _abi.OK, _abi.last_error()
        st = _abi.rsim_server_stats_get(srv)
    finally:
        _abi.rsim_server_destroy(srv)
    assert st.completed == len(reqs) and st.failed == 0
    assert st.peak_in_flight >= 2
    sample = rng.choice(len(reqs), size=max(1, len(reqs) // 20), replace=False)
    for i in sample:
        r, f = reqs[i], frames[i]
        V, Ns, L = f.radar.V, f.radar.Ns, f.radar.L
        ent = np.stack([rng.integers(0, V, 32), rng.integers(0, Ns, 32), rng.integers(0, L, 32)], axis=1)
        ref = oracle.cube_entries(f.radar, f.pixels, ent)
        got = cubes[i].cpu().numpy()[ent[:, 0], ent[:, 1], ent[:, 2]]
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        print(f"request {i}: M={f.radar.M} N={f.radar.N} Ns={Ns} L={L} grid={r['grid']} {r['tier']}: {err:.3e}")
        assert err <= TOL[r["tier"]], (i, r["tier"], err)


def test_server_admission_respects_budget(env):
    torch, _abi, device, ctx = env
    reqs = _requests(8, seed=9)
    frames = [synth.request_frame(r) for r in reqs]
    pxs = [device.upload(f) for f in frames]
    cubes = [device.cube_tensor(f.radar) for f in frames]
    need = [_abi.rsim_workspace_size(ctx.h, f.radar, f.pixels.P, _abi.TIERS[r["tier"]])
            for r, f in zip(reqs, frames)]
    budget = max(need) + min(need) // 2  # at most about one request at a time
    srv = _abi.rsim_server_create(ctx.h, slots=4, hbm_budget_bytes=budget)
    try:
        ts = [_abi.rsim_server_submit(srv, _abi.make_request(f.radar, px, _abi.TIERS[r["tier"]], cb))
              for r, f, px, cb in zip(reqs, frames, pxs, cubes)]
        for t in ts:
            assert _abi.rsim_server_wait(srv, t, 60000) == _abi.OK
        st = _abi.rsim_server_stats_get(srv)
        assert st.peak_reserved_bytes <= budget
        assert st.completed == 8
        # a request larger than the whole budget is refused at submit
        big = Radar(M=4, N=12, Ns=512, L=256)
        bpx = synth.random_frame(big, 512, 512, seed=1, mask_frac=0.3)
        bcube = device.cube_tensor(big)
        assert _abi.rsim_workspace_size(ctx.h, big, bpx.P, 0) > budget
        with pytest.raises(_abi.RsimError) as e:
            _abi.rsim_server_submit(srv, _abi.make_request(big, device.upload(bpx), 0, bcube))
        assert e.value.status == _abi.ERR_BUDGET
    finally:
        _abi.rsim_server_destroy(srv)
    for r, f, px, cb in zip(reqs, frames, pxs, cubes):
        assert np.array_equal(cb.cpu().numpy(), ctx.synth(f.radar, px, r["tier"]).cpu().numpy())


@pytest.mark.parametrize("policy,age_ms,sleep_s,overtakes", [
    ("first_fit", 10000, 0.0, 1),        # the small request passes the one that does not fit
    ("shortest_first", 10000, 0.0, 1),
    ("first_fit", -1, 0.0, 0),           # strict FIFO: nothing overtakes
    ("first_fit", 1, 0.01, 0),           # the waiting request reached its age limit first
])
def test_server_overtaking_and_age_limit(env, policy, age_ms, sleep_s, overtakes):
    """Request A runs; B has A's workspace size, so it does not fit beside A in the budget;
    C is small and fits.  C may start before B only while B is younger than the age limit."""
    import time
    torch, _abi, device, ctx = env
    big = Radar(M=4, N=12, Ns=512, L=256)
    fa = synth.random_frame(big, 256, 256, seed=21, mask_frac=0.3)
    fb = synth.random_frame(big, 256, 256, seed=22, mask_frac=0.3)
    small = synth.parity_frame(seed=23, n_az=20, n_el=20)
    wa = _abi.rsim_workspace_size(ctx.h, big, fa.P, _abi.TIER_FP32)
    wc = _abi.rsim_workspace_size(ctx.h, small.radar, small.pixels.P, _abi.TIER_FP32)
    budget = wa + wc + (1 << 20)
    assert 2 * wa > budget
    srv = _abi.rsim_server_create(ctx.h, slots=3, hbm_budget_bytes=budget, policy=policy, age_limit_ms=age_ms)
    cubes = [device.cube_tensor(big), device.cube_tensor(big), device.cube_tensor(small.radar)]
    pxs = [device.upload(fa), device.upload(fb), device.upload(small)]
    radars = [big, big, small.radar]
    try:
        ta = _abi.rsim_server_submit(srv, _abi.make_request(big, pxs[0], _abi.TIER_FP32, cubes[0]))
        tb = _abi.rsim_server_submit(srv, _abi.make_request(big, pxs[1], _abi.TIER_FP32, cubes[1]))
        time.sleep(sleep_s)
        tc = _abi.rsim_server_submit(srv, _abi.make_request(small.radar, pxs[2], _abi.TIER_FP32, cubes[2]))
        for t in (ta, tb, tc):
            assert _abi.rsim_server_wait(srv, t, 60000) == _abi.OK, _abi.last_error()
        st = _abi.rsim_server_stats_get(srv)
    finally:
        _abi.rsim_server_destroy(srv)
    assert st.completed == 3 and st.peak_reserved_bytes <= budget
    assert st.overtakes == overtakes
    for r, px, cb in zip(radars, pxs, cubes):
        assert np.array_equal(cb.cpu().numpy(), ctx.synth(r, px, "fp32").cpu().numpy())


def test_server_express_slot_serves_short_requests_first(env):
    """With one general slot held by a long request and another long one queued, a short
    request runs at once on the express slot (it overtakes the queued long one) and
    finishes while the first long request is still running; every result equals the
    request run alone."""
    torch, _abi, device, ctx = env
    big = Radar(M=4, N=12, Ns=512, L=256)
    fa = synth.random_frame(big, 256, 256, seed=31, mask_frac=0.3)
    fb = synth.random_frame(big, 256, 256, seed=32, mask_frac=0.3)
    small = synth.parity_frame(seed=33, n_az=20, n_el=20)
    pxs = [device.upload(fa), device.upload(fb), device.upload(small)]
    radars = [big, big, small.radar]
    cubes = [device.cube_tensor(r) for r in radars]
    srv = _abi.rsim_server_create(ctx.h, slots=1, express_slots=1)
    try:
        ts = [_abi.rsim_server_submit(srv, _abi.make_request(r, px, _abi.TIER_FP32, cb))
              for r, px, cb in zip(radars, pxs, cubes)]
        assert _abi.rsim_server_wait(srv, ts[2], 30000) == _abi.OK
        assert _abi.rsim_server_wait(srv, ts[0], 0) == _abi.ERR_TIMEOUT  # the long one still runs
        for t in ts[:2]:
            assert _abi.rsim_server_wait(srv, t, 60000) == _abi.OK
        st = _abi.rsim_server_stats_get(srv)
    finally:
        _abi.rsim_server_destroy(srv)
    assert st.completed == 3 and st.overtakes == 1
    for r, px, cb in zip(radars, pxs, cubes):
        assert np.array_equal(cb.cpu().numpy(), ctx.synth(r, px, "fp32").cpu().numpy())


def test_server_cancel_and_errors(env):
    torch, _abi, device, ctx = env
    # one slot so that later requests stay queued behind a long first one
    big = Radar(M=4, N=12, Ns=512, L=256)
    bpx = device.upload(synth.random_frame(big, 256, 256, seed=2, mask_frac=0.3))
    bcube = device.cube_tensor(big)
    small = synth.parity_frame(seed=5, n_az=20, n_el=20)
    spx = device.upload(small)
    bad = synth.parity_frame(seed=6, n_az=20, n_el=20, mask_frac=0.0)
    bad.pixels.vel[3] = np.inf
    badpx = device.upload(bad)
    srv = _abi.rsim_server_create(ctx.h, slots=1)
    try:
        t0 = _abi.rsim_server_submit(srv, _abi.make_request(big, bpx, _abi.TIER_FP32, bcube))
        c1 = device.cube_tensor(small.radar)
        t1 = _abi.rsim_server_submit(srv, _abi.make_request(small.radar, spx, _abi.TIER_FP32, c1))
        c2 = device.cube_tensor(bad.radar)
        t2 = _abi.rsim_server_submit(srv, _abi.make_request(bad.radar, badpx, _abi.TIER_FP32, c2))
        assert _abi.rsim_server_cancel(srv, t1) == _abi.OK
        assert _abi.rsim_server_wait(srv, t1, 10000) == _abi.ERR_CANCELLED
        assert _abi.rsim_server_wait(srv, t0, 0) in (_abi.ERR_TIMEOUT, _abi.OK)
        assert _abi.rsim_server_wait(srv, t0, 120000) in (_abi.OK, _abi.ERR_NOT_FOUND)
        assert _abi.rsim_server_wait(srv, t2, 60000) == _abi.ERR_NONFINITE
        assert _abi.rsim_server_wait(srv, 987654, 10) == _abi.ERR_NOT_FOUND
        st = _abi.rsim_server_stats_get(srv)
        assert st.cancelled == 1 and st.failed == 1
    finally:
        _abi.rsim_server_destroy(srv)


def test_autotune_caches_plan(env, tmp_path):
    torch, _abi, device, ctx = env
    from paper_2307_09226_gb300 import device as dev
    cache = tmp_path / "tune.json"
    os.environ["RSIM_TUNE_CACHE"] = str(cache)
    try:
        c2 = dev.Context(0)
        f = synth.parity_frame(seed=7, M=2, N=4, Ns=128, L=64, n_az=64, n_el=64)
        plan = _abi.rsim_autotune(c2.h, f.radar, f.pixels.P, _abi.TIER_SPLIT_FP16)
        assert plan.tuned == 1 and 1 <= plan.splits <= 64
        got = _abi.rsim_get_plan(c2.h, f.radar, f.pixels.P, _abi.TIER_SPLIT_FP16)
        assert got.as_dict() == plan.as_dict()
        data = json.loads(cache.read_text())
        assert [plan.splits, plan.grid, plan.tile_n, plan.group_chunks] in data.values()
        cube = c2.synth(f.radar, dev.upload(f), "split_fp16").cpu().numpy()
        assert oracle.rel_l2(cube, oracle.cube_separable(f.radar, f.pixels)) <= 2e-5
        c2.close()
        c3 = dev.Context(0)  # a new context reads the cache file
        got3 = _abi.rsim_get_plan(c3.h, f.radar, f.pixels.P, _abi.TIER_SPLIT_FP16)
        assert got3.tuned == 1 and got3.as_dict() == plan.as_dict()
        c3.close()
    finally:
        os.environ.pop("RSIM_TUNE_CACHE", None)


@pytest.mark.parametrize("tier", ["split_fp16", "split_bf16", "fp32"])
def test_autotune_picks_tile_shapes_per_bucket(env, tier):
    """The tuner chooses the tile per shape: L = 40 allows only a 40-column tile, L = 256
    a 64- or 128-column tile (tensor tiers); the FP32 tier picks a 64- or 128-row n tile.
    Each tuned plan serves its whole pixel-count bucket and passes parity."""
    torch, _abi, device, ctx = env
    from paper_2307_09226_gb300 import device as dev
    c = dev.Context(0)
    try:
        chosen = {}
        for L in (40, 256):
            f = synth.parity_frame(seed=50 + L, M=2, N=4, Ns=128, L=L, n_az=60, n_el=50)  # P = 3000
            plan = _abi.rsim_autotune(c.h, f.radar, f.pixels.P, _abi.TIERS[tier])
            chosen[L] = plan.as_dict()
            print(tier, L, chosen[L])
            if tier == "fp32":
                assert plan.tile_n in (64, 128) and plan.group_chunks == 0
            else:
                assert plan.tile_n == (40 if L == 40 else plan.tile_n) and plan.tile_n in (40, 64, 128)
                assert 1 <= plan.group_chunks <= 40
            # the bucket (2049..4096 pixels) shares the plan; the next bucket does not
            same = _abi.rsim_get_plan(c.h, f.radar, 4096, _abi.TIERS[tier])
            assert same.as_dict() == plan.as_dict()
            other = _abi.rsim_get_plan(c.h, f.radar, 4097, _abi.TIERS[tier])
            assert other.tuned == 0
            ref = oracle.cube_separable(f.radar, f.pixels)
            got = c.synth(f.radar, dev.upload(f), tier).cpu().numpy()
            assert c.sync_status() == _abi.OK
            assert oracle.rel_l2(got, ref) <= TOL[tier]
        if tier != "fp32":
            assert chosen[40]["tile_n"] == 40 and chosen[256]["tile_n"] in (64, 128)
    finally:
        c.close()


def test_batch_runs_the_tuned_plan_of_its_largest_frame(env):
    """A batch takes the plan of its largest frame's shape bucket: after tuning that bucket
    (here pinned to a non-default tile and group length), every frame of an uneven batch
    equals the same frame alone under the same plan, bit for bit, and meets the oracle."""
    torch, _abi, device, ctx = env
    from paper_2307_09226_gb300 import device as dev
    c = dev.Context(0)
    try:
        radar = Radar(M=2, N=4, Ns=128, L=136)
        frames = [synth.random_frame(radar, a, b, seed=70 + i, mask_frac=0.3)
                  for i, (a, b) in enumerate([(80, 60), (60, 50), (80, 64)])]
        P = max(f.P for f in frames)  # 5120: bucket 4097..8192
        _abi.rsim_set_plan(c.h, radar, P, _abi.TIER_SPLIT_FP16, splits=3, tile_n=64, group_chunks=17)
        assert _abi.rsim_get_plan(c.h, radar, 3000, _abi.TIER_SPLIT_FP16).tile_n != 64  # another bucket
        pxs = [dev.upload(f) for f in frames]
        cubes = c.synth_batch(radar, pxs, "split_fp16")
        assert c.sync_status() == _abi.OK
        for f, px, cb in zip(frames, pxs, cubes):
            got = cb.cpu().numpy()
            # alone, each frame's own bucket: pin the same plan there so the kernels match
            _abi.rsim_set_plan(c.h, radar, f.P, _abi.TIER_SPLIT_FP16, splits=3, tile_n=64, group_chunks=17)
            alone = c.synth(radar, px, "split_fp16").cpu().numpy()
            assert np.array_equal(got, alone)
            assert oracle.rel_l2(got, oracle.cube_separable(radar, f)) <= 2e-5
    finally:
        c.close()


@pytest.mark.parametrize("tier", ["split_fp16", "split_bf16", "bf16"])
@pytest.mark.parametrize("tile_n,group", [(8, 1), (16, 7), (64, 40), (128, 0), (24, 0)])
def test_pinned_tile_shapes_pass_parity(env, tier, tile_n, group):
    """Every column tile (N = 2 NT from 16 to 256) and group length the plan allows gives
    a cube within the tier's bar, on a ragged frame with two or more column tiles."""
    torch, _abi, device, ctx = env
    f = synth.parity_frame(seed=61, M=2, N=3, Ns=96, L=136, n_az=71, n_el=70)
    if tier == "bf16" and group == 0:
        group = 384
    _abi.rsim_set_plan(ctx.h, f.radar, f.pixels.P, _abi.TIERS[tier], splits=3, tile_n=tile_n,
                       group_chunks=group)
    got_plan = _abi.rsim_get_plan(ctx.h, f.radar, f.pixels.P, _abi.TIERS[tier])
    assert got_plan.tile_n == tile_n and got_plan.splits == 3
    ref = oracle.cube_separable(f.radar, f.pixels)
    got = ctx.synth(f.radar, device.upload(f), tier).cpu().numpy()
    assert ctx.sync_status() == _abi.OK
    err = oracle.rel_l2(got, ref)
    print(tier, tile_n, group, f"{err:.3e}")
    assert err <= TOL[tier]


def test_fp32_tile_64_passes_parity_and_bad_plans_are_rejected(env):
    torch, _abi, device, ctx = env
    f = synth.parity_frame(seed=62, M=1, N=3, Ns=200, L=72, n_az=90, n_el=40)
    _abi.rsim_set_plan(ctx.h, f.radar, f.pixels.P, _abi.TIER_FP32, splits=2, tile_n=64)
    got = ctx.synth(f.radar, device.upload(f), "fp32").cpu().numpy()
    assert ctx.sync_status() == _abi.OK
    assert oracle.rel_l2(got, oracle.cube_separable(f.radar, f.pixels)) <= 2e-5
    for kw in (dict(tile_n=96), dict(variant=2)):
        with pytest.raises(_abi.RsimError) as e:
            _abi.rsim_set_plan(ctx.h, f.radar, f.pixels.P, _abi.TIER_FP32, splits=2, **kw)
        assert e.value.status == _abi.ERR_INVALID_ARG
    for kw in (dict(tile_n=136), dict(tile_n=12), dict(group_chunks=41), dict(variant=2)):
        with pytest.raises(_abi.RsimError) as e:
            _abi.rsim_set_plan(ctx.h, f.radar, f.pixels.P, _abi.TIER_SPLIT_FP16, splits=2, **kw)
        assert e.value.status == _abi.ERR_INVALID_ARG
