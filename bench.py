"""Benchmark of TDM-MIMO data-cube synthesis on GB300 (one JSON line on stdout).

Workload (default): one frame of M=3 Tx x N=4 Rx (12 virtual channels), N_s=256,
L=128, 256x256 pixels with 30% background misses (complex64 out), seeded
synthetic buffers.  A step is one whole synthesis through the library: valid-pixel
compaction, FP64 pixel-to-path phases, the contraction over pixels (tier chosen by
--tier; default the fastest tier within the 2e-5 accuracy bar) and the ordered split
reduction.  The metric is path-samples per second, a path-sample being one
(valid pixel, channel, fast-time, slow-time) term of the sum.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--tier T] [--impl reference]

--impl reference times the CPU FP64 oracle (the only other implementation of this
path) on a bounded sample of the same workload.  Under torchrun each rank runs its
own frame (frames are independent: weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
ACCURACY_TIERS = ("split_fp16", "split_bf16", "fp32")  # within 2e-5 of the FP64 oracle


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device="cpu") -> float:
    """Max of a per-rank time over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(samples_per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput in Gpath-samples/s: every rank synthesises its own frame
    (independent units), so the job's work is world x steps frames in the slowest
    rank's time."""
    return samples_per_rank * world * steps / (max_ms * 1e-3) / 1e9


def rank_seed(rank: int) -> int:
    """Seed of the frame a rank synthesises (rank 0 runs the reference frame)."""
    return 2 + rank


class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def _cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def _valid_count(px) -> int:
    """Pixels that hit something: non-zero complex strength."""
    import numpy as np
    return int(((np.asarray(px.sigma_re) != 0) | (np.asarray(px.sigma_im) != 0)).sum())


def _rel_l2(got, ref) -> float:
    """Normwise relative L2 error over all entries."""
    import numpy as np
    got = np.asarray(got, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((got - ref).ravel())
    return float(num / den) if den > 0 else float(num)


def _cpu_reference(frame):
    """The CPU-baseline leg: the oracle (FP64 separable form) on the whole frame, timed on
    the host cores.  Its cube is also the reference of the GPU tiers' accuracy.  Returns
    (cube, path-samples/s, cores, sample)."""
    import oracle
    r = frame.radar
    t0 = time.perf_counter()
    ref = oracle.cube_separable(r, frame.pixels)
    dt = time.perf_counter() - t0
    pv = _valid_count(frame.pixels)
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return ref, pv * r.V * r.Ns * r.L / dt, cores, f"{r.V} of {r.V} channels x all {pv} valid pixels x {r.Ns}x{r.L}"


def _cpu_one_core(frame):
    """The oracle on one host core: channel 0 of the frame in a child process whose BLAS
    and OpenMP pools hold one thread.  Returns (path-samples/s, sample, seconds)."""
    import subprocess
    r = frame.radar
    pv = _valid_count(frame.pixels)
    code = ("import sys, time; sys.path.insert(0, %r); import oracle; from paper_2307_09226_gb300 import synth; "
            "f = synth.config2(); t = time.perf_counter(); oracle.cube_separable(f.radar, f.pixels, channels=[0]); "
            "print(time.perf_counter() - t)" % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        dt = float(out.stdout.strip().splitlines()[-1])
    except Exception:
        return None, None, None
    return pv * r.Ns * r.L / dt, f"1 of {r.V} channels x all {pv} valid pixels x {r.Ns}x{r.L}", dt


def _roofline(tier, prof_contract_ms, launches, samples, peaks, peak_kind):
    """Roofline of the contraction kernel (its own CUDA-event time, without the operand
    builder): algorithmic work is 8 real flops (one complex MAC) per path-sample."""
    avg_ms = prof_contract_ms / max(launches, 1)
    flops = 8.0 * samples
    achieved = flops / (avg_ms * 1e-3) / 1e12
    if tier == "fp32":
        # FP32 FMA pipe: 152 SMs x 128 lanes x 2 flops x max SM clock
        clk = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * clk * 1e6 / 1e12
        return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "direct_sum", "kernel_ms": round(avg_ms, 5),
                "peak_source": f"FP32 FMA: 152 SM x 128 lanes x 2 x {clk:.0f} MHz"}
    peak = peaks["bf16_tflops"]
    executed = flops * (3 if tier.startswith("split") else 1) / (avg_ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": round(achieved, 3), "peak": peak, "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": None, "kernel": "umma_contract",
            "kernel_ms": round(avg_ms, 5), "executed_tflops": round(executed, 3),
            "peak_source": f"bf16 dense burst ({peak_kind})"}


def _cpu_sample(frame, target_s=12.0):
    """Time the CPU oracle on a bounded sample of the frame: whole channels of the full
    pixel set, as many as fit in ~target_s seconds."""
    import numpy as np
    import oracle
    from paper_2307_09226_gb300 import synth  # noqa: F401
    r = frame.radar
    pv = _valid_count(frame.pixels)
    t0 = time.perf_counter()
    oracle.cube_separable(r, frame.pixels, channels=[0])
    one = time.perf_counter() - t0
    nch = max(1, min(r.V, int(target_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    oracle.cube_separable(r, frame.pixels, channels=list(range(nch)))
    dt = time.perf_counter() - t0
    samples = pv * nch * r.Ns * r.L
    try:
        import threadpoolctl  # noqa: F401
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return samples / dt, cores, f"{nch} of {r.V} channels x all {pv} valid pixels x {r.Ns}x{r.L}", dt


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from paper_2307_09226_gb300 import synth
    frame = synth.config2()
    for _ in range(args.warmup):
        _cpu_sample(frame, target_s=2.0)
    vals = []
    t0 = time.perf_counter()
    info = None
    for _ in range(args.steps):
        v, cores, sample, dt = _cpu_sample(frame, target_s=6.0)
        vals.append(v)
        info = (cores, sample)
    total = time.perf_counter() - t0
    value = statistics.median(vals) / 1e9
    line = {"impl": "reference", "metric": "cube synth Gpath-samples/s at rel err<=2e-5 vs FP64",
            "value": value, "unit": "Gpath-samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / max(args.steps, 1) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": frame.meta["workload"], "tier": "oracle_fp64_separable",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "Gpath-samples/s", "cores": info[0],
                             "kind": "oracle", "sample": info[1]},
            "e2e": {"value": value, "unit": "Gpath-samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import __graft_entry__
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_2307_09226_gb300 import _abi, device, synth

    frame = synth.config2(seed=rank_seed(rank))  # each rank its own frame (independent units)
    radar = frame.radar
    ctx = device.Context(local)
    px = device.upload(frame)
    pv = _valid_count(frame.pixels)
    samples = pv * radar.V * radar.Ns * radar.L

    tiers = [args.tier] if args.tier else list(ACCURACY_TIERS)
    # the CPU-baseline leg (rank 0): the oracle timed on the host cores; its cube is the
    # FP64 reference of the accuracy check, outside the timed region
    ref = cpu_v = cores = sample = None
    if rank == 0:
        ref, cpu_v, cores, sample = _cpu_reference(frame)
    errs = {}
    usable = []
    for t in tiers:
        try:
            # every tier runs (and is checked with) the tuned plan of the frame's shape bucket
            ensure_tuned(ctx, radar, frame.pixels.P, t)
            cube = ctx.synth(radar, px, t)
            st = ctx.sync_status()
        except _abi.RsimError as e:
            if e.status == _abi.ERR_UNSUPPORTED:
                continue
            raise
        if st != _abi.OK:
            raise RuntimeError(f"tier {t}: status {st}")
        if ref is not None:
            errs[t] = _rel_l2(cube.cpu().numpy(), ref)
        usable.append(t)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def time_tier(t, steps, warmup, profile=False):
        cube = device.cube_tensor(radar)
        for _ in range(warmup):
            ctx.synth(radar, px, t, cube=cube)
        torch.cuda.synchronize()
        if profile:
            _abi.rsim_profile_enable(ctx.h, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for i in range(steps):
            flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
            ev[i][0].record(stream)
            ctx.synth(radar, px, t, cube=cube)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = _abi.rsim_profile_read(ctx.h) if profile else None
        if profile:
            _abi.rsim_profile_enable(ctx.h, False)
        return ms, prof

    # pick the fastest tier within the accuracy bar (short probe), then time it
    if len(usable) > 1:
        probe = {t: statistics.median(time_tier(t, 5, 2)[0]) for t in usable
                 if errs.get(t, 0.0) <= 2e-5}
        tier = min(probe, key=probe.get)
    else:
        tier = usable[0]
        probe = {}

    sampler = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.25)
    ms, _ = time_tier(tier, args.steps, args.warmup)
    clocks = sampler.stop()
    # stage times and launch counts from a second run of the same steps with the library's
    # stage events on (the events sit between the kernels of a call, so this run is not
    # the timed one)
    _, prof = time_tier(tier, args.steps, 2, profile=True)
    step_ms = max_over_ranks(sum(ms), device="cuda")
    value = weak_scaling_value(samples, ws, args.steps, step_ms)

    # end to end through the C ABI on host buffers (rsim_synth_host): pinned host pixel
    # arrays are copied in, the cube synthesised and copied back to pinned host memory by
    # the library, every step inside the timed region
    host = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            for k, a in zip(device.FIELDS, frame.pixels.arrays())}
    out_host = device.cube_tensor(radar, device="cpu").pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_host.numel() * out_host.element_size()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.synth_host(radar, host, tier, cube=out_host, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(sum(e2e_ms), device="cuda")
    e2e_value = weak_scaling_value(samples, ws, args.steps, e2e_total)

    if rank == 0:
        peaks, kind = _peaks()
        roof = _roofline(tier, prof.contract_ms - prof.operand_ms, prof.calls, samples, peaks, kind)
        traffic = _load_traffic(tier)
        if traffic is not None:
            roof["traffic"] = traffic
        if roof.get("kernel") == "umma_contract":
            # the device's measured rate on the contraction's own MMA instruction: the
            # ceiling of the executed rate (the cuBLAS peak above also spends time outside
            # its MMAs, so a kernel can execute above it)
            mma = _abi.rsim_measure_mma_rate(ctx.h) / 1e12
            roof["mma_rate_tflops"] = round(mma, 1)
            roof["executed_frac_of_mma_rate"] = round(roof["executed_tflops"] / mma, 4)
        one_v, one_sample, _ = _cpu_one_core(frame)
        batch = run_batch(ctx, tier, steps=max(3, min(args.steps, 10)), warmup=3) if not args.no_extras else None
        serving = run_serving(ctx) if not args.no_extras else None
        raycast = run_raycast(ctx, tier) if not args.no_extras else None
        nufft = run_nufft(ctx, frame, px, ref, args.steps, args.warmup) if not args.no_extras else None
        if nufft is not None:
            nufft["speedup_vs_headline_tier"] = round(step_ms / args.steps / nufft["ms_per_step"], 3)
            # config 4 (64 walking frames) through the NUFFT tier as well
            nb = run_batch(ctx, "nufft", steps=max(3, min(args.steps, 10)), warmup=3)
            nufft["batch"] = {k: nb[k] for k in ("workload", "frames", "ms_per_batch", "value", "unit", "doppler_time")}
        line = {
            "metric": "cube synth Gpath-samples/s at rel err<=2e-5 vs FP64",
            "value": value, "unit": "Gpath-samples/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if tier == "fp32" else
            ("fp16x2+f32acc" if tier == "split_fp16" else "bf16x2+f32acc"),
            "data": "synthetic",
            "config": {"workload": frame.meta["workload"], "tier": tier, "P": radar and frame.pixels.P,
                       "plan": _abi.rsim_get_plan(ctx.h, radar, frame.pixels.P, _abi.TIERS[tier]).as_dict(),
                       "P_valid": pv, "V": radar.V, "Ns": radar.Ns, "L": radar.L,
                       "path_samples_per_frame": samples, "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{ws}"},
            "rel_err": errs,
            "tiers_probe_ms": {k: round(v, 4) for k, v in probe.items()},
            "stage_ms": {"prep": prof.prep_ms / prof.calls, "contract": prof.contract_ms / prof.calls,
                         "operand_build": prof.operand_ms / prof.calls,
                         "reduce": prof.reduce_ms / prof.calls},
            "gpu_launches": prof.kernels,
            "roofline": roof,
            "cpu_baseline": {"value": cpu_v / 1e9, "unit": "Gpath-samples/s", "cores": cores,
                             "kind": "oracle", "sample": sample, "cpu_model": _cpu_model(),
                             "host_cores": os.cpu_count(),
                             "one_core": None if one_v is None else
                             {"value": one_v / 1e9, "unit": "Gpath-samples/s", "sample": one_sample}},
            "cube_write_gbs": round(radar.V * radar.Ns * radar.L * 8 / (step_ms / args.steps * 1e-3) / 1e9, 2),
            "e2e": {"value": e2e_value, "unit": "Gpath-samples/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clocks,
            "batch": batch,
            "serving": serving,
            "raycast": raycast,
            "nufft": nufft,
        }
        print(json.dumps(line))
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


KERNEL_SOURCES = {"fp32": "k_direct.cu", "split_fp16": "k_umma.cu", "split_bf16": "k_umma.cu",
                  "bf16": "k_umma.cu", "fp16": "k_umma.cu"}


def kernel_source_hash(tier):
    import hashlib
    p = os.path.join(ROOT, "paper_2307_09226_gb300", "csrc", KERNEL_SOURCES[tier])
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


def _load_traffic(tier):
    """DRAM bytes per launch of the contraction kernel, from the ncu capture recorded in
    profiles/traffic.txt (lines: tier  source-hash  bytes).  None when nothing was
    recorded for this tier or the kernel source has changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    want = kernel_source_hash(tier)
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 3 and not line.startswith("#") and parts[0] == tier and parts[1] == want:
                return float(parts[2])
    return None


def ensure_tuned(ctx, radar, P, tier):
    """Tune the plan of (radar, P, tier)'s shape bucket unless a tuned plan is already
    cached (RSIM_TUNE_CACHE, which main() points at a file in the temp folder by default,
    so a second run of the same command, e.g. under a profiler, reuses the plans)."""
    from paper_2307_09226_gb300 import _abi
    if not _abi.rsim_get_plan(ctx.h, radar, P, _abi.TIERS[tier]).tuned:
        _abi.rsim_autotune(ctx.h, radar, P, _abi.TIERS[tier])


def run_batch(ctx, tier, steps, warmup):
    """Config 4: 64 walking-pedestrian frames (uneven valid-pixel counts) in one
    rsim_synth_batch call per step; inputs resident, L2 flushed between steps."""
    import numpy as np
    import torch
    from paper_2307_09226_gb300 import device, synth
    frames = synth.walking_batch(n_frames=64)
    radar = frames[0].radar
    pxs = [device.upload(f) for f in frames]
    cubes = [device.cube_tensor(radar) for _ in frames]
    pvs = [_valid_count(f.pixels) for f in frames]
    samples = sum(pvs) * radar.V * radar.Ns * radar.L
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    # the batch runs with the tuned plan of its shape bucket (the plan of its largest frame)
    from paper_2307_09226_gb300 import _abi
    P = max(f.pixels.P for f in frames)
    plan = None
    if tier in _abi.TIERS and tier != "nufft":
        ensure_tuned(ctx, radar, P, tier)
        plan = _abi.rsim_get_plan(ctx.h, radar, P, _abi.TIERS[tier]).as_dict()
    for _ in range(warmup):
        ctx.synth_batch(radar, pxs, tier, cubes=cubes)
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.synth_batch(radar, pxs, tier, cubes=cubes)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    # Section III's Doppler-time method on the batch: range-Doppler maps, max-power
    # velocity per CPI with a zero-Doppler notch (the wall is static), E_velo vs torso
    from paper_2307_09226_gb300 import _abi
    power = torch.empty((len(frames), radar.Ns, radar.L), dtype=torch.float32, device="cuda")
    vest = torch.empty(len(frames), dtype=torch.float32, device="cuda")
    _abi.rsim_range_doppler(ctx.h, radar, cubes, power, vest, skip_static=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    _abi.rsim_range_doppler(ctx.h, radar, cubes, power, vest, skip_static=True)
    b.record()
    torch.cuda.synchronize()
    truth = [f.meta["v_torso"] for f in frames]
    return {"workload": "walking-64x256x256-V12-Ns256-L128", "tier": tier, "plan": plan, "frames": len(frames),
            "P_valid_min": min(pvs), "P_valid_max": max(pvs), "ms_per_batch": round(t, 4),
            "value": samples / (t * 1e-3) / 1e9, "unit": "Gpath-samples/s", "steps": steps,
            "doppler_time": {"ms_64_frames": round(a.elapsed_time(b), 4),
                             "e_velo_m_s": round(float(np.mean(np.abs(vest.cpu().numpy() - np.asarray(truth)))), 4)}}


def run_nufft(ctx, frame, px, ref, steps, warmup):
    """The NUFFT form of the same config-2 frame (the alternative to the tensor-core
    contraction): accuracy against the FP64 oracle, device time per frame with the L2
    flushed between steps, the stage split, and the CPU NUFFT reference on two channels."""
    import torch
    import oracle.nufft as nu
    from paper_2307_09226_gb300 import _abi, device
    radar = frame.radar
    pv = _valid_count(frame.pixels)
    cube = device.cube_tensor(radar)
    ctx.synth(radar, px, "nufft", cube=cube)
    err = _rel_l2(cube.cpu().numpy(), ref)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        ctx.synth(radar, px, "nufft", cube=cube)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record()
        ctx.synth(radar, px, "nufft", cube=cube)
        ev[i][1].record()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    _abi.rsim_profile_enable(ctx.h, True)
    for i in range(steps):
        flush.fill_(float(i))
        ctx.synth(radar, px, "nufft", cube=cube)
    prof = _abi.rsim_profile_read(ctx.h)
    _abi.rsim_profile_enable(ctx.h, False)
    samples = pv * radar.V * radar.Ns * radar.L
    t = sum(ms) / len(ms)
    # spreading (the dominant kernel): 49 taps x (re, im) x two words = 196 shared atomic
    # lane-operations per (channel, point) record, against the rate this device performs
    # such atomics (measured by the library's probe on the same GPU), with the derived
    # one-wavefront-per-clock figure beside it
    spread_ms = prof.main_ms / prof.calls
    lane_ops = 196.0 * radar.V * pv
    peaks, _ = _peaks()
    clk = peaks.get("sm_max_mhz", 2070.0)
    derived = 152 * 32 * clk * 1e6 / 1e12
    measured = _abi.rsim_measure_smem_atomics(ctx.h) / 1e12
    achieved = lane_ops / (spread_ms * 1e-3) / 1e12
    roof = {"bound": "smem", "kernel": "nu_spread", "achieved": round(achieved, 3), "peak": round(measured, 3),
            "unit": "T lane-op/s", "frac": round(achieved / measured, 4), "kernel_ms": round(spread_ms, 5),
            "peak_source": "measured: non-returning conflict-free 32-bit shared atomics at the spreading "
                           "kernel's occupancy (rsim_measure_smem_atomics, this GPU)",
            "derived_peak": round(derived, 3), "frac_of_derived": round(achieved / derived, 4),
            "derived_source": f"one 32-lane wavefront per clock: 152 SM x 32 lanes x {clk:.0f} MHz",
            "algorithmic": "196 shared atomic lane-operations per (channel, point) record"}
    # the accuracy each gridding kernel width buys, and its time (the same frame)
    from dataclasses import replace as _replace
    widths = {}
    for w in (4, 5, 6, 7, 8):
        rw = _replace(radar, nufft_width=w)
        for _ in range(3):
            ctx.synth(rw, px, "nufft", cube=cube)
        wms = []
        for i in range(10):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.synth(rw, px, "nufft", cube=cube)
            b.record()
            torch.cuda.synchronize()
            wms.append(a.elapsed_time(b))
        widths[w] = {"ms_per_step": round(statistics.median(wms), 4),
                     "rel_err": _rel_l2(cube.cpu().numpy(), ref)}
    t0 = time.perf_counter()
    nu.cube_nufft(radar, frame.pixels, w=7, channels=[0, 1])
    cpu_s = time.perf_counter() - t0
    return {"workload": frame.meta["workload"], "tier": "nufft", "kernel_width": 7,
            "value": samples / (t * 1e-3) / 1e9, "unit": "Gpath-samples/s", "ms_per_step": round(t, 4),
            "rel_err": err, "steps": steps, "gpu_launches": prof.kernels,
            "stage_ms": {"prep": prof.prep_ms / prof.calls, "nufft": prof.contract_ms / prof.calls,
                         "binning": prof.operand_ms / prof.calls, "spreading": spread_ms,
                         "ffts": (prof.contract_ms - prof.operand_ms) / prof.calls - spread_ms},
            "roofline": roof,
            "by_kernel_width": widths,
            "speedup_vs_headline_tier": None,
            "cpu_baseline": {"value": pv * 2 * radar.Ns * radar.L / cpu_s / 1e9, "unit": "Gpath-samples/s",
                             "cores": 1, "kind": "oracle",
                             "sample": "CPU NUFFT reference (numpy FP64, width 7), channels 0-1 of the frame"}}


def run_raycast(ctx, tier, steps=10, warmup=3):
    """The rendering step on the GPU: a 256x256 render of a random 12-primitive scene
    (rays per second, device time, L2 flushed between steps) against the FP64 oracle on
    the host; then Section III's walking experiment on rendered frames: 64 frames of the
    analytic pedestrian (one lap of 100 frames at 24 Hz on a 3 m circle, so 4.52 m/s)
    rendered, synthesised in one batch call and turned into a Doppler-time trace, with
    E_velo against each frame's torso closing speed."""
    import numpy as np
    import torch
    import oracle.raycast as rc
    from paper_2307_09226_gb300 import _abi, device, synth
    n_az, n_el = 256, 256
    # scenes are marshalled to rsim_primitive arrays once, outside the device-timed region
    scene = _abi.primitives_array(synth.random_scene(seed=7, n_prims=12))
    out = {k: torch.empty(n_az * n_el, dtype=torch.float32, device="cuda") for k in device.FIELDS}
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        ctx.raycast(scene, n_az, n_el, synth.CAMERA_FOV, out=out)
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.raycast(scene, n_az, n_el, synth.CAMERA_FOV, out=out)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    t0 = time.perf_counter()
    rc.raycast(synth.random_scene(seed=7, n_prims=12), n_az, n_el, *synth.CAMERA_FOV)
    cpu_s = time.perf_counter() - t0
    rays = n_az * n_el
    # walking experiment on rendered frames
    radar = synth.Radar(M=3, N=4, Ns=256, L=128)
    F = 64
    scenes = [synth.walking_scene(f) for f in range(F)]
    scene_arrays = [_abi.primitives_array(sc) for sc, _ in scenes]
    pxs = [{k: torch.empty(n_az * n_el, dtype=torch.float32, device="cuda") for k in device.FIELDS}
           for _ in range(F)]
    cubes = [device.cube_tensor(radar) for _ in range(F)]
    power = torch.empty((F, radar.Ns, radar.L), dtype=torch.float32, device="cuda")
    vest = torch.empty(F, dtype=torch.float32, device="cuda")

    def pipeline():
        for sc, px in zip(scene_arrays, pxs):
            ctx.raycast(sc, n_az, n_el, synth.CAMERA_FOV, out=px)
        ctx.synth_batch(radar, pxs, tier, cubes=cubes)
        _abi.rsim_range_doppler(ctx.h, radar, cubes, power, vest, skip_static=True)

    pipeline()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pipeline()
    b.record()
    torch.cuda.synchronize()
    truth = np.array([tr["closing_speed"] for _, tr in scenes])
    est = vest.cpu().numpy()
    return {"workload": f"random-12-primitives-{n_az}x{n_el}", "ms": round(t, 4),
            "value": rays / (t * 1e-3) / 1e9, "unit": "Grays/s",
            "ray_primitive_tests_per_s": rays * scene.size / (t * 1e-3), "steps": steps,
            "cpu_oracle": {"ms": round(cpu_s * 1e3, 2), "kind": "oracle", "cores": 1,
                           "sample": "the same render, numpy FP64"},
            "walking": {"frames": F, "pixels": f"{n_az}x{n_el}", "tier": tier,
                        "ms_render_synth_doppler": round(a.elapsed_time(b), 4),
                        "e_velo_m_s": round(float(np.mean(np.abs(est - truth))), 4),
                        "speed_m_s": round(scenes[0][1]["speed"], 3)}}


def run_serving(ctx, tune_budget_s=45.0, slots=None, schedule=None):
    """Config 5: Poisson stream of mixed requests (M 2-4, N 4-12, Ns 128-512, L 64-256,
    64^2..512^2 pixels, FP32 and split-BF16 tiers) into the continuous-batching server:
    n_warmup requests, a new tally, then n_requests measured; latency is submit ->
    completion.  Offered loads 0.5 and 0.7 x the measured capacity with first-fit
    admission, and 0.7 with shortest-first admission.  The requests cycle over `pool`
    distinct frames resident on the device (a frame's previous request has finished
    before it is reused).  Before any timing, the pool's shape buckets are tuned, smallest
    estimated work first, until tune_budget_s has passed; the rest keep the default plan."""
    import numpy as np
    import torch
    from paper_2307_09226_gb300 import _abi, device, synth
    cfg = synth.load_config(5)
    n_requests, n_warmup, pool = cfg["requests"], cfg["warmup_requests"], cfg["distinct_frames"]
    slots = cfg["slots"] if slots is None else slots
    seed, age_ms, express = cfg["seed"], cfg["age_limit_ms"], cfg["express_slots"]
    reqs = synth.serving_requests(pool, seed=seed)
    frames = [synth.request_frame(r) for r in reqs]
    pxs = [device.upload(f) for f in frames]
    cubes = [device.cube_tensor(f.radar) for f in frames]
    made = [_abi.make_request(f.radar, px, _abi.TIERS[r["tier"]], cb)
            for r, f, px, cb in zip(reqs, frames, pxs, cubes)]
    # tune the shape buckets of the pool
    keys = {}
    for r, f in zip(reqs, frames):
        rd = f.radar
        key = (r["tier"], rd.V, rd.Ns, rd.L, (int(f.pixels.P) - 1).bit_length())
        work = f.pixels.P * rd.V * rd.Ns * rd.L * (10.0 if r["tier"] == "fp32" else 1.0)
        keys.setdefault(key, (work, rd, int(f.pixels.P), r["tier"]))
    t_tune = time.perf_counter()
    tuned = set()
    for key, (work, rd, P, tier) in sorted(keys.items(), key=lambda kv: kv[1][0]):
        if time.perf_counter() - t_tune > tune_budget_s:
            break
        ensure_tuned(ctx, rd, P, tier)
        tuned.add(key)
    tune_s = time.perf_counter() - t_tune
    on_tuned = sum(1 for r, f in zip(reqs, frames)
                   if (r["tier"], f.radar.V, f.radar.Ns, f.radar.L, (int(f.pixels.P) - 1).bit_length()) in tuned)
    # capacity: every pool request once, back to back, on one server slot
    srv = _abi.rsim_server_create(ctx.h, slots=1)
    t0 = time.perf_counter()
    for m in made:
        _abi.rsim_server_wait(srv, _abi.rsim_server_submit(srv, m), -1)
    alone_s = (time.perf_counter() - t0) / len(made)
    _abi.rsim_server_destroy(srv)
    rng = np.random.default_rng(seed + 1)

    def run(load, policy, n_express, n_general=None):
        rate = load / alone_s
        n_general = slots if n_general is None else n_general
        srv = _abi.rsim_server_create(ctx.h, slots=n_general, policy=policy, age_limit_ms=age_ms,
                                      express_slots=n_express)
        bad = 0

        def stream(n, first):
            nonlocal bad
            gaps = rng.exponential(1.0 / rate, n)
            tickets = {}
            due = time.perf_counter()
            for j in range(first, first + n):
                due += gaps[j - first]
                prev = tickets.pop(j - pool, None)  # the same frame's previous request
                if prev is not None:
                    bad += _abi.rsim_server_wait(srv, prev, -1) != _abi.OK
                delay = due - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[j] = _abi.rsim_server_submit(srv, made[j % pool])
            for t in tickets.values():
                bad += _abi.rsim_server_wait(srv, t, -1) != _abi.OK

        stream(n_warmup, 0)
        _abi.rsim_server_stats_reset(srv)
        stream(n_requests, n_warmup)
        st = _abi.rsim_server_stats_get(srv)
        _abi.rsim_server_destroy(srv)
        torch.cuda.synchronize()
        return {"offered_load": load, "policy": policy, "slots": n_general, "express_slots": n_express,
                "rate_req_s": round(rate, 2),
                "requests": int(st.completed),
                "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3), "mean_ms": round(st.mean_ms, 3),
                "max_ms": round(st.max_ms, 3), "p99_queue_ms": round(st.p99_queue_ms, 3),
                "max_queue_ms": round(st.max_queue_ms, 3), "overtakes": int(st.overtakes),
                "req_per_s": round(st.completed / max(st.busy_s, 1e-9), 2),
                "value": st.path_samples / max(st.busy_s, 1e-9) / 1e9, "unit": "Gpath-samples/s",
                "failed": int(st.failed) + bad, "peak_in_flight": int(st.peak_in_flight)}

    loads = cfg["offered_loads"]
    if schedule is None:
        # the configured server at each load, shortest-first at the first load, and the same
        # number of slots without express slots (all general) for comparison
        schedule = ([(x, "first_fit", express) for x in loads] + [(loads[0], "shortest_first", express)] +
                    [(loads[0], "first_fit", 0, slots + express)])
    runs = [run(*item) for item in schedule]
    head = dict(runs[0])
    head.update({"workload": cfg["workload"],
                 "warmup_requests": n_warmup, "distinct_frames": pool, "age_limit_ms": age_ms,
                 "alone_mean_ms": round(alone_s * 1e3, 3),
                 "tuning": {"buckets": len(keys), "tuned": len(tuned), "requests_on_tuned_plans": on_tuned,
                            "pool": pool, "seconds": round(tune_s, 1)},
                 "by_load_and_policy": runs})
    return head


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--tier", default=None, choices=[None, "fp32", "split_fp16", "split_bf16", "bf16", "fp16"])
    ap.add_argument("--impl", default="library", choices=["library", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batch (64 frames) and serving (Poisson mix) measurements")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    import tempfile
    os.environ.setdefault("RSIM_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "rsim_tune_cache.json"))
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
