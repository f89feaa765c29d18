"""The multi-GPU path of bench.py on CPU: two gloo ranks (world size 2).

Frames are independent, so ranks share nothing on the data path: each draws its own
frame, and only the timing is combined (max over ranks, weak scaling)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2307_09226_gb300 import synth
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    f = synth.config2(seed=bench.rank_seed(rank))
    out[rank] = (t, float(np.nansum(f.pixels.range[np.isfinite(f.pixels.range)])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_draw_distinct_frames():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]


def test_weak_scaling_value():
    import bench
    # 2 ranks x 3 steps x 1e9 samples in 1.5 s -> 4 Gpath-samples/s
    assert bench.weak_scaling_value(10 ** 9, 2, 3, 1500.0) == pytest.approx(4.0)
    assert bench.max_over_ranks(3.5) == 3.5
