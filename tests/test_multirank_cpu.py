"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks each build their own batch
(weak scaling: no data-path collective) and the timing is the max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    r, w, local = bench.dist_env()
    seed = None if r == 0 else bench.shard_seed(1002, r)
    wl = synth.workload("square4", F=3, seed=seed)
    t_local = [1.0 + r, 10.0 - r]
    t_max = bench.reduce_max(t_local, w, torch.device("cpu"))
    dist.barrier()
    out[rank] = (r, w, float(wl["frames"].sum()), t_max)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_frames_and_take_max_timing():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    r0, r1 = out[0], out[1]
    assert (r0[0], r0[1]) == (0, 2) and (r1[0], r1[1]) == (1, 2)
    assert r0[2] != r1[2], "each rank must process its own batch of frames"
    assert r0[3] == r1[3] == [2.0, 10.0]  # element-wise max over ranks
