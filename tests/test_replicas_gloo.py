"""The multi-GPU form of the bench is replicas (independent droplet instances, one per rank, no collective on
the data path): its host logic -- per-rank instance seeds and the whole-job rate from the slowest rank --
checked with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_1907_00890_gb300 import synth
    r, w, local = bench.dist_env()
    c = synth.config_droplet(16, seed_offset=r)
    ms_local = 2.0 + 3.0 * r  # rank 1 is the slow one
    ms_max, value = bench.job_rate(ms_local, int(np.prod(c["n"])), 2, w, torch.device("cpu"))
    out[rank] = (r, w, local, ms_max, value, float(c["u"].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert (r0[0], r0[1], r0[2]) == (0, 2, 0) and (r1[0], r1[1], r1[2]) == (1, 2, 1)
    cells = 16 ** 3
    for r in (r0, r1):
        assert r[3] == pytest.approx(5.0)                           # the slowest rank's time on every rank
        assert r[4] == pytest.approx(2 * cells * 2 / 5e-3 / 1e6)    # all ranks' cells over that time
    assert r0[5] != r1[5]                                           # each rank solves its own instance
