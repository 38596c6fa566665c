"""The replica path's host logic with two gloo ranks on CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2103_14921_gb300 import replicas
    ws, r, lr = replicas.world()
    secs = 2.0 + rank                       # rank 1 is the slow one
    value, t = replicas.job_throughput(units_per_rank=16.0, seconds_this_rank=secs)
    out[rank] = (ws, r, lr, value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        ws, r, lr, value, t = out[rank]
        assert (ws, r, lr) == (2, rank, rank)
        assert t == 3.0                      # max over ranks
        assert abs(value - 2 * 16.0 / 3.0) < 1e-12


def test_single_process_is_identity():
    from paper_2103_14921_gb300 import replicas
    value, t = replicas.job_throughput(10.0, 4.0)
    assert t == 4.0 and value == 2.5
