"""Host logic of multi-GPU replicas, exercised by two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2005_12338_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = [replicas.rank_seed(rank, k) for k in range(3)]
        t = replicas.max_over_ranks(1.5 + rank)  # rank 1 is the slowest
        out[rank] = (seeds, t, replicas.job_throughput(19200, 3, world, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_on_cpu():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    s0, t0, v0 = res[0]
    s1, t1, v1 = res[1]
    assert set(s0).isdisjoint(s1)          # independent draws per rank
    assert t0 == t1 == 2.5                 # both see the slowest rank's time
    assert v0 == v1 == pytest.approx(19200 * 3 * 2 / 2.5)


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.rank_seed(0, 5) == 5
    with pytest.raises(ValueError):
        replicas.rank_seed(0, replicas.RANK_SEED_STRIDE)
