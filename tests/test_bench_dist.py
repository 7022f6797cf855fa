"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
value is the max over ranks and the whole-job throughput sums the replicas."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slower one
    out[rank] = bench.max_over_ranks(ms, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 15.0
    import bench
    # two replicas of 1e9 nnz, 10 steps in 20 ms each -> 1000 GNNZ/s
    assert bench.whole_job_gnnz(1e9, 10, 20.0, 2) == pytest.approx(1000.0)


def test_single_rank_max_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, device="cpu") == 3.5
