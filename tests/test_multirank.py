"""The N > 1 path of bench.py (replicas only): each rank times its own solve and the job time
is the maximum over ranks.  Two gloo ranks on the CPU exercise the reduction and the
aggregation without a GPU."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank                    # rank 1 is the slow replica
    m = bench.max_over_ranks(ms)
    out[rank] = (m, bench.job_throughput(1000, m, world), bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_throughput():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        m, thr, env = out[r]
        assert m == 150.0
        assert thr == pytest.approx(2 * 1000 / 0.150)
        assert env == (2, r, 0)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(100, 1000.0, 1) == pytest.approx(100.0)
