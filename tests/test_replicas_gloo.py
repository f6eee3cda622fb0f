"""Multi-rank path of bench.py on CPU: two gloo ranks, no GPU.

With N > 1 every rank runs an independent replica of the workload (the step
has no data-path collective; weak scaling).  The only exchange is the timing:
all ranks agree on the slowest rank's step time, and the whole-job throughput
is N replicas' node updates over that time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    local_time = 0.010 * (rank + 1)  # rank 1 is the slowest
    t = bench.slowest_rank_time(local_time, dist, torch, "cpu")
    out[rank] = (t, bench.whole_job_mlups(2_097_152, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(0.020)
    assert res[0][1] == pytest.approx(2 * 2_097_152 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_time(0.5, None, torch, "cpu") == 0.5
    assert bench.whole_job_mlups(1000, 1, 0.001) == pytest.approx(1.0)
