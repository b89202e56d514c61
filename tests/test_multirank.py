"""The N > 1 path of bench.py is replicas only: each rank advances its own
copy of the workload and only the timed region (maximum over ranks) and the
units processed (sum over ranks) are reduced.  Checked here with two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t, u = bench.job_time_and_units(0.5 + rank, 1000.0 * (rank + 1))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_time_max_and_units_sum():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    manager = mp.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (1.5, 3000.0) and out[1] == (1.5, 3000.0)


def test_single_process_needs_no_process_group():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_and_units(0.25, 7.0) == (0.25, 7.0)
