"""The replica path of bench.py at world size 2 over gloo on the CPU: the
step time is the slowest rank's, the units are summed over ranks, and the
oracle arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.reduce_max(10.0 + 5.0 * rank)          # rank 1 is the slow one
    units = bench.reduce_sum(1e9 * (rank + 1))       # different workloads per rank
    value = bench.job_value(units, ms)
    # the oracle arm: every rank but 0 returns at once, without building anything
    class A:
        pass
    rc = bench.run_reference(A()) if rank != 0 else 0
    dist.destroy_process_group()
    out.put((rank, ms, units, value, rc))


def test_replicas_take_max_time_and_sum_units():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, value, rc in res:
        assert ms == 15.0
        assert units == 3e9
        assert value == pytest.approx(3e9 / 0.015 / 1e9)
        assert rc == 0


def test_single_process_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(7.5) == 7.5
    assert bench.reduce_sum(2.0) == 2.0
    assert bench.job_value(2e9, 1000.0) == pytest.approx(2.0)
