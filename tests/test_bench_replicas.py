"""The multi-GPU path of bench.py runs independent replicas (a single graph does not shard;
there is no collective on the data path).  Its host logic is checked here with two gloo
ranks on the CPU: the whole-job value is every rank's updates over the slowest rank's time,
and every rank agrees on it."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    secs = [2.0, 3.0][rank]
    upd = [100.0, 140.0][rank]
    value, total = bench.replica_throughput(secs, upd, ws)
    dist.barrier()
    q.put((rank, value, total))
    dist.destroy_process_group()


def test_single_rank_is_local_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(2.0, 100.0, 1) == (50.0, 2.0)


def test_two_gloo_replicas_take_the_slowest_rank():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, total in res:
        assert total == 3.0
        assert value == pytest.approx(240.0 / 3.0, rel=1e-12)
