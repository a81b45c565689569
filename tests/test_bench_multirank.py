"""The multi-process path of bench.py on CPU: two gloo ranks agree on the slowest rank's
time (max over ranks) and report the whole-job throughput over all ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(dist, 10.0 + 3.0 * rank, "cpu")
    v = bench.job_value(world, 100.0, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 13.0                    # the slower rank's time on every rank
        assert v == pytest.approx(200.0 / 13.0)


def test_single_process_values():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(None, 4.5, "cpu") == 4.5
    assert bench.job_value(1, 30.0, 2.0) == 15.0
