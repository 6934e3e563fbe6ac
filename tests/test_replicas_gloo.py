"""The N > 1 benchmark path (independent replicas, max-reduced timing) with
two gloo ranks on the CPU: no GPU, no data-path collective."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms = 100.0 * (rank + 1)  # the slower rank decides the job time
    value, worst = bench.replica_throughput(total_ms, steps=10, world=world)
    out.put((rank, value, worst))
    dist.destroy_process_group()


def test_two_replicas_report_whole_job_throughput():
    torch_mp = pytest.importorskip("torch.multiprocessing")
    ctx = torch_mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, worst in res:
        assert worst == 200.0
        assert value == pytest.approx(2 * 10 / 0.2)


def test_single_replica_needs_no_process_group():
    import bench
    value, worst = bench.replica_throughput(50.0, steps=5, world=1)
    assert worst == 50.0 and value == pytest.approx(100.0)
