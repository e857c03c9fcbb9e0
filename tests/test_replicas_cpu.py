"""The multi-process path of bench.py on CPU: two gloo ranks (replicas only,
no data-path collective) aggregate their timings as max over ranks and report
the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    value, max_ms = bench.replica_throughput(local_ms, 20, ws)
    bench.barrier(ws)
    out[rank] = (value, max_ms)
    dist.destroy_process_group()


def test_two_replicas_max_over_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, max_ms = out[r]
        assert max_ms == 150.0
        assert value == pytest.approx(2 * 20 / 0.150)


def test_single_process_is_identity():
    import bench
    value, max_ms = bench.replica_throughput(200.0, 10, 1)
    assert max_ms == 200.0 and value == pytest.approx(50.0)
