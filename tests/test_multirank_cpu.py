"""The benchmark's multi-rank aggregation (max over ranks of the timed region,
whole-job throughput over all ranks' replicas), run as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench.dist_env()
        local_ms = [120.0, 80.0][rank]           # rank 0 is the slower one
        m = bench.max_over_ranks(local_ms, ws, torch.device("cpu"))
        v = bench.job_throughput(1000, ws, 10, m)
        q.put((rank, got_ws, got_rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got_ws, got_rank, m, v in res:
        assert got_ws == 2 and got_rank == rank
        assert m == 120.0                      # max over ranks
        assert v == pytest.approx(2 * 1000 * 10 / 0.120)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.job_throughput(100, 1, 4, 2000.0) == pytest.approx(200.0)
