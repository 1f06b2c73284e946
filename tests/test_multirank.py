"""N > 1 host logic of the benchmark on CPU: world_size 2 over gloo, no GPU.

Rays are independent and the canvas is read-only, so ranks are replicas with
no collective on the data path; the only cross-rank step is the timing
aggregate (slowest rank, all ranks' rays)."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 50.0][rank]
    rays = [1000, 3000][rank]
    q.put((rank, bench.aggregate_ranks(ms, rays, world, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in (0, 1):
        ms_max, value = out[r]
        assert ms_max == 50.0
        assert value == pytest.approx(4000 / 0.050 / 1e6)


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_ranks(20.0, 2_000_000, 1, "cpu") == (20.0, pytest.approx(100.0))
