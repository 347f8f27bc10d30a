"""The N > 1 path of bench.py (independent replicas, max-over-ranks timing)
exercised with two gloo ranks on the CPU."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank
    slow = bench.max_over_ranks(local_ms, dist, "cpu")
    seed = bench.replica_seed(3, rank)
    value = bench.whole_job_tflops(7.33e11, world, slow)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slow, seed, value))


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]          # both see the slowest rank
    assert [o[2] for o in out] == [3, 4]                  # distinct replica seeds
    assert abs(out[0][3] - 2 * 7.33e11 / 0.150 / 1e12) < 1e-9   # whole-job flops over the slowest time


def test_single_process_path():
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.replica_seed(3, 0) == 3
