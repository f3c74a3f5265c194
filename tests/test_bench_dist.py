"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per
GPU on a real node) reduce their timings with a max, the whole-job value
counts every replica's nodes, and only rank 0 runs the oracle arm."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mx = bench.ranks_max([1.0 + rank, 10.0 - rank, 3.0], "cpu")

    class A:
        gpus, steps, warmup = world, 1, 3

    out = bench.run_reference(A, world, rank) if rank != 0 else "rank0"
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mx, out))


def test_two_gloo_ranks_reduce_with_max_and_rank0_reports():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict((r, (mx, out)) for r, mx, out in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r][0] == [2.0, 10.0, 3.0]  # element-wise max over ranks
    assert res[1][1] is None                   # rank 1 runs nothing for the oracle arm


def test_job_value_counts_every_replica():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    K, Np = 524288, 45
    one = bench.job_gdofs(1, K, Np, 3.0)
    assert bench.job_gdofs(4, K, Np, 3.0) == pytest.approx(4 * one)
    assert one == pytest.approx(K * Np / 3e-3 / 1e9)
