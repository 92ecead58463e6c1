"""The multi-rank path of bench.py (replicas, max-over-ranks timing, whole-job
throughput) on world_size 2 with the gloo backend, on CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    # rank 1 is the slow one
    secs = 2.0 if rank == 1 else 1.0
    smax = bench.reduce_max(secs)
    v = bench.throughput(256 * 10, smax, ws)
    q.put((rank, ws, r, local, smax, v))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, smax, v in out:
        assert (ws, r, local) == (2, rank, rank)
        assert smax == 2.0
        assert v == pytest.approx(256 * 10 * 2 / 2.0)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max(3.5) == 3.5
    assert bench.throughput(100, 0.5, 1) == 200.0
    os.environ.pop("CUDA_VISIBLE_DEVICES", None)
    assert bench.physical_gpu(0) == "0"
    os.environ["CUDA_VISIBLE_DEVICES"] = "5,7"
    try:
        assert bench.physical_gpu(1) == "7"
    finally:
        os.environ.pop("CUDA_VISIBLE_DEVICES", None)
