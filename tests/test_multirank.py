"""Host-side logic of the multi-rank benchmark path on CPU with gloo and
world size 2: every rank gets its own cloud, the timing is the maximum over
ranks, and the throughput counts the points of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workloads.get("blobs_small")
    rw = bench.rank_workload(w, rank)
    x = rw.points(64)
    elapsed = 1.5 + rank          # the second rank is slower
    t = bench.max_over_ranks(elapsed, dist, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, rw.seed)
    firsts = [None] * world
    dist.all_gather_object(firsts, float(x[0, 0]))
    out[rank] = (t, seeds, firsts, bench.throughput(world, w.n, 5, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, seeds, firsts, thr = out[r]
        assert t == 2.5                          # max over ranks
        assert seeds == [0, 1]                   # one cloud per rank
        assert firsts[0] != firsts[1]
        assert thr == pytest.approx(world * 2000 * 5 / 2.5)
