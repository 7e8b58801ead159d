"""Host logic of the multi-rank benchmark on CPU (gloo, world size 2): each rank's inputs are
disjoint (every pixel and problem is an independent solve, Sec. 3, so ranks share no data),
and the reported time is the maximum over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = bench.rank_workload(rank, world)
    seeds = torch.tensor(wl["image_seeds"] + [wl["em_seed"]], dtype=torch.int64)
    gathered = [torch.zeros_like(seeds) for _ in range(world)]
    dist.all_gather(gathered, seeds)
    t = torch.tensor([1.5 + rank], dtype=torch.float64)     # a rank's timed seconds
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    if rank == 0:
        q.put(([g.tolist() for g in gathered], float(t.item())))
    dist.destroy_process_group()


def test_rank_partition_and_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    gathered, tmax = q.get(timeout=5)
    img0, img1 = set(gathered[0][:-1]), set(gathered[1][:-1])
    assert len(img0) == 3 and len(img1) == 3 and not (img0 & img1)
    assert gathered[0][-1] != gathered[1][-1]
    assert tmax == 2.5


def test_rank_workload_rejects_bad_rank():
    sys.path.insert(0, ROOT)
    import bench
    with pytest.raises(ValueError):
        bench.rank_workload(2, 2)
