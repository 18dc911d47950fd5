"""The multi-process path of bench.py on CPU (world size 2, gloo): the
timing reduction takes the slowest rank, the ensemble is split into disjoint
shards covering every instance, and the whole-job throughput counts all
ranks' cells.  A rank that fails is reported by the launcher, not hidden."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, dist)
    owned = bench.shard(48, rank, world)
    total_owned = bench.sum_over_ranks(len(owned), dist)
    cells = 1000 * (rank + 1)
    cells_all = bench.sum_over_ranks(cells, dist)
    value = bench.throughput(cells_all, 5, mx)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{mx} {total_owned} {value} {' '.join(map(str, owned))}\n")
    dist.destroy_process_group()


def test_two_rank_reduction_and_sharding(tmp_path):
    world = 2
    mp.spawn(worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    for r in rows:
        assert float(r[0]) == 20.0                   # max over ranks
        assert int(float(r[1])) == 48                # shards cover all instances
        assert float(r[2]) == pytest.approx(3000 * 5 / 20e-3)
    owned = [set(map(int, r[3:])) for r in rows]
    assert owned[0].isdisjoint(owned[1]) and owned[0] | owned[1] == set(range(48))


def failing_worker(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    if rank == 1:
        raise RuntimeError("rank 1 failed before its step")
    dist.destroy_process_group()


def test_failed_rank_is_reported():
    # a rank that raises makes the launcher raise on the host; no GPU involved
    with pytest.raises(Exception):
        mp.spawn(failing_worker, args=(2, free_port()), nprocs=2, join=True)
