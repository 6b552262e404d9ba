"""The multi-GPU path is replicas only: each rank takes its own instances, no collective on
the data path; the timing is the maximum over ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    specs = bench._instances(rank, 6)
    keys = torch.tensor([hash((s[2], tuple(s[3]))) & 0x7FFFFFFF for s in specs], dtype=torch.int64)
    gathered = [torch.zeros_like(keys) for _ in range(world)]
    dist.all_gather(gathered, keys)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put(([g.tolist() for g in gathered], t.item(), [s[2] for s in specs]))
    dist.destroy_process_group()


def test_two_ranks_shard_disjoint_instances_and_time_is_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered, tmax, primes0 = got
    assert not set(gathered[0]) & set(gathered[1])      # disjoint instance sets
    assert tmax == 2.0                                   # max over ranks
    assert primes0 == [7, 11, 13, 17, 19, 23]            # rank 0 keeps the prime cycle of the workload
