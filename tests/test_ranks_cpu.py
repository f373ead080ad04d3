"""Host logic of the multi-GPU bench path on CPU ranks (gloo, world size 2):
ensemble members sharded across ranks cover every member exactly once, and
the max / sum reductions that give the whole-job time and cell count.
No GPU is used."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.shard(range(256), rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = bench.reduce_over_ranks(10.0 + rank, "max", dist)
    c = bench.reduce_over_ranks(len(mine) * 1000, "sum", dist)
    if rank == 0:
        out.put((got, t, c))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_and_reductions_on_two_cpu_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, t, c = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(x for part in got for x in part)
    assert flat == list(range(256))
    assert all(len(part) == 128 for part in got)
    assert t == 11.0
    assert c == 256 * 1000


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.5) == 3.5
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
