"""The weak-scaling bookkeeping of the multi-rank benchmark, on CPU with gloo, 2 ranks."""
import os

import torch.multiprocessing as mp

from paper_2609_17674_b300 import dist as tdist


def test_shard_covers_units_once():
    for n in (1, 7, 64):
        for world in (1, 2, 3, 8):
            got = sum((tdist.shard(n, world, r) for r in range(world)), [])
            assert got == list(range(n))


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, cs = tdist.reduce_measurement(10.0 + 5 * rank, 1e12 * (rank + 1))
    q.put((rank, ms, cs, tdist.rank_seed(1002, rank)))
    dist.destroy_process_group()


def test_reduce_measurement_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]          # max over ranks
    assert [o[2] for o in out] == [3e12, 3e12]          # sum over ranks
    assert out[0][3] != out[1][3]                        # independent problems per rank
