"""Multi-rank bookkeeping on CPU with gloo, 2 ranks: the measurement reduction of the
benchmark and the sharding of the batched bands across ranks."""
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


def _band_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    from paper_2609_17674_b300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    full = synth.gb_bands(n_bands=7, P=16, log2n=(10, 11))
    sub, idx = tdist.shard_problems(full, world, rank)
    # the shard is the owned block of the full set, keyed by its global indices
    assert sub.problem_base == idx[0]
    for j, b in enumerate(idx):
        assert np.array_equal(sub.problems[j].d, full.problems[b].d)
        assert sub.bounds(j) == full.bounds(b)
    owned = [None] * world
    dist.all_gather_object(owned, idx)
    cs = float(sum(full.problems[b].n for b in idx))
    ms, cs_tot = tdist.reduce_measurement(3.0 + rank, cs)
    q.put((rank, owned, ms, cs_tot, float(sum(p.n for p in full.problems))))
    dist.destroy_process_group()


def test_bands_sharded_across_two_ranks_gloo():
    """Every band is owned by exactly one rank, each rank's workload is its block of the full
    set with the global band indices as Philox keys, and the reduced count is the whole
    set's."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_band_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owned = out[0][1]
    assert sorted(sum(owned, [])) == list(range(7)) and owned == out[1][1]
    assert all(o[2] == 4.0 for o in out)            # slowest rank
    assert all(o[3] == o[4] for o in out)           # every band counted once


def test_exchange_plan_delivers_every_ancestor_row():
    """Brute force: after the planned exchange every rank holds, in its own order, exactly the
    rows the ancestors name (ragged shards, two problems, ancestors from anywhere)."""
    import numpy as np

    rng = np.random.default_rng(5)
    for P_glob, world in ((10, 3), (64, 2), (7, 4), (1, 1)):
        n_prob = 2
        shards = tdist.particle_shards(P_glob, world)
        assert sum(c for _, c in shards) == P_glob
        anc = np.sort(rng.integers(0, P_glob, (n_prob, P_glob)), axis=1)
        local = []   # row ids (problem, global particle) held by each rank, in its order
        for b, c in shards:
            local.append([(q, b + j) for q in range(n_prob) for j in range(c)])
        plans = [tdist.exchange_plan(anc, shards, r) for r in range(world)]
        for r in range(world):
            recv = []
            for s_ in range(world):
                recv += [local[s_][i] for i in plans[s_][0][r]]
            assert len(recv) == int(plans[r][1].sum())
            got = [recv[t] for t in plans[r][2]]
            b, c = shards[r]
            want = [(q, int(anc[q, b + j])) for q in range(n_prob) for j in range(c)]
            assert got == want


def _exchange_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P_glob, n_prob = 37, 2
    shards = tdist.particle_shards(P_glob, world)
    b, c = shards[rank]
    ids = torch.tensor([[1000.0 * qq + b + j for j in range(c)] for qq in range(n_prob)])
    full = tdist.all_gather_particles(ids, shards)          # every rank: all ids, global order
    anc = np.sort(np.random.default_rng(3).integers(0, P_glob, (n_prob, P_glob)), axis=1)
    rows = torch.stack([ids.ravel(), -ids.ravel()], dim=1)    # two columns per row
    new = tdist.exchange_rows(rows, anc, shards, rank)
    s = torch.tensor([float(rank + 1)])
    tdist.all_reduce_sum(s)
    q.put((rank, full.numpy().tolist(), new.numpy().tolist(), float(s[0])))
    dist.destroy_process_group()


def test_particle_exchange_two_ranks_gloo():
    """2 gloo ranks, 37 particles of 2 problems: the all-gather returns every rank's block in
    global order and the exchange leaves each rank with the rows of its ancestors."""
    import numpy as np

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    P_glob = 37
    anc = np.sort(np.random.default_rng(3).integers(0, P_glob, (2, P_glob)), axis=1)
    shards = tdist.particle_shards(P_glob, 2)
    for rank, full, new, s in out:
        assert np.array_equal(np.array(full), [[1000.0 * qq + i for i in range(P_glob)]
                                               for qq in range(2)])
        b, c = shards[rank]
        want = [1000.0 * qq + anc[qq, b + j] for qq in range(2) for j in range(c)]
        assert [row[0] for row in new] == want and [row[1] for row in new] == [-w for w in want]
        assert s == 3.0
