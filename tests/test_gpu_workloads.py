"""Batched ragged problems and data assimilation through the C ABI.

- several independent problems with different N_b, K_true and prior bounds in one
  context: one SMC stage per problem against the oracle (FP64 path), and the
  64-band Galactic-binary workload at full size on a sample of particles;
- assimilation (reuse bridge, Eq. reuse_bridge): likelihood of the new samples
  after tsmc_assimilate, one posterior-start stage against the oracle, and the
  paper's consistency claim (posterior-start matches prior-start on all data).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import TOL, assert_eval_parity, dev_tensor, population, torch

pytestmark = pytest.mark.gpu


def _ragged_pulse_workload(P=96, seed=77):
    rng = synth._rng(seed)
    probs = [synth.pulse_problem(rng, n, k, 0.1) for n, k in ((700, 2), (1024, 3), (1500, 4))]
    return synth.Workload("ragged", synth.PULSE, 6, P, probs, synth.PULSE_LO, synth.PULSE_HI,
                          synth.PULSE_LOGMASK, n_mut=2, seed=seed)


def test_ragged_problems_one_stage_match_oracle_fp64():
    wl = _ragged_pulse_workload()
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    b, lz, _ = ctx.run_stage(0, use_graph=True)
    z, K, _, _ = ctx.get_population()
    z, K = z.cpu().numpy(), K.cpu().numpy()
    P = wl.P
    for pb in range(3):
        res = oracle.Oracle(wl, pb).smc_run(P, max_stages=1)
        assert b[pb] == pytest.approx(res["beta"][0], abs=1e-13)
        assert lz[pb] == pytest.approx(res["logz"], rel=1e-11, abs=1e-11)
        Kg = K[pb * P:(pb + 1) * P]
        assert np.mean(Kg == res["K"]) > 0.95
        same = Kg == res["K"]
        close = np.all(np.isclose(z[pb * P:(pb + 1) * P], res["z"], rtol=1e-8, atol=1e-8),
                       axis=(1, 2))
        assert np.mean(close[same]) > 0.9


def test_batched_bands_full_size_sampled():
    """64 GB bands, N_b from 2^14 to 2^18, 2048 particles each, one launch."""
    t = torch()
    wl = synth.gb_bands()
    nb = len(wl.problems)
    zs, Ks = [], []
    for b in range(nb):
        z, K = synth.prior_population(wl, 100 + b, wl.P)
        zs.append(z)
        Ks.append(K)
    z, K = np.concatenate(zs), np.concatenate(Ks)
    ctx = sampler.open_context(wl, capi.MIXED)
    zd, Kd = dev_tensor(z, t.float64), dev_tensor(K, t.int32)
    ctx.set_population(zd, Kd, beta=[0.6] * nb)
    bt = dev_tensor(np.full(nb, 0.6), t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    t.cuda.synchronize()
    rng = np.random.default_rng(5)
    for b in rng.choice(nb, 4, replace=False):
        idx = b * wl.P + rng.choice(wl.P, 3, replace=False)
        res = oracle.Oracle(wl, int(b)).logl_grad(z[idx], K[idx], 0.6)
        assert_eval_parity(None, res, lo[idx], ln[idx], lp[idx], g[idx], K[idx], TOL[capi.MIXED], 4)


def test_assimilate_likelihood_of_new_samples():
    t = torch()
    wl = synth.assimilation_pulse_k14(P=64, n_full=1 << 14)
    pr = wl.problems[0]
    z, K = population(wl, 3, 64)
    n1 = 1 << 12
    for prec in (capi.FP64, capi.MIXED):
        ctx = sampler.open_context(wl, prec, n_use=n1, n_capacity=[pr.n])
        ctx.set_population(dev_tensor(z, t.float64), dev_tensor(K, t.int32), beta=[1.0])
        ctx.assimilate(0, pr.d[n1:1 << 13])
        _, _, lo, ln = ctx.get_population()
        res = oracle.Oracle(wl, n=1 << 13, n1=n1).logl_grad(z, K, 0.0)
        np.testing.assert_allclose(ln.cpu().numpy(), res["ll_new"], rtol=TOL[prec])
        np.testing.assert_allclose(lo.cpu().numpy(), res["ll_old"], rtol=TOL[prec])
        b, lz, _ = ctx.temper_state()
        assert b[0] == 0.0 and lz[0] == 0.0


def test_assimilate_refuses_a_population_still_tempered():
    """The reuse bridge starts from the posterior of the data held so far: at beta < 1 the
    call is refused (TSMC_ESTATE) and changes nothing; at beta = 1 it goes ahead."""
    t = torch()
    wl = synth.assimilation_pulse_k14(P=64, n_full=1 << 14)
    pr = wl.problems[0]
    z, K = population(wl, 3, 64)
    n1 = 1 << 12
    ctx = sampler.open_context(wl, capi.FP64, n_use=n1, n_capacity=[pr.n])
    zd, Kd = dev_tensor(z, t.float64), dev_tensor(K, t.int32)
    ctx.set_population(zd, Kd, beta=[0.4])
    _, _, lo0, ln0 = ctx.get_population()
    with pytest.raises(capi.TsmcError, match="tsmc error -6"):
        ctx.assimilate(0, pr.d[n1:1 << 13])
    _, _, lo1, ln1 = ctx.get_population()
    assert t.equal(lo0, lo1) and t.equal(ln0, ln1)
    assert ctx.temper_state()[0][0] == 0.4
    ctx.set_population(zd, Kd, beta=[1.0])
    ctx.assimilate(0, pr.d[n1:1 << 13])
    assert ctx.temper_state()[0][0] == 0.0


def test_posterior_start_stage_matches_oracle_fp64():
    """First stage after assimilation: old samples untempered, new ones tempered by beta."""
    wl = synth.pulse_workload("assim", 2048, 3, 5, 128, 12, n_mut=2)
    pr = wl.problems[0]
    n1 = 1024
    ora = oracle.Oracle(wl, n=n1, n1=0)
    first = ora.smc_run(128, max_stages=200)     # prior start on the first half
    ctx = sampler.open_context(wl, capi.FP64, n_use=n1, n_capacity=[pr.n])
    t = torch()
    ctx.set_population(dev_tensor(first["z"], t.float64), dev_tensor(first["K"], t.int32),
                       beta=[1.0])
    ctx.assimilate(0, pr.d[n1:])
    eps = first["eps"]
    ctx.set_kernel_params([eps])
    b, lz, _ = ctx.run_stage(500, use_graph=False)
    z, K, _, _ = ctx.get_population()
    ora2 = oracle.Oracle(wl, n=pr.n, n1=n1)
    res = ora2.smc_run(128, init_prior=False, z=first["z"], K=first["K"], stage0=500,
                       max_stages=1, eps=eps)
    assert b[0] == pytest.approx(res["beta"][0], abs=1e-13)
    assert lz[0] == pytest.approx(res["logz"], rel=1e-11, abs=1e-11)
    assert np.mean(K.cpu().numpy() == res["K"]) > 0.95


def test_posterior_start_consistent_with_prior_start():
    """Sec. 5: updating a posterior with new data reaches the same K posterior and evidence
    as a run from the prior on all the data, in fewer stages."""
    wl = synth.pulse_workload("assim", 4096, 5, 10, 1024, 21)
    pr = wl.problems[0]
    n1 = 2048
    seeds = range(4)
    full_h, full_z, two_h, two_z, st_full, st_post = [], [], [], [], [], []
    for s in seeds:
        wl.seed = s
        ctx = sampler.open_context(wl, capi.MIXED)
        out = sampler.run_smc(ctx, max_stages=400)
        _, K, _, _ = ctx.get_population()
        full_h.append(np.bincount(K.cpu().numpy(), minlength=11) / wl.P)
        full_z.append(out["logz"][-1][0])
        st_full.append(out["n_stages"])
        ctx.close()
        ctx = sampler.open_context(wl, capi.MIXED, n_use=n1, n_capacity=[pr.n])
        out1 = sampler.run_smc(ctx, max_stages=400)
        ctx.assimilate(0, pr.d[n1:])
        out2 = sampler.run_smc(ctx, max_stages=400, stage0=1000, init_prior=False)
        _, K, _, _ = ctx.get_population()
        two_h.append(np.bincount(K.cpu().numpy(), minlength=11) / wl.P)
        two_z.append(out1["logz"][-1][0] + out2["logz"][-1][0])
        st_post.append(out2["n_stages"])
        ctx.close()
    hf, hs = np.mean(full_h, 0), np.std(full_h, 0, ddof=1) / 2
    ht, hts = np.mean(two_h, 0), np.std(two_h, 0, ddof=1) / 2
    assert np.all(np.abs(hf - ht) <= 3 * np.sqrt(hs**2 + hts**2) + 0.03), (hf, ht)
    zf, zs = np.mean(full_z), np.std(full_z, ddof=1) / 2
    zt, zts = np.mean(two_z), np.std(two_z, ddof=1) / 2
    assert abs(zf - zt) <= 3 * math.hypot(zs, zts) + 0.5, (zf, zt)
    assert np.mean(st_post) < np.mean(st_full)


def test_sharded_bands_reproduce_the_whole_set_fp64():
    """Independent problems split into blocks, each block a context of its own with
    problem_base = its first global index (what a rank runs under torchrun), give exactly
    the results of one context over all of them: no exchange between blocks is needed."""
    from paper_2609_17674_b300 import dist as tdist

    t = torch()
    full = synth.gb_bands(n_bands=5, P=48, log2n=(10, 11))
    full.n_mut = 2

    def run(wl):
        ctx = sampler.open_context(wl, capi.FP64)
        ctx.init_population()
        for s in range(3):
            ctx.run_stage(s, use_graph=False)
        z, K, lo, ln = ctx.get_population()
        b, lz, e = ctx.temper_state()
        res = (z.cpu().numpy(), K.cpu().numpy(), ln.cpu().numpy(), b, lz)
        ctx.close()
        return res

    whole = run(full)
    parts = [run(tdist.shard_problems(full, 2, r)[0]) for r in range(2)]
    for i in range(5):
        assert np.array_equal(np.concatenate([p[i] for p in parts]), whole[i]), i


def _particle_shard_worker(rank, world, port, q, P_glob, stages):
    import copy
    import os

    import torch
    import torch.distributed as dist

    from paper_2609_17674_b300 import capi, sampler, synth
    from paper_2609_17674_b300 import dist as tdist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)   # host-side collectives
    torch.cuda.set_device(0)
    wl = synth.pulse_workload("shard", 2048, 3, 6, P_glob, 77, n_mut=2)
    shards = tdist.particle_shards(P_glob, world)
    b, c = shards[rank]
    wl_r = copy.copy(wl)
    wl_r.P = c
    ctx = sampler.open_context(wl_r, capi.FP64, particle_shard=(b, P_glob))
    ctx.init_population()
    hist = []
    for st in range(stages):
        beta, logz, _ = tdist.sharded_stage(ctx, st, shards, rank)
        hist.append((float(beta[0]), float(logz[0])))
    z, K, _, _ = ctx.get_population()
    q.put((rank, hist, z.cpu().numpy(), K.cpu().numpy()))
    ctx.close()
    dist.destroy_process_group()


def test_particle_sharded_stages_match_single_context_fp64():
    """The particles of one problem split over two processes (each its own context with
    particles_global and particle_base; gloo collectives on the host, so no kernel waits on
    another process): the all-gathered log-likelihoods give the same beta, evidence and
    ancestors as one context over all particles, the exchange brings each process the rows
    of its ancestors, and after two stages of moves (metric and step size from all-reduced
    sums, added in another order) K agrees exactly and z to 1e-9."""
    import socket

    import torch.multiprocessing as mp

    from paper_2609_17674_b300 import dist as tdist

    P_glob, stages = 256, 2
    wl = synth.pulse_workload("shard", 2048, 3, 6, P_glob, 77, n_mut=2)
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    ref = [ctx.run_stage(s, use_graph=False) for s in range(stages)]
    zr, Kr, _, _ = (x.cpu().numpy() for x in ctx.get_population())
    ctx.close()
    mpc = mp.get_context("spawn")
    q = mpc.Queue()
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    procs = [mpc.Process(target=_particle_shard_worker, args=(r, 2, port, q, P_glob, stages))
             for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in range(2)), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, hist, _, _ in out:
        assert hist[0] == (float(ref[0][0][0]), float(ref[0][1][0]))   # first stage: bitwise
        assert hist[1][0] == pytest.approx(float(ref[1][0][0]), abs=1e-12)
        assert hist[1][1] == pytest.approx(float(ref[1][1][0]), rel=1e-11, abs=1e-9)
    shards = tdist.particle_shards(P_glob, 2)
    zs = np.concatenate([o[2] for o in out])
    Ks = np.concatenate([o[3] for o in out])
    assert [c for _, c in shards] == [o[3].shape[0] for o in out]
    np.testing.assert_array_equal(Ks, Kr)
    np.testing.assert_allclose(zs, zr, rtol=1e-9, atol=1e-9)
