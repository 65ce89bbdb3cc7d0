"""Host-side logic of the Python layer that needs no GPU: the stage loop of run_smc
driven by a fake context."""
import numpy as np

from paper_2609_17674_b300 import sampler


class _FakeContext:
    """Two problems whose beta reaches 1 after 3 and 5 stages; records the calls."""

    def __init__(self, finish=(3, 5)):
        self.finish = np.array(finish)
        self.stages, self.inits, self.graphs = [], 0, []

    def init_population(self):
        self.inits += 1

    def run_stage(self, stage, use_graph=True, read=True):
        self.stages.append(stage)
        self.graphs.append(use_graph)
        k = len(self.stages)
        beta = np.minimum(1.0, k / self.finish)
        return beta, -0.5 * k * np.ones(2), 100.0 * np.ones(2)


def test_run_smc_stops_when_every_problem_reaches_beta_one():
    ctx = _FakeContext()
    out = sampler.run_smc(ctx, max_stages=50, stage0=7, use_graph=False)
    assert ctx.inits == 1
    assert ctx.stages == [7, 8, 9, 10, 11]           # consecutive, from stage0
    assert ctx.graphs == [False] * 5
    assert out["n_stages"] == 5 and out["beta"].shape == (5, 2)
    assert np.all(out["beta"][-1] == 1.0) and not np.all(out["beta"][-2] == 1.0)
    assert out["logz"][-1, 0] == -2.5


def test_run_smc_respects_max_stages_and_posterior_start():
    ctx = _FakeContext(finish=(3, 100))
    out = sampler.run_smc(ctx, max_stages=4, init_prior=False)
    assert ctx.inits == 0                            # posterior start: population given
    assert ctx.stages == [0, 1, 2, 3] and out["n_stages"] == 4
    assert out["beta"][-1, 1] < 1.0


def test_autotune_reads_its_cache_without_a_device(tmp_path):
    """A cached launch shape for the workload's key (model, precision, N_max, K_max,
    P_total) is returned as stored; other keys in the file are ignored."""
    import json

    from paper_2609_17674_b300 import autotune, capi, synth

    wl = synth.pulse_n1024_k3()
    key = [wl.model, capi.MIXED, 1024, wl.kmax, wl.P]
    best = {"threads": 96, "samples_per_thread": 32, "ms": {"96x32": 1.0}}
    other = {"threads": 256, "samples_per_thread": 16, "ms": {}}
    f = tmp_path / "tune.json"
    json.dump([{"key": [wl.model, capi.FP64, 1024, wl.kmax, wl.P], "best": other},
               {"key": key, "best": best}], open(f, "w"))
    autotune._cache.clear()
    assert autotune.tune(wl, capi.MIXED, cache_file=str(f)) == best
