"""The allocation-free resampling entry point against the context path.

tsmc_resample_systematic_static serves callers that cannot allocate device memory
(stream capture in progress, device memory owned by a host framework's pool,
loops that must not take cudaMalloc's implicit synchronisation).  Its scratch is a
fixed static device array, so this test checks that two calls in a row, reusing
that scratch, give exactly the ancestors the context path (tsmc_temper_reweight_
resample) gives for the same log-weights, and that oversize requests are refused.
Collected last on purpose; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2609_17674_b300 import capi, sampler, synth

pytestmark = pytest.mark.gpu


def _context_ancestors(wl, stage):
    """Ancestors and the log-weights the context path used in its first stage."""
    import torch

    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    _, _, _, ln = ctx.get_population()
    ell = ln.cpu().numpy()
    beta, _, _ = ctx.temper_reweight_resample(stage)
    anc = ctx.get_ancestors().cpu().numpy()
    # first stage starts at beta = 0, so delta = beta_new exactly and logw = delta * ell
    P = wl.P
    logw = np.concatenate([beta[b] * ell[b * P:(b + 1) * P] for b in range(len(wl.problems))])
    return ctx, logw, anc


def test_static_resampling_matches_context_path_twice():
    import torch

    wl = synth.pulse_workload("noalloc", 1024, 3, 8, 700, 31, n_problems=2)
    stream = torch.cuda.Stream()
    results = []
    for stage in (3, 4):    # two calls in a row share (and reuse) the static scratch
        ctx, logw, anc = _context_ancestors(wl, stage)
        logw_d = torch.as_tensor(logw, device="cuda")
        out = torch.full((logw.shape[0],), -1, dtype=torch.int32, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())   # the fill above runs on torch's stream
        capi.resample_systematic_static(logw_d, 2, wl.P, wl.seed, stage, out, stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, anc)
        results.append(got)
        ctx.close()
    assert not np.array_equal(results[0], results[1])   # different stages, different draws


def test_static_resampling_rejects_oversize():
    import torch

    stream = torch.cuda.Stream()
    logw = torch.zeros(65537, dtype=torch.float64, device="cuda")
    out = torch.zeros(65537, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.TsmcError, match="static scratch limit"):
        capi.resample_systematic_static(logw, 1, 65537, 1, 0, out, stream)
    with pytest.raises(capi.TsmcError, match="static limit of 256"):
        capi.resample_systematic_static(logw, 257, 2, 1, 0, out, stream)


def test_static_resampling_binding_checks_buffers():
    """The binding refuses buffers the kernel would overrun or misread (the C side cannot
    check device buffer sizes): too short, wrong dtype, not contiguous, on the host."""
    import torch

    stream = torch.cuda.Stream()
    logw = torch.zeros(64, dtype=torch.float64, device="cuda")
    out = torch.zeros(64, dtype=torch.int32, device="cuda")
    for lw, o in ((logw[:63], out), (logw, out[:32]), (logw.float(), out),
                  (logw, out.long()), (torch.zeros(128, dtype=torch.float64, device="cuda")[::2],
                                       out), (logw.cpu(), out)):
        with pytest.raises(ValueError):
            capi.resample_systematic_static(lw, 2, 32, 1, 0, o, stream)
