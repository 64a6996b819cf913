"""The allocation-free entry point for local derivatives.

Some callers cannot allocate device memory (an application whose own
allocator owns all of it, or a framework that forbids allocations while it
records work), so they cannot create a context either. For them the library
offers nqs_logpsi_grad_noalloc, which keeps its working arrays in a fixed
device array instead of allocating. These tests call it through the C ABI
and compare it with nqs_logpsi_grad on the same inputs, twice in a row (the
shared array keeps the previous call's contents), at the tolerances of the
other gradient tests: relative 1e-10 in float64, 1e-5 in float32.

This file is collected last on purpose, so that a failure here cannot stop
the rest of the suite.
"""

import numpy as np
import pytest
import torch

from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, problem_of, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('fp32', 1e-5)])
@pytest.mark.parametrize('case', [('j1j2_10x10', {'n_layers': 3}), ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14,
                                                                                    'channels': 16, 'n_layers': 3})])
def test_noalloc_grad_matches_context_entry_point(case, prec, tol):
    nqs = lib()
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    prob = problem_of(w, **over)
    P = nqs.nqs_param_count(prob)
    for call, seed in enumerate((41, 42)):
        cfg = dev(configs_for(w, 7 + call, seed=seed, **over))
        want = ctx.logpsi_grad(cfg, prec).cpu().numpy()
        out = torch.full((2 * cfg.shape[0], P), float('nan'), dtype=torch.float64, device='cuda')
        nqs.nqs_logpsi_grad_noalloc(prob, ctx.params, cfg, out, prec)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_err(got, want) <= tol


def test_noalloc_rejects_problems_beyond_the_fixed_array():
    nqs = lib()
    prob = nqs.make_problem('j1j2', 36, n_layers=16, channels=32)
    P = nqs.nqs_param_count(prob)
    params = torch.zeros(P, dtype=torch.float64, device='cuda')
    cfg = torch.ones((1, 36 * 36), dtype=torch.int8, device='cuda')
    out = torch.empty((2, P), dtype=torch.float64, device='cuda')
    with pytest.raises(nqs.NQSError) as ei:
        nqs.nqs_logpsi_grad_noalloc(prob, params, cfg, out, 'fp64')
    assert ei.value.code == -7
    assert 'fixed array' in str(ei.value)
