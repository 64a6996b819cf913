"""The allocation-free entry point for local derivatives.

Some callers cannot allocate device memory (an application whose own
allocator owns all of it, or a framework that forbids allocations from
libraries), so they cannot create a context either. For them the library
offers nqs_logpsi_grad_noalloc, which keeps its working arrays in a fixed
device array instead of allocating. These tests call it through the C ABI,
twice in a row (the shared array keeps the previous call's contents), and
check its output two ways: against nqs_logpsi_grad on the same inputs (the
same kernels run, so the arrays must be bitwise equal) and against the
oracle's backward at the tolerances of the other gradient tests (relative
1e-10 in float64, 1e-4 with float32 internals).

This file is collected last on purpose, so that a failure here cannot stop
the rest of the suite.
"""

import numpy as np
import pytest
import torch

from oracle import cnn
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of, problem_of, rel_err

pytestmark = pytest.mark.gpu

CASES = [('j1j2_10x10', {'n_layers': 3}),
         ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 16, 'n_layers': 3})]


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('fp32', 1e-4), ('bf16', 1e-4)])
@pytest.mark.parametrize('case', CASES, ids=[c[0] for c in CASES])
def test_noalloc_grad_matches_context_entry_point_and_oracle(case, prec, tol):
    nqs = lib()
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    prob = problem_of(w, **over)
    spec, _ = oracle_of(w, **over)
    P = nqs.nqs_param_count(prob)
    for call, seed in enumerate((41, 42)):
        n = 7 + call
        cfg_np = configs_for(w, n, seed=seed, **over)
        cfg = dev(cfg_np)
        want = ctx.logpsi_grad(cfg, prec)
        out = torch.full((2 * n, P), float('nan'), dtype=torch.float64, device='cuda')
        nqs.nqs_logpsi_grad_noalloc(prob, ctx.params, cfg, out, prec)
        torch.cuda.synchronize()
        assert torch.equal(out, want)
        got = out.cpu().numpy()
        _, _, dA, dPhi = cnn.backward(params, cfg_np, spec)
        assert rel_err(got[:n], dA) <= tol
        assert rel_err(got[n:], dPhi) <= tol


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
