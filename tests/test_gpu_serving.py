"""Continuous batching of SR steps (paper_2204_07816_gb300.serving): every
request's trajectory is the same alone and in the mix (bitwise: every
reduction runs in a fixed order), requests that arrive later join while
others run, and admission respects the memory budget."""

import numpy as np
import pytest

import nqs_synth
from tests.gpu_common import lib

pytestmark = pytest.mark.gpu


def _requests():
    from paper_2204_07816_gb300.serving import Request
    specs = [
        dict(model='j1j2', L=6, J2=0.45, n_layers=4, channels=16, n_samples=512, n_chains=64, n_steps=3, arrival=0.0),
        dict(model='j1j2', L=8, J2=0.55, n_layers=3, channels=32, n_samples=512, n_chains=32, n_steps=2, arrival=0.0),
        dict(model='tj', L=6, n_up=15, n_down=15, n_layers=3, channels=16, n_samples=256, n_chains=32, n_steps=2,
             arrival=0.05),
        dict(model='j1j2', L=10, J2=0.5, n_layers=3, channels=16, n_samples=512, n_chains=64, n_steps=2, arrival=0.1),
    ]
    out = []
    for i, s in enumerate(specs):
        c_in = 1 if s['model'] == 'j1j2' else 3
        params = nqs_synth.random_params(c_in, s['channels'], s['n_layers'], seed=100 + i)
        out.append(Request(rid=i, seed=7 + i, params=params, **s))
    return out


def test_results_same_alone_and_in_the_mix():
    lib()
    from paper_2204_07816_gb300.serving import Server
    reqs = _requests()
    alone = {}
    for r in _requests():
        r.arrival = 0.0
        res, _ = Server().run([r])
        alone[r.rid] = res[r.rid]
    server = Server()
    mixed, summary = server.run(reqs)
    assert summary['sr_steps'] == sum(r.n_steps for r in reqs)
    assert summary['p99_ms'] >= summary['p50_ms'] > 0
    for rid, a in alone.items():
        b = mixed[rid]
        assert np.array_equal(a.params, b.params)
        assert a.energies == b.energies
        assert a.cg_iters == b.cg_iters


def test_admission_waits_for_memory():
    lib()
    from paper_2204_07816_gb300.serving import Server, footprint_bytes
    reqs = _requests()[:2]
    for r in reqs:
        r.arrival = 0.0
    budget = max(footprint_bytes(r) for r in reqs) + 1   # room for one request at a time
    server = Server(hbm_budget_bytes=budget)
    res, summary = server.run(reqs)
    ev = server.events
    admit1 = [t for t, k, rid in ev if k == 'admit' and rid == 1][0]
    retire0 = [t for t, k, rid in ev if k == 'retire' and rid == 0][0]
    assert admit1 >= retire0
    assert summary['requests'] == 2


@pytest.mark.parametrize('model', ['j1j2', 'tj'])
def test_sm_limit_changes_no_result(model):
    """A context held to a few SMs (nqs_set_sm_limit: smaller grids, several
    chain groups per sampler block) produces bitwise the chains, log psi,
    E_loc, O_k and SR update of the unlimited context."""
    import torch
    from tests.gpu_common import WL, make_ctx
    w = WL['j1j2_10x10'] if model == 'j1j2' else WL['tj_12x12']
    over = {'n_layers': 3} if model == 'j1j2' else {'L': 8, 'n_up': 28, 'n_down': 28, 'n_layers': 3, 'channels': 16}
    outs = []
    for limit in (0, 6):
        ctx, _ = make_ctx(w, seed=5, **over)
        ctx.set_sm_limit(limit)
        cfg, lp = ctx.sample(200, 2, 1, 3, 'bf16')
        e = ctx.local_energy(cfg, None, 'bf16')
        O = ctx.logpsi_grad(cfg, 'bf16')
        delta, info = ctx.sr_solve(O, e, eps=1e-3, rtol=1e-8, max_iter=500, lr=0.01, apply_update=False)
        ctx.sync()
        outs.append((cfg, lp, e, O, delta))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    nqs = lib()
    with pytest.raises(nqs.NQSError):
        ctx.set_sm_limit(100000)
