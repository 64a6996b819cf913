"""Shared helpers for the GPU parity tests: build/load the library, make
contexts, and move seeded inputs between numpy and the device."""

import numpy as np
import pytest
import torch

import nqs_synth
from oracle import cnn, hamiltonian

WL = nqs_synth.WORKLOADS


def lib():
    """Build and load the library; with NQS_CHECKED=1 the checked build (device-side index checks)."""
    import os
    from paper_2204_07816_gb300 import build
    if os.environ.get('NQS_CHECKED') == '1':
        os.environ['NQS_LIBRARY'] = build.build(checked=True)
    else:
        build.build()
    from paper_2204_07816_gb300 import nqs
    return nqs


def problem_of(w, **over):
    nqs = lib()
    d = dict(w)
    d.update(over)
    if d['model'] == 'j1j2':
        return nqs.make_problem('j1j2', d['L'], J1=d['J1'], J2=d['J2'], n_up=d['n_up'], n_down=d['n_down'],
                                sign_rule=d.get('sign_rule', False), n_layers=d['n_layers'], channels=d['channels'])
    return nqs.make_problem('tj', d['L'], t=d['t'], J=d['J'], n_up=d['n_up'], n_down=d['n_down'],
                            n_layers=d['n_layers'], channels=d['channels'])


def oracle_of(w, **over):
    d = dict(w)
    d.update(over)
    spec = cnn.NetSpec(d['L'], d['c_in'], d['channels'], d['n_layers'])
    if d['model'] == 'j1j2':
        ham = hamiltonian.J1J2(d['L'], d['J1'], d['J2'], sign_rule=d.get('sign_rule', False))
    else:
        ham = hamiltonian.TJ(d['L'], d['t'], d['J'])
    return spec, ham


def make_ctx(w, seed=0, param_seed=1, scale=0.5, params=None, **over):
    nqs = lib()
    d = dict(w)
    d.update(over)
    if params is None:
        params = nqs_synth.random_params(d['c_in'], d['channels'], d['n_layers'], param_seed, scale=scale)
    tp = torch.tensor(params, dtype=torch.float64, device='cuda')
    ctx = nqs.Context(problem_of(w, **over), tp, seed=seed)
    return ctx, params


def configs_for(w, count, seed, **over):
    d = dict(w)
    d.update(over)
    N = d['L'] ** 2
    return nqs_synth.random_configs(N, d['n_up'], d['n_down'], count, seed)


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_err(a, b):
    """Largest absolute difference over the batch divided by the largest
    magnitude of the reference b over the batch: a per-batch relative bound
    (an entry much smaller than the batch's largest is held to the same
    absolute error, not to the bound relative to itself)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


requires_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason='needs a CUDA GPU')
