"""Grouped local energies across problems (nqs_local_energy_multi) and the
chunked bond enumeration of large lattices, against the single-problem
entry point and the FP64 oracle."""

import numpy as np
import pytest
import torch

import nqs_synth
from oracle import eloc
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of, problem_of

pytestmark = pytest.mark.gpu

MIX = [
    ('j1j2_10x10', {}),
    ('j1j2_10x10', {'L': 6, 'n_up': 18, 'n_down': 18, 'J2': 0.4, 'n_layers': 4}),
    ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 16, 'n_layers': 3}),
    ('j1j2_16x16', {'n_layers': 3}),
    ('tj_12x12', {}),
    ('j1j2_10x10', {'L': 8, 'n_up': 32, 'n_down': 32, 'channels': 32, 'n_layers': 3}),
]


@pytest.mark.parametrize('prec', ['bf16', 'fp64'])
def test_grouped_equals_single_problem_launches(prec):
    nqs = lib()
    mix = MIX if prec == 'bf16' else MIX[:3]
    ctxs, cfgs, singles = [], [], []
    for i, (name, over) in enumerate(mix):
        w = WL[name]
        ctx, _ = make_ctx(w, param_seed=10 + i, **over)
        cfg = dev(configs_for(w, 5 + 3 * i, seed=20 + i, **over))
        ctxs.append(ctx)
        cfgs.append(cfg)
        singles.append(ctx.local_energy(cfg, None, prec))
    outs = nqs.local_energy_multi(ctxs, cfgs, prec)
    torch.cuda.synchronize()
    for a, b in zip(outs, singles):
        assert torch.equal(a, b)


def test_grouped_rejects_unsupported_channel_count():
    nqs = lib()
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w)          # 4 channels
    with pytest.raises(nqs.NQSError) as ei:
        nqs.local_energy_multi([ctx], [dev(configs_for(w, 2, 1))], 'bf16')
    assert ei.value.code == -7


def test_chunked_enumeration_large_lattice_vs_oracle():
    """20 x 20 J1-J2 has 1,600 bonds: the tensor-core E_loc walks them in two
    chunks; energy per site within 1e-4 of the oracle on the same samples."""
    w = WL['j1j2_10x10']
    over = {'L': 20, 'n_up': 200, 'n_down': 200, 'channels': 16, 'n_layers': 2}
    ctx, params = make_ctx(w, **over)
    spec, ham = oracle_of(w, **over)
    cfg = configs_for(w, 2, seed=30, **over)
    got = ctx.local_energy(dev(cfg), None, 'bf16').cpu().numpy()
    want = eloc.local_energy(params, cfg, spec, ham)
    assert abs(got[:, 0].mean() - want.real.mean()) / 400 <= 1e-4
    assert np.abs(got[:, 1] - want.imag).max() / 400 <= 1e-4


def test_chunked_enumeration_36x36_zero_network():
    """36 x 36 (5,184 bonds, six chunks): a zero network gives exactly
    (J1 + J2) N / 2 for every configuration."""
    w = WL['j1j2_10x10']
    over = {'L': 36, 'n_up': 648, 'n_down': 648, 'channels': 16, 'n_layers': 3}
    P = lib().nqs_param_count(problem_of(w, **over))
    ctx, _ = make_ctx(w, params=np.zeros(P), **over)
    e = ctx.local_energy(dev(configs_for(w, 3, seed=31, **over)), None, 'bf16').cpu().numpy()
    assert np.all(e[:, 0] == 0.75 * 1296) and np.all(e[:, 1] == 0.0)
