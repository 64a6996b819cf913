"""GPU checks of the e4m3 (FP8) form of the local energy: the row form with
layer 0 in bf16 and layers >= 1 on e4m3 operands (activations saturated to
+-448, weights scaled per output channel), fp32 accumulation, float64 ratios
and sums, through the C ABI.

Tolerances, from the arithmetic: e4m3 keeps 3 mantissa bits, so every
activation and weight of layers >= 1 carries a relative rounding error of up
to 2^-4 (against 2^-9 for bf16); these errors are independent from entry to
entry, so log psi moves by about 2^-4 / sqrt(C) per site and layer summed in
quadrature over N sites, a few 1e-2 for the networks here (an emulation of
the same operand rounding in float64 gave at most 0.034 on 16x16 and 0.017
on 10x10). The local energy of one sample takes differences of log psi
between configurations that share most of their activations, so its error
per site stays near 1e-3 (emulation: at most 1.2e-3); the tests hold it to
5e-3 per site and sample. The energy per site over a batch must be within
1e-4 of the float64 result on the same samples, the validity condition of
the fast forms; the float64 reference is the library's FP64 path, itself
held to 1e-10 of the oracle, with the oracle beside it on a subset.
"""

import numpy as np
import pytest
import torch

from oracle import eloc
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of, problem_of

pytestmark = pytest.mark.gpu

CASES = [
    ('j1j2_10x10', {}, 256),
    ('j1j2_4x4', {'channels': 16, 'n_layers': 3}, 256),
    ('j1j2_10x10', {'L': 7, 'n_up': 25, 'n_down': 24, 'n_layers': 5}, 256),
    ('j1j2_10x10', {'L': 13, 'n_up': 85, 'n_down': 84, 'n_layers': 3}, 128),
    ('tj_12x12', {'L': 7, 'n_up': 22, 'n_down': 22, 'channels': 16, 'n_layers': 4}, 256),
]


def _ids(c):
    return c[0] + ''.join('-%s%s' % kv for kv in c[1].items())


@pytest.mark.parametrize('case', CASES, ids=_ids)
def test_fp8_local_energy_within_the_energy_bar(case):
    name, over, n = case
    w = WL[name]
    L = over.get('L', w['L'])
    N = L * L
    nqs = lib()
    assert nqs.tc_plan(problem_of(w, **over), 'local_energy', n)['row_form'] == 1
    ctx, params = make_ctx(w, **over)
    cfg_h = configs_for(w, n, seed=51, **over)
    x = dev(cfg_h)
    e8 = ctx.local_energy(x, None, 'fp8').cpu().numpy()
    e64 = ctx.local_energy(x, None, 'fp64').cpu().numpy()
    eb = ctx.local_energy(x, None, 'bf16').cpu().numpy()
    d = np.abs(e8[:, 0] - e64[:, 0]) / N
    mean_site = abs(e8[:, 0].mean() - e64[:, 0].mean()) / N
    print('%s: energy/site %.2e, max per sample %.2e (bf16: %.2e, %.2e)' % (
        _ids(case), mean_site, d.max(), abs(eb[:, 0].mean() - e64[:, 0].mean()) / N,
        (np.abs(eb[:, 0] - e64[:, 0]) / N).max()))
    assert mean_site <= 1e-4
    assert d.max() <= 5e-3
    assert (np.abs(e8[:, 1] - e64[:, 1]) / N).max() <= 5e-3
    # the e4m3 operands are really used: the results differ from the bf16 form's
    assert np.abs(e8 - eb).max() > 1e-7
    # the oracle on a subset
    spec, ham = oracle_of(w, **over)
    want = eloc.local_energy(params, cfg_h[:6], spec, ham)
    assert (np.abs(e8[:6, 0] - want.real) / N).max() <= 5e-3


def test_fp8_deterministic_and_ignores_supplied_logpsi():
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    x = dev(configs_for(w, 96, seed=52))
    a = ctx.local_energy(x, None, 'fp8')
    b = ctx.local_energy(x, None, 'fp8')
    lp = ctx.logpsi(x, 'bf16')
    c = ctx.local_energy(x, lp, 'fp8')     # the sample's log psi is recomputed in FP8
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)


def test_fp8_zero_network_is_exact():
    """A zero network is uniform in any precision: SiLU(0) = 0 is exact in
    e4m3, so every ratio is 1 and E_loc = (J1 + J2) N / 2 exactly."""
    w = WL['j1j2_10x10']
    P = lib().nqs_param_count(problem_of(w))
    ctx, _ = make_ctx(w, params=np.zeros(P))
    e = ctx.local_energy(dev(configs_for(w, 16, seed=53)), None, 'fp8').cpu().numpy()
    assert np.all(e[:, 0] == 75.0) and np.all(e[:, 1] == 0.0)


def test_fp8_refused_where_not_offered():
    nqs = lib()
    w = WL['j1j2_10x10']
    ctx32, _ = make_ctx(w, channels=32, n_layers=3)
    x = dev(configs_for(w, 4, seed=54))
    with pytest.raises(nqs.NQSError) as ei:          # 32 channels: no e4m3 plan
        ctx32.local_energy(x, None, 'fp8')
    assert ei.value.code == -7
    ctx, _ = make_ctx(w)
    with pytest.raises(nqs.NQSError) as ei:          # FP8 is offered for local energies only
        ctx.logpsi(x, 'fp8')
    assert ei.value.code == -1
