"""GPU checks of the tensor-core (tcgen05, bf16 operands, fp32 accumulation)
path against the FP64 oracle, through the C ABI.

Tolerances (derived in the design notes): bf16 stores every activation with
a relative rounding error of at most 2^-9, so a network of n_l layers carries
a relative error of order n_l * 2^-9 in each activation; log psi sums N*C
such terms with weights of order 0.5/sqrt(C). Measured |d log psi| on these
workloads stays below 2e-3, and the tests hold it to 5e-3 per configuration.
The energy per site over a batch must be within 1e-4 of the oracle's on the
same samples (the validity condition of the fast path).
"""

import numpy as np
import pytest
import torch

from oracle import cnn, ed, eloc, sampler
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of

pytestmark = pytest.mark.gpu

TC_CASES = [
    ('j1j2_10x10', {}),
    ('j1j2_16x16', {'n_layers': 4}),
    ('tj_12x12', {}),
    ('j1j2_4x4', {'channels': 16, 'n_layers': 3}),
    ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 16, 'n_layers': 4}),
]


def _ids(c):
    return c[0] + ''.join('-%s%s' % kv for kv in c[1].items())


@pytest.mark.parametrize('case', TC_CASES, ids=_ids)
def test_logpsi_bf16_close_to_oracle(case):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 150, seed=21, **over)
    got = ctx.logpsi(dev(cfg), 'bf16').cpu().numpy()
    a, phi = cnn.forward(params, cfg, spec)
    da = np.abs(got[:, 0] - a).max()
    dp = np.abs(got[:, 1] - phi).max()
    print('max |d log|psi|| = %.3e, max |d phi| = %.3e (scale %.3e)' % (da, dp, np.abs(a).max()))
    assert da <= 5e-3 and dp <= 5e-3


@pytest.mark.parametrize('case', TC_CASES[:3], ids=_ids)
def test_logpsi_bf16_independent_of_batch_slot(case):
    """A configuration's bf16 log psi does not depend on which other
    configurations share its group, nor on its slot (bitwise)."""
    name, over = case
    w = WL[name]
    ctx, _ = make_ctx(w, **over)
    cfg = configs_for(w, 64, seed=22, **over)
    x = dev(cfg)
    a1 = ctx.logpsi(x, 'bf16')
    perm = torch.randperm(64, generator=torch.Generator().manual_seed(0)).cuda()
    a2 = ctx.logpsi(x[perm].contiguous(), 'bf16')
    assert torch.equal(a1[perm], a2)
    a3 = ctx.logpsi(x[:7].contiguous(), 'bf16')
    assert torch.equal(a1[:7], a3)


@pytest.mark.parametrize('case', TC_CASES[:3], ids=_ids)
def test_local_energy_bf16_energy_per_site(case):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, ham = oracle_of(w, **over)
    n = 48 if name != 'j1j2_16x16' else 12
    cfg = configs_for(w, n, seed=23, **over)
    got = ctx.local_energy(dev(cfg), None, 'bf16').cpu().numpy()
    want = eloc.local_energy(params, cfg, spec, ham)
    N = w['L'] ** 2
    e_site = abs(got[:, 0].mean() - want.real.mean()) / N
    print('energy per site bf16 - oracle = %.3e; max |dE_loc| = %.3e' % (e_site, np.abs(got[:, 0] - want.real).max()))
    assert e_site <= 1e-4


def test_local_energy_bf16_deterministic_across_batches():
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    cfg = dev(configs_for(w, 40, seed=24))
    e1 = ctx.local_energy(cfg, None, 'bf16')
    e2 = ctx.local_energy(cfg[10:20].contiguous(), None, 'bf16')
    assert torch.equal(e1[10:20], e2)


CONE_CASES = TC_CASES + [
    ('j1j2_10x10', {'L': 7, 'n_up': 25, 'n_down': 24, 'n_layers': 5}),
    ('tj_12x12', {'channels': 16}),
    ('j1j2_10x10', {'L': 24, 'n_up': 288, 'n_down': 288, 'n_layers': 6}),
]


@pytest.mark.parametrize('case', CONE_CASES, ids=_ids)
def test_local_energy_bf16_cones_equal_dense(case, monkeypatch):
    """Connected configurations evaluated on their cones only (rolled into a
    common frame, rows outside the cone copied from the sample's own
    activations) give bitwise the local energies of the dense forward, and
    the sample's supplied-log-psi path (dense) agrees to rounding."""
    name, over = case
    w = WL[name]
    ctx, _ = make_ctx(w, **over)
    n = 24 if over.get('L', w['L']) >= 24 else 48
    cfg = dev(configs_for(w, n, seed=31, **over))
    monkeypatch.setenv('NQS_TC_ROWS', '0')      # cones belong to the tap form
    monkeypatch.setenv('NQS_TC_CONES', '1')     # also where the plan would not use them by default
    cone = ctx.local_energy(cfg, None, 'bf16')
    monkeypatch.delenv('NQS_TC_CONES')
    monkeypatch.setenv('NQS_TC_DENSE', '1')
    dense = ctx.local_energy(cfg, None, 'bf16')
    monkeypatch.delenv('NQS_TC_DENSE')
    torch.cuda.synchronize()
    assert torch.equal(cone, dense)
    again = ctx.local_energy(cfg, None, 'bf16')     # default plan choice
    assert torch.equal(again, cone)


ROW_CASES = [
    ('j1j2_10x10', {}),
    ('j1j2_10x10', {'sign_rule': True}),
    ('j1j2_4x4', {'channels': 16, 'n_layers': 3}),
    ('j1j2_10x10', {'L': 7, 'n_up': 25, 'n_down': 24, 'n_layers': 5}),
    ('j1j2_10x10', {'L': 12, 'n_up': 72, 'n_down': 72, 'n_layers': 4}),
    ('j1j2_10x10', {'L': 11, 'n_up': 61, 'n_down': 60, 'n_layers': 3}),
    ('j1j2_10x10', {'L': 13, 'n_up': 85, 'n_down': 84, 'n_layers': 3}),
    ('tj_12x12', {'L': 7, 'n_up': 22, 'n_down': 22, 'channels': 16, 'n_layers': 4}),
]


@pytest.mark.parametrize('case', ROW_CASES, ids=_ids)
@pytest.mark.parametrize('give_logpsi', [False, True])
def test_local_energy_row_form_equals_tap_form(case, give_logpsi, monkeypatch):
    """The row form (rows = lattice row x configuration, x positions along
    tensor-memory columns, the three dx taps of a kernel row in one N = 3C
    MMA) accumulates every output's taps in the tap form's order onto a
    zeroed accumulator, so its local energies equal the tap form's bitwise,
    and both stay within the bf16 bar of the oracle."""
    nqs = lib()
    from tests.gpu_common import problem_of
    name, over = case
    w = WL[name]
    L = over.get('L', w['L'])
    plan = nqs.tc_plan(problem_of(w, **over), 'local_energy', 4096)
    assert plan['row_form'] == 1 and plan['blocks_per_sm'] == 2
    ctx, params = make_ctx(w, **over)
    cfg_h = configs_for(w, 37, seed=41, **over)
    cfg = dev(cfg_h)
    lp = ctx.logpsi(cfg, 'bf16') if give_logpsi else None
    rows = ctx.local_energy(cfg, lp, 'bf16')
    monkeypatch.setenv('NQS_TC_ROWS', '0')
    tap = ctx.local_energy(cfg, lp, 'bf16')
    monkeypatch.delenv('NQS_TC_ROWS')
    torch.cuda.synchronize()
    assert torch.equal(rows, tap)
    spec, ham = oracle_of(w, **over)
    want = eloc.local_energy(params, cfg_h[:8], spec, ham)
    got = rows[:8].cpu().numpy()
    assert abs(got[:, 0].mean() - want.real.mean()) / L ** 2 <= 1e-4


def test_local_energy_bf16_zero_network():
    w = WL['j1j2_10x10']
    from tests.gpu_common import problem_of
    P = lib().nqs_param_count(problem_of(w))
    ctx, _ = make_ctx(w, params=np.zeros(P))
    e = ctx.local_energy(dev(configs_for(w, 16, seed=25)), None, 'bf16').cpu().numpy()
    assert np.all(e[:, 0] == 75.0) and np.all(e[:, 1] == 0.0)


def test_local_energy_bf16_largest_lattice(monkeypatch):
    """36 x 36 (the largest lattice of the serving mix; 16 channels, 7
    layers; the plain paths' per-block working sets do not fit on chip at
    this size): a zero network gives exactly (J1 + J2) N / 2 for every
    sample, log psi agrees with the oracle's forward, and the cone-restricted
    local energy equals the dense one bitwise."""
    from tests.gpu_common import problem_of
    w = WL['j1j2_10x10']
    over = {'L': 36, 'n_up': 648, 'n_down': 648, 'n_layers': 7}
    P = lib().nqs_param_count(problem_of(w, **over))
    cfg_h = configs_for(w, 6, seed=27, **over)
    cfg = dev(cfg_h)
    zero, _ = make_ctx(w, params=np.zeros(P), **over)
    e0 = zero.local_energy(cfg, None, 'bf16').cpu().numpy()
    assert np.all(e0[:, 0] == 0.75 * 1296) and np.all(e0[:, 1] == 0.0)
    ctx, params = make_ctx(w, param_seed=28, **over)
    spec, _ = oracle_of(w, **over)
    a, phi = cnn.forward(params, cfg_h[:3], spec)
    lp = ctx.logpsi(cfg[:3], 'bf16').cpu().numpy()
    # the bf16 rounding of 1,296 sites' activations shifts log psi by a nearly common offset (about 4e-6 per
    # site); ratios of amplitudes, which the sampler and E_loc use, cancel it
    assert np.abs(lp[:, 0] - a).max() <= 1e-5 * 1296 and np.abs(lp[:, 1] - phi).max() <= 1e-5 * 1296
    assert np.abs((lp[1:, 0] - lp[0, 0]) - (a[1:] - a[0])).max() <= 1e-3
    e = ctx.local_energy(cfg, None, 'bf16')
    assert bool(torch.isfinite(e).all())
    monkeypatch.setenv('NQS_TC_DENSE', '1')
    assert torch.equal(ctx.local_energy(cfg, None, 'bf16'), e)


def test_bf16_unsupported_shapes_fail_loudly():
    nqs = lib()
    w = WL['j1j2_4x4']          # 4 channels: below the tensor-core N granularity
    ctx, _ = make_ctx(w)
    with pytest.raises(nqs.NQSError) as ei:
        ctx.local_energy(dev(configs_for(w, 2, 1)), None, 'bf16')
    assert ei.value.code == -7


def test_sampler_bf16_chi_square():
    """bf16 sampler on 4x4 (16 channels) against the oracle's enumerated |psi|^2."""
    from scipy import stats
    w = WL['j1j2_4x4']
    over = {'channels': 16, 'n_layers': 2}
    ctx, params = make_ctx(w, seed=5, scale=0.8, **over)
    spec, _ = oracle_of(w, **over)
    basis = ed.sector_basis(16, 8, 8)
    a, _ = cnn.forward(params, basis, spec)
    p = np.exp(2 * (a - a.max()))
    p /= p.sum()
    n_ch = 4096
    cfg, lp = ctx.sample(n_ch, 1, 1, 30, 'bf16')
    samples = cfg.cpu().numpy()
    assert np.all(samples.sum(1) == 0)
    keys = ed.config_keys(basis)
    idx = np.searchsorted(keys, ed.config_keys(samples))
    assert np.all(keys[idx] == ed.config_keys(samples))
    order = np.argsort(p)
    cum = np.cumsum(p[order])
    bins = np.empty(p.size, dtype=int)
    bins[order] = np.minimum((cum * 32).astype(int), 31)
    used = np.unique(bins)
    bins = np.searchsorted(used, bins)
    exp_c = np.bincount(bins, weights=p, minlength=used.size) * n_ch
    obs = np.bincount(bins[idx], minlength=used.size)
    chi2 = ((obs - exp_c) ** 2 / exp_c).sum()
    assert stats.chi2.sf(chi2, used.size - 1) > 1e-3


def test_sampler_bf16_chi_square_tj():
    """bf16 sampler on a t-J 4x4 sector (2 up, 2 down, 12 holes: 10,920
    states; 16 channels) against the oracle's enumerated |psi|^2."""
    from scipy import stats
    w = WL['tj_12x12']
    over = {'L': 4, 'n_up': 2, 'n_down': 2, 'channels': 16, 'n_layers': 2}
    ctx, params = make_ctx(w, seed=15, param_seed=25, scale=1.5, **over)
    spec, _ = oracle_of(w, **over)
    basis = ed.sector_basis(16, 2, 2)
    a, _ = cnn.forward(params, basis, spec)
    p = np.exp(2 * (a - a.max()))
    p /= p.sum()
    assert p.max() / p.min() > 100.0
    n_ch = 4096
    cfg, _ = ctx.sample(n_ch, 1, 1, 40, 'bf16')
    samples = cfg.cpu().numpy()
    assert np.all((samples == 1).sum(1) == 2) and np.all((samples == -1).sum(1) == 2)
    keys = ed.config_keys(basis)
    idx = np.searchsorted(keys, ed.config_keys(samples))
    assert np.all(keys[idx] == ed.config_keys(samples))
    order = np.argsort(p)
    cum = np.cumsum(p[order])
    bins = np.empty(p.size, dtype=int)
    bins[order] = np.minimum((cum * 32).astype(int), 31)
    used = np.unique(bins)
    bins = np.searchsorted(used, bins)
    exp_c = np.bincount(bins, weights=p, minlength=used.size) * n_ch
    obs = np.bincount(bins[idx], minlength=used.size)
    chi2 = ((obs - exp_c) ** 2 / exp_c).sum()
    assert stats.chi2.sf(chi2, used.size - 1) > 1e-3


def test_sampler_bf16_conserves_sector_tj():
    w = WL['tj_12x12']
    ctx, _ = make_ctx(w, seed=6)
    cfg, lp = ctx.sample(64, 2, 1, 2, 'bf16')
    c = cfg.cpu().numpy()
    assert np.all((c == 1).sum(1) == 63) and np.all((c == -1).sum(1) == 63) and np.all((c == 0).sum(1) == 18)
    # the stored log psi is the bf16 log psi of the stored configuration
    again = ctx.logpsi(cfg, 'bf16')
    assert torch.equal(again, lp)


def test_sampler_counts_bf16():
    """Move and acceptance counters of the tensor-core sampler: accepted <= moves
    <= proposals, and with all-zero weights (|psi| uniform) every move is
    accepted."""
    w = WL['j1j2_4x4']
    over = {'channels': 16, 'n_layers': 3}
    ctx, _ = make_ctx(w, **over)
    ctx.sample(64, 4, 1, 2, 'bf16')
    moves, acc = ctx.sampler_counts(reset=True)
    assert 0 < acc <= moves <= 64 * 6 * 16
    zero = np.zeros(nqs_param_count_of(w, **over))
    ctx0, _ = make_ctx(w, params=zero, **over)
    ctx0.sample(64, 4, 1, 2, 'bf16')
    m0, a0 = ctx0.sampler_counts()
    assert m0 > 0 and a0 == m0


def test_sampler_bf16_waves_of_chains():
    """More chains than one wave of co-resident sampler blocks (one chain per
    block, three blocks per SM: more than 456 chains on 152 SMs): every chain
    still has its block, later waves start as blocks retire. A chain's path
    depends only on its index and the seed, so the first 300 chains of a
    1,200-chain run equal a 300-chain run bitwise (configurations and log psi),
    and an SM share (fewer blocks, each taking several chains in turn) gives
    the 1,200 chains bitwise too."""
    w = WL['j1j2_10x10']
    over = {'n_layers': 3}
    from tests.gpu_common import problem_of
    plan = lib().tc_plan(problem_of(w, **over), 'sample', 1200)
    assert (plan['G'], plan['slots'], plan['grid']) == (1, 1, 1200)
    ctx_a, _ = make_ctx(w, seed=9, **over)
    cfg_a, lp_a = ctx_a.sample(1200, 2, 1, 2, 'bf16')
    ctx_b, _ = make_ctx(w, seed=9, **over)
    cfg_b, lp_b = ctx_b.sample(300, 2, 1, 2, 'bf16')
    ctx_c, _ = make_ctx(w, seed=9, **over)
    ctx_c.set_sm_limit(8)
    cfg_c, lp_c = ctx_c.sample(1200, 2, 1, 2, 'bf16')
    torch.cuda.synchronize()
    assert torch.equal(cfg_a[:600], cfg_b) and torch.equal(lp_a[:600], lp_b)
    assert torch.equal(cfg_a, cfg_c) and torch.equal(lp_a, lp_c)
    # and the stored log psi is the bf16 log psi of the stored configuration
    assert torch.equal(ctx_a.logpsi(cfg_a, 'bf16'), lp_a)


def nqs_param_count_of(w, **over):
    from tests.gpu_common import problem_of
    return lib().nqs_param_count(problem_of(w, **over))
