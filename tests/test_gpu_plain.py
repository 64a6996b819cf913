"""GPU parity of the CUDA-core paths (float64 and float32) against the FP64
oracle, through the C ABI.

Tolerances: integers (connected lists, sampler chains) bit-exact; float64
log psi and E_loc relative 1e-10 (the path's stated bound); float32
log psi 1e-4 absolute and energy per site 1e-5.
"""

import numpy as np
import pytest
import torch

from oracle import cnn, eloc, sampler, sr
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of, problem_of, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    ('j1j2_4x4', {}),
    ('j1j2_4x4', {'sign_rule': True}),
    ('j1j2_10x10', {}),
    ('tj_12x12', {}),
    ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 8, 'n_layers': 3}),
    ('j1j2_16x16', {'n_layers': 3}),
]


def _ids(c):
    return c[0] + ''.join('-%s%s' % kv for kv in c[1].items())


@pytest.mark.parametrize('case', CASES, ids=_ids)
def test_connected_lists_bit_exact(case):
    name, over = case
    w = WL[name]
    ctx, _ = make_ctx(w, **over)
    _, ham = oracle_of(w, **over)
    cfg = configs_for(w, 40, seed=5, **over)
    n_conn, pairs, h, hdiag = ctx.connected(dev(cfg))
    n_conn, pairs, h, hdiag = (t.cpu().numpy() for t in (n_conn, pairs, h, hdiag))
    for s in range(cfg.shape[0]):
        d, conn = ham.connected(cfg[s])
        assert n_conn[s] == len(conn)
        got = [(int(pairs[s, k, 0]), int(pairs[s, k, 1]), float(h[s, k])) for k in range(n_conn[s])]
        assert got == [(i, j, float(v)) for i, j, v in conn]
        assert abs(hdiag[s] - d) <= 1e-12 * max(1.0, abs(d))


def test_connected_edge_configs():
    """All-up-but-one, checkerboard and hole-cluster states."""
    w = WL['tj_12x12']
    over = {'L': 4, 'n_up': 6, 'n_down': 6, 'channels': 4, 'n_layers': 2}
    ctx, _ = make_ctx(w, **over)
    _, ham = oracle_of(w, **over)
    cfg = np.array([[1] * 6 + [-1] * 6 + [0] * 4, [0] * 4 + [1, -1] * 6, [1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 1, -1]],
                   dtype=np.int8)
    n_conn, pairs, h, hdiag = (t.cpu().numpy() for t in ctx.connected(dev(cfg)))
    for s in range(3):
        d, conn = ham.connected(cfg[s])
        assert [(int(pairs[s, k, 0]), int(pairs[s, k, 1]), float(h[s, k])) for k in range(n_conn[s])] == \
            [(i, j, float(v)) for i, j, v in conn]


@pytest.mark.parametrize('case', CASES, ids=_ids)
def test_logpsi_fp64(case):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 37, seed=6, **over)
    got = ctx.logpsi(dev(cfg), 'fp64').cpu().numpy()
    a, phi = cnn.forward(params, cfg, spec)
    assert rel_err(got[:, 0], a) <= 1e-12
    assert rel_err(got[:, 1], phi) <= 1e-12


@pytest.mark.parametrize('case', CASES, ids=_ids)
def test_logpsi_fp32(case):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 37, seed=6, **over)
    got = ctx.logpsi(dev(cfg), 'fp32').cpu().numpy()
    a, phi = cnn.forward(params, cfg, spec)
    assert np.abs(got[:, 0] - a).max() <= 1e-4
    assert np.abs(got[:, 1] - phi).max() <= 1e-4


@pytest.mark.parametrize('case', CASES[:5], ids=_ids)
@pytest.mark.parametrize('give_logpsi', [False, True])
def test_local_energy_fp64(case, give_logpsi):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, ham = oracle_of(w, **over)
    n = 24 if w['L'] <= 4 or over.get('L', 99) <= 6 else 6
    cfg = configs_for(w, n, seed=7, **over)
    lp = None
    if give_logpsi:
        a, phi = cnn.forward(params, cfg, spec)
        lp = dev(np.stack([a, phi], 1))
    got = ctx.local_energy(dev(cfg), lp, 'fp64').cpu().numpy()
    want = eloc.local_energy(params, cfg, spec, ham)
    assert rel_err(got[:, 0] + 1j * got[:, 1], want) <= 1e-10


def test_local_energy_fp64_16x16_sampled():
    w = WL['j1j2_16x16']
    over = {'n_layers': 3}
    ctx, params = make_ctx(w, **over)
    spec, ham = oracle_of(w, **over)
    cfg = configs_for(w, 3, seed=8)
    got = ctx.local_energy(dev(cfg), None, 'fp64').cpu().numpy()
    want = eloc.local_energy(params, cfg, spec, ham)
    assert rel_err(got[:, 0] + 1j * got[:, 1], want) <= 1e-10


def test_local_energy_fp32_energy_per_site():
    w = WL['j1j2_10x10']
    ctx, params = make_ctx(w)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, 16, seed=9)
    got = ctx.local_energy(dev(cfg), None, 'fp32').cpu().numpy()
    want = eloc.local_energy(params, cfg, spec, ham)
    assert abs(got[:, 0].mean() - want.real.mean()) / 100 <= 1e-5
    assert rel_err(got[:, 0], want.real) <= 1e-4


def test_zero_network_closed_form_on_gpu():
    """All parameters zero: E_loc = (J1 + J2) N / 2 for every configuration."""
    w = WL['j1j2_10x10']
    P = lib().nqs_param_count(problem_of(w))
    ctx, _ = make_ctx(w, params=np.zeros(P))
    cfg = configs_for(w, 32, seed=10)
    for prec in ('fp64', 'fp32'):
        e = ctx.local_energy(dev(cfg), None, prec).cpu().numpy()
        assert np.all(e[:, 0] == 75.0) and np.all(e[:, 1] == 0.0)


def test_empty_batch_and_bad_args():
    nqs = lib()
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w)
    empty = torch.zeros((0, 16), dtype=torch.int8, device='cuda')
    assert ctx.local_energy(empty).shape == (0, 2)
    assert ctx.logpsi(empty).shape == (0, 2)
    with pytest.raises(nqs.NQSError) as ei:
        ctx.local_energy(dev(configs_for(w, 2, 1)), precision=7)
    assert ei.value.code == -1
    with pytest.raises(TypeError):
        ctx.local_energy(torch.zeros((2, 16), dtype=torch.int8))


def test_nonfinite_is_reported_at_sync():
    nqs = lib()
    w = WL['j1j2_4x4']
    params = np.full(196, 0.3)
    params[-8:-4] = 1e308     # w_a enormous: a overflows, E_loc ratios are inf/nan
    ctx, _ = make_ctx(w, params=params)
    ctx.local_energy(dev(configs_for(w, 4, 1)))
    with pytest.raises(nqs.NQSError) as ei:
        ctx.sync()
    assert ei.value.code == -4
    ctx.sync()   # the flag was cleared


@pytest.mark.parametrize('prec', ['fp64'])
def test_sampler_chains_bit_exact_fp64(prec):
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, seed=3, scale=0.8)
    spec, _ = oracle_of(w)
    cfg, lp = ctx.sample(16, 8, 1, 4, prec)
    ch0 = sampler.init_chains(3, 16, sampler.canonical_values(16, 8, 8))
    counts = {}
    want_cfg, want_lp, ch_end, _, _, step = sampler.metropolis(params, spec, ch0, 0, 3, 8, 1, 4, counts=counts)
    assert np.array_equal(cfg.cpu().numpy(), want_cfg)
    # move and acceptance counters: exactly the oracle's
    assert ctx.sampler_counts(reset=True) == (counts['moves'], counts['accepted'])
    assert ctx.sampler_counts() == (0, 0)
    assert rel_err(lp.cpu().numpy(), want_lp) <= 1e-12
    chains, gstep = ctx.get_chains(16)
    assert gstep == step and np.array_equal(chains.cpu().numpy(), ch_end)
    # a second call continues the same chains
    cfg2, _ = ctx.sample(16, 2, 2, 0, prec)
    want2 = sampler.metropolis(params, spec, ch_end, step, 3, 2, 2, 0)[0]
    assert np.array_equal(cfg2.cpu().numpy(), want2)


def test_sampler_chains_bit_exact_tj_fp64():
    w = WL['tj_12x12']
    over = {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 8, 'n_layers': 3}
    ctx, params = make_ctx(w, seed=11, **over)
    spec, _ = oracle_of(w, **over)
    cfg, _ = ctx.sample(8, 3, 1, 2, 'fp64')
    ch0 = sampler.init_chains(11, 8, sampler.canonical_values(36, 15, 14))
    want = sampler.metropolis(params, spec, ch0, 0, 11, 3, 1, 2)[0]
    assert np.array_equal(cfg.cpu().numpy(), want)


def test_chain_checkpoint_resume():
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, seed=4)
    ctx.sample(16, 2, 1, 2, 'fp64')
    chains, step = ctx.get_chains(16)
    saved = chains.clone()
    a, _ = ctx.sample(16, 3, 1, 0, 'fp64')
    ctx2, _ = make_ctx(w, seed=4, params=params)
    ctx2.set_chains(saved, step)
    b, _ = ctx2.sample(16, 3, 1, 0, 'fp64')
    assert torch.equal(a, b)


@pytest.mark.parametrize('case', [('j1j2_4x4', {}), ('tj_12x12', {'L': 4, 'n_up': 6, 'n_down': 5, 'channels': 4, 'n_layers': 2}),
                                  ('j1j2_10x10', {'n_layers': 3})], ids=_ids)
def test_logpsi_grad_fp64(case):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 9, seed=12, **over)
    O = ctx.logpsi_grad(dev(cfg), 'fp64').cpu().numpy()
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    assert rel_err(O[:9], dA) <= 1e-10
    assert rel_err(O[9:], dPhi) <= 1e-10


@pytest.mark.parametrize('case', [('j1j2_10x10', {}), ('tj_12x12', {}), ('j1j2_16x16', {'n_layers': 3}),
                                  ('j1j2_4x4', {'channels': 16, 'n_layers': 2})], ids=_ids)
@pytest.mark.parametrize('prec', ['fp32', 'bf16'])
def test_logpsi_grad_fp32_internals(case, prec):
    name, over = case
    w = WL[name]
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 5, seed=13, **over)
    O = ctx.logpsi_grad(dev(cfg), prec).cpu().numpy()
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    assert rel_err(O[:5], dA) <= 1e-4
    assert rel_err(O[5:], dPhi) <= 1e-4


def test_sr_solve_matches_oracle():
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=31)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, 1024, seed=32)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, ham)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    delta, info = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-12, max_iter=10000)
    d_dense, em = sr.solve_dense(dA, dPhi, e, 1e-4)
    assert info['converged'] and info['resid'] <= 1e-12
    assert np.linalg.norm(delta.cpu().numpy() - d_dense) <= 1e-8 * np.linalg.norm(d_dense)
    assert abs(info['energy'] - em) <= 1e-12 * abs(em)
    d_cg, it, _, _ = sr.cg(dA, dPhi, e, 1e-4, 1e-8, 10000)
    _, info8 = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-8)
    # CG iteration counts drift with the rounding near the tolerance: the float64 oracle's dot products against
    # the CUDA path's double-float S.x products (about 46-bit products, errors near 1e-15 of the terms' sum)
    assert abs(info8['iters'] - it) <= max(5, it // 5)


def test_sr_update_applied_in_place():
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=33)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, 256, seed=34)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, ham)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    delta, info = ctx.sr_solve(O, E, eps=1e-3, rtol=1e-10, lr=0.05, apply_update=True)
    torch.cuda.synchronize()
    assert np.allclose(ctx.params.cpu().numpy(), params - 0.05 * delta.cpu().numpy(), rtol=0, atol=1e-15)


def test_sr_not_converged_status():
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=35)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, 128, seed=36)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, ham)
    _, info = ctx.sr_solve(dev(np.concatenate([dA, dPhi], 0)), dev(np.stack([e.real, e.imag], 1)), rtol=1e-14,
                           max_iter=1)
    assert not info['converged'] and info['iters'] == 1


@pytest.mark.parametrize('where', ['O', 'eloc'])
def test_sr_nonfinite_input_leaves_params_unchanged(where):
    # a NaN in O (or E_loc) makes the solve non-finite: NQS_ERR_NONFINITE, and apply_update must not write
    # the NaN step into the parameters
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=37)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, 128, seed=38)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, ham)
    O = np.concatenate([dA, dPhi], 0)
    E = np.stack([e.real, e.imag], 1)
    if where == 'O':
        O[5, 7] = np.nan
    else:
        E[3, 0] = np.nan
    before = ctx.params.clone()
    nqs = lib()
    with pytest.raises(nqs.NQSError) as ei:
        ctx.sr_solve(dev(O), dev(E), eps=1e-3, rtol=1e-10, lr=0.05, apply_update=True)
    assert ei.value.code == -4
    torch.cuda.synchronize()
    assert torch.equal(ctx.params, before)

