"""GPU parity of the paper's CNN1 / CNN2 families (Sec. 5.2; the reading is
stated in include/nqs.h and the oracle's cnn_paper module) on the CUDA-core
paths, through the C ABI: log psi, local energies, local derivatives, the
vector-Jacobian product and the Metropolis chains against the FP64 oracle.
Bars: FP64 relative 1e-12 (log psi) / 1e-10 (E_loc, O_k), phi exactly, the
chains bit for bit; FP32 |d log psi| <= 1e-4 per site, energy per site
within 1e-5, O_k relative 1e-4."""

import numpy as np
import pytest
import torch

import nqs_synth
from oracle import cnn, cnn_paper, eloc, hamiltonian, sampler
from tests.gpu_common import dev, lib, rel_err

pytestmark = pytest.mark.gpu

# (kind, model, L, channels, blocks)
CASES = [('cnn1', 'j1j2', 4, 4, 2), ('cnn1', 'j1j2', 6, 8, 3), ('cnn1', 'tj', 4, 4, 2),
         ('cnn2', 'j1j2', 4, 4, 2), ('cnn2', 'j1j2', 5, 8, 3), ('cnn2', 'tj', 6, 8, 2)]


def _ids(c):
    return '%s-%s-L%d-C%d-B%d' % c


def setup(case, seed=1):
    kind, model, L, C, B = case
    nqs = lib()
    N = L * L
    c_in = 1 if model == 'j1j2' else 3
    if model == 'j1j2':
        nu, nd = N // 2, N - N // 2
        prob = nqs.make_problem('j1j2', L, J1=1.0, J2=0.5, n_up=nu, n_down=nd, n_layers=B, channels=C, net=kind)
        ham = hamiltonian.J1J2(L, 1.0, 0.5)
    else:
        nu, nd = (N - 3) // 2, (N - 3) - (N - 3) // 2
        prob = nqs.make_problem('tj', L, t=1.0, J=0.4, n_up=nu, n_down=nd, n_layers=B, channels=C, net=kind)
        ham = hamiltonian.TJ(L, 1.0, 0.4)
    spec = cnn_paper.PaperSpec(kind, L, c_in, C, B)
    params = nqs_synth.random_paper_params(kind, c_in, C, B, seed)
    assert nqs.nqs_param_count(prob) == cnn_paper.param_count(spec) == params.size
    ctx = nqs.Context(prob, torch.tensor(params, dtype=torch.float64, device='cuda'), seed=seed)
    return ctx, params, spec, ham, (N, nu, nd)


@pytest.mark.parametrize('case', CASES, ids=[_ids(c) for c in CASES])
def test_logpsi(case):
    ctx, params, spec, _, (N, nu, nd) = setup(case)
    cfg = nqs_synth.random_configs(N, nu, nd, 40, seed=2)
    a, phi = cnn.forward(params, cfg, spec)
    got = ctx.logpsi(dev(cfg), 'fp64').cpu().numpy()
    assert rel_err(got[:, 0], a) <= 1e-12
    assert np.array_equal(got[:, 1], phi)
    got32 = ctx.logpsi(dev(cfg), 'fp32').cpu().numpy()
    assert np.abs(got32[:, 0] - a).max() <= 1e-4 * N


@pytest.mark.parametrize('case', CASES, ids=[_ids(c) for c in CASES])
@pytest.mark.parametrize('give_logpsi', [False, True])
def test_local_energy(case, give_logpsi):
    ctx, params, spec, ham, (N, nu, nd) = setup(case)
    cfg = nqs_synth.random_configs(N, nu, nd, 24, seed=3)
    want = eloc.local_energy(params, cfg, spec, ham)
    x = dev(cfg)
    lp = ctx.logpsi(x, 'fp64') if give_logpsi else None
    got = ctx.local_energy(x, lp, 'fp64').cpu().numpy()
    assert rel_err(got[:, 0] + 1j * got[:, 1], want) <= 1e-10
    got32 = ctx.local_energy(x, None, 'fp32').cpu().numpy()
    assert abs(got32[:, 0].mean() - want.real.mean()) / N <= 1e-5


@pytest.mark.parametrize('case', CASES, ids=[_ids(c) for c in CASES])
def test_local_derivatives_and_vjp(case):
    ctx, params, spec, _, (N, nu, nd) = setup(case)
    cfg = nqs_synth.random_configs(N, nu, nd, 9, seed=4)
    _, _, dA, _ = cnn.backward(params, cfg, spec)
    O = ctx.logpsi_grad(dev(cfg), 'fp64').cpu().numpy()
    assert rel_err(O[:9], dA) <= 1e-10
    assert not O[9:].any()                          # d phi = 0 for a product of real neurons
    O32 = ctx.logpsi_grad(dev(cfg), 'fp32').cpu().numpy()
    assert rel_err(O32[:9], dA) <= 1e-4
    g = np.random.default_rng(5).standard_normal((9, 2))
    v = ctx.logpsi_vjp(dev(cfg), torch.from_numpy(g).cuda(), 'fp64').cpu().numpy()
    assert rel_err(v, g[:, 0] @ dA) <= 1e-10


@pytest.mark.parametrize('case', [CASES[0], CASES[3], CASES[5]], ids=[_ids(c) for c in (CASES[0], CASES[3], CASES[5])])
def test_sampler_chains_bit_exact_fp64(case):
    ctx, params, spec, _, (N, nu, nd) = setup(case, seed=6)
    cfg, lp = ctx.sample(8, 4, 1, 3, 'fp64')
    ch0 = sampler.init_chains(6, 8, sampler.canonical_values(N, nu, nd))
    want_cfg, want_lp, _, _, _, _ = sampler.metropolis(params, spec, ch0, 0, 6, 4, 1, 3)
    assert np.array_equal(cfg.cpu().numpy(), want_cfg)
    assert rel_err(lp.cpu().numpy()[:, 0], want_lp[:, 0]) <= 1e-12
    assert np.array_equal(lp.cpu().numpy()[:, 1], want_lp[:, 1])


def test_constant_network_closed_form_on_gpu():
    case = ('cnn2', 'j1j2', 6, 4, 2)
    ctx, params, spec, ham, (N, nu, nd) = setup(case)
    ctx.params.zero_()
    ctx.params[-1] = 0.7
    e = ctx.local_energy(dev(nqs_synth.random_configs(N, nu, nd, 8, seed=7)), None, 'fp64').cpu().numpy()
    assert np.allclose(e[:, 0], 0.75 * N, rtol=0, atol=1e-12) and np.abs(e[:, 1]).max() <= 1e-12


def test_tensor_core_precision_refused_for_paper_nets():
    nqs = lib()
    ctx, _, _, _, (N, nu, nd) = setup(('cnn1', 'j1j2', 4, 16, 2))
    with pytest.raises(nqs.NQSError) as ei:
        ctx.local_energy(dev(nqs_synth.random_configs(N, nu, nd, 2, seed=8)), None, 'bf16')
    assert ei.value.code == -7
    bad = nqs.make_problem('j1j2', 5, n_up=13, n_down=12, n_layers=2, channels=4, net='cnn1')   # odd N
    assert nqs.nqs_param_count(bad) == -1
