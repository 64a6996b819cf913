"""log psi as a torch.autograd.Function, and the vector-Jacobian product
behind its backward (nqs_logpsi_vjp): the gradient must be the oracle's
sum_s g_a[s] d a_s/d theta + g_phi[s] d phi_s/d theta (relative 1e-10 in
float64, 1e-4 with float32 internals), computed without the [2n, P] matrix,
and the same bits whatever the grid."""

import numpy as np
import pytest
import torch

from oracle import cnn
from tests.gpu_common import WL, configs_for, dev, make_ctx, oracle_of, rel_err

pytestmark = pytest.mark.gpu

CASES = [('j1j2_10x10', {}), ('tj_12x12', {'L': 6, 'n_up': 15, 'n_down': 14, 'channels': 16, 'n_layers': 3}),
         ('j1j2_4x4', {})]


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('fp32', 1e-4), ('bf16', 1e-4)])
@pytest.mark.parametrize('case', CASES, ids=[c[0] for c in CASES])
def test_autograd_gradient_matches_oracle(case, prec, tol):
    from paper_2204_07816_gb300.autograd import logpsi
    name, over = case
    w = WL[name]
    if prec == 'bf16' and over.get('channels', w['channels']) not in (16, 32):
        pytest.skip('the bf16 forward runs on the tensor cores, which need 16 or 32 channels')
    ctx, params = make_ctx(w, **over)
    spec, _ = oracle_of(w, **over)
    cfg = configs_for(w, 11, seed=40, **over)
    rng = np.random.default_rng(41)
    ca, cp = rng.standard_normal(11), rng.standard_normal(11)
    p = ctx.params.requires_grad_(True)
    lp = logpsi(p, dev(cfg), ctx, prec)
    loss = (lp[:, 0] * dev(ca) + lp[:, 1] * dev(cp)).sum()
    loss.backward()
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    want = ca @ dA + cp @ dPhi
    assert rel_err(p.grad.cpu().numpy(), want) <= tol


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('bf16', 1e-4)])
@pytest.mark.parametrize('n', [0, 1, 37, 2500])
def test_vjp_equals_contraction_of_local_derivatives(n, prec, tol):
    """nqs_logpsi_vjp against g @ O with O from nqs_logpsi_grad, for batch
    sizes below, at and above the 1,024 chunks of the fixed-order sum (n =
    2,500: chunks of three samples, the last one ragged), and n = 0."""
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w, n_layers=3)
    cfg = dev(configs_for(w, max(n, 1), seed=42, n_layers=3)[:n])
    g = torch.from_numpy(np.random.default_rng(43).standard_normal((n, 2))).cuda()
    got = ctx.logpsi_vjp(cfg, g, prec)
    if n == 0:
        assert torch.equal(got, torch.zeros_like(got))
        return
    O = ctx.logpsi_grad(cfg, prec)
    want = g[:, 0] @ O[:n] + g[:, 1] @ O[n:]
    assert rel_err(got.cpu().numpy(), want.cpu().numpy()) <= tol


def test_vjp_bitwise_independent_of_grid():
    """Chunks depend on n only and are summed in order: a context held to a
    few SMs (a smaller grid) gives the same bits."""
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    cfg = dev(configs_for(w, 300, seed=44))
    g = torch.from_numpy(np.random.default_rng(45).standard_normal((300, 2))).cuda()
    for prec in ('fp64', 'bf16'):
        a = ctx.logpsi_vjp(cfg, g, prec).clone()
        ctx.set_sm_limit(7)
        b = ctx.logpsi_vjp(cfg, g, prec).clone()
        ctx.set_sm_limit(0)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


def test_autograd_requires_the_context_params():
    from paper_2204_07816_gb300.autograd import logpsi
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w)
    other = ctx.params.clone().requires_grad_(True)
    with pytest.raises(ValueError):
        logpsi(other, dev(configs_for(w, 2, 1)), ctx)
