"""log psi as a torch.autograd.Function: its gradient is the oracle's
vector-Jacobian product of the per-sample log-derivatives, also when the
[2n, P] derivative matrix is produced in several chunks."""

import numpy as np
import pytest
import torch

from oracle import cnn
from tests.gpu_common import WL, configs_for, dev, make_ctx, oracle_of, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('fp32', 1e-4)])
@pytest.mark.parametrize('max_bytes', [None, 2 * 11792 * 8 * 3])
def test_autograd_gradient_matches_oracle(prec, tol, max_bytes):
    from paper_2204_07816_gb300.autograd import logpsi
    w = WL['j1j2_10x10']
    ctx, params = make_ctx(w)
    spec, _ = oracle_of(w)
    cfg = configs_for(w, 11, seed=40)
    rng = np.random.default_rng(41)
    ca, cp = rng.standard_normal(11), rng.standard_normal(11)
    p = ctx.params.requires_grad_(True)
    lp = logpsi(p, dev(cfg), ctx, prec, max_bytes)
    loss = (lp[:, 0] * dev(ca) + lp[:, 1] * dev(cp)).sum()
    loss.backward()
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    want = ca @ dA + cp @ dPhi
    assert rel_err(p.grad.cpu().numpy(), want) <= tol


def test_autograd_requires_the_context_params():
    from paper_2204_07816_gb300.autograd import logpsi
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w)
    other = ctx.params.clone().requires_grad_(True)
    with pytest.raises(ValueError):
        logpsi(other, dev(configs_for(w, 2, 1)), ctx)
