"""The 16x16 network of the full-size workload (32 channels, 8 layers,
P = 65,120): local derivatives against the oracle's backward, and the SR
solve at that P against the oracle's sample-space solve."""

import numpy as np
import pytest

from oracle import cnn, sr
from tests.gpu_common import WL, configs_for, dev, make_ctx, oracle_of, rel_err

pytestmark = pytest.mark.gpu

W16 = WL['j1j2_16x16']


def test_parameter_count():
    ctx, _ = make_ctx(W16)
    assert ctx.P == 65120


@pytest.mark.parametrize('prec,tol', [('fp64', 1e-10), ('fp32', 1e-4), ('bf16', 1e-4)])
def test_logpsi_grad_full_network(prec, tol):
    ctx, params = make_ctx(W16, param_seed=81)
    spec, _ = oracle_of(W16)
    cfg = configs_for(W16, 3, seed=82)
    O = ctx.logpsi_grad(dev(cfg), prec).cpu().numpy()
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    assert rel_err(O[:3], dA) <= tol
    assert rel_err(O[3:], dPhi) <= tol


@pytest.mark.parametrize('as_float', [False, True])
def test_sr_solves_at_full_parameter_count(as_float):
    """CG (parameter space) and the sample-space Cholesky solve on the GPU
    against the oracle's sample-space solve, P = 65,120 and 256 samples; O
    in full float64 (both planes of the CG's double-float split) and made of
    floats (the float plane alone, as the bf16 local derivatives are)."""
    ctx, _ = make_ctx(W16)
    P, n = ctx.P, 256
    rng = np.random.default_rng(83)
    dA = rng.normal(size=(n, P)) + rng.normal(size=P)
    dPhi = 0.5 * rng.normal(size=(n, P))
    if as_float:
        dA = dA.astype(np.float32).astype(np.float64)
        dPhi = dPhi.astype(np.float32).astype(np.float64)
    e = -300.0 + rng.normal(size=n) + 0.2j * rng.normal(size=n)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, em = sr.solve_woodbury(dA, dPhi, e, 1e-4)
    d_cg, info = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-10, max_iter=10000)
    assert info['converged'] and info['resid'] <= 1e-10
    assert np.linalg.norm(d_cg.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
    assert abs(info['energy'] - em) <= 1e-12 * abs(em)
    d_wb, iw = ctx.sr_solve_woodbury(O, E, eps=1e-4)
    assert np.linalg.norm(d_wb.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
