"""Sample-space (Woodbury) SR solve on the GPU against the oracle: the
parameter-space dense solve where P is small, the oracle's sample-space
solve at 10x10 sizes, and the GPU's own CG on the same system."""

import numpy as np
import pytest
import torch

from oracle import cnn, eloc, sr
from tests.gpu_common import WL, configs_for, dev, lib, make_ctx, oracle_of

pytestmark = pytest.mark.gpu


def _synthetic_sr(n, P, seed):
    """Seeded O [2n, P] with column means well away from zero (exercises the
    centring) and complex local energies."""
    rng = np.random.default_rng(seed)
    dA = rng.normal(size=(n, P)) + 3.0 * rng.normal(size=P)
    dPhi = 0.5 * rng.normal(size=(n, P)) - 2.0 * rng.normal(size=P)
    e = -20.0 + rng.normal(size=n) + 0.3j * rng.normal(size=n)
    return dA, dPhi, e


@pytest.mark.parametrize('n_s', [16, 100, 1024])
def test_woodbury_matches_dense_solve_4x4(n_s):
    """4x4 network (P = 196): 2 N_s = 32 (one partial block), 200 (ragged
    last block) and 2,048 (32 blocks)."""
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=71)
    spec, ham = oracle_of(w)
    cfg = configs_for(w, n_s, seed=72)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, ham)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    for eps in (1e-4, 1e-2):
        delta, info = ctx.sr_solve_woodbury(O, E, eps=eps)
        want, em = sr.solve_dense(dA, dPhi, e, eps)
        got = delta.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
        assert abs(info['energy'] - em) <= 1e-12 * abs(em)
        assert info['resid'] <= 1e-10
        # the GPU's CG on the parameter-space system reaches the same delta
        d_cg, ic = ctx.sr_solve(O, E, eps=eps, rtol=1e-12, max_iter=10000)
        assert ic['converged']
        assert np.linalg.norm(d_cg.cpu().numpy() - got) <= 1e-9 * np.linalg.norm(want)


def test_woodbury_10x10_sizes_against_oracle():
    """P = 11,792 (10x10, 16 channels, 6 layers) with 300 samples: 2 N_s = 600
    is far below P, the regime the sample-space form is for."""
    nqs = lib()
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    P = ctx.P
    n = 300
    dA, dPhi, e = _synthetic_sr(n, P, seed=73)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    delta, info = ctx.sr_solve_woodbury(O, E, eps=1e-4)
    want, em = sr.solve_woodbury(dA, dPhi, e, 1e-4)
    got = delta.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-9 * np.linalg.norm(want)
    assert abs(info['energy'] - em) <= 1e-12 * abs(em)
    assert info['resid'] <= 1e-9
    # bitwise repeatable
    d2, _ = ctx.sr_solve_woodbury(O, E, eps=1e-4)
    assert torch.equal(d2, delta)


def test_woodbury_update_and_degenerate_cases():
    nqs = lib()
    w = WL['j1j2_4x4']
    ctx, params = make_ctx(w, param_seed=74)
    P = ctx.P
    dA, dPhi, e = _synthetic_sr(40, P, seed=75)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    delta, _ = ctx.sr_solve_woodbury(O, E, eps=1e-3, lr=0.05, apply_update=True)
    torch.cuda.synchronize()
    assert np.allclose(ctx.params.cpu().numpy(), params - 0.05 * delta.cpu().numpy(), rtol=0, atol=1e-15)
    # equal local energies: F = 0, so delta = 0 and the residual is 0
    flat = torch.zeros_like(E)
    flat[:, 0] = -3.25
    d0, info0 = ctx.sr_solve_woodbury(O, flat, eps=1e-3)
    assert torch.count_nonzero(d0).item() == 0 and info0['resid'] == 0.0
    assert info0['energy'] == complex(-3.25, 0.0)
    # a single sample: the centred O is zero, delta = 0
    d1, _ = ctx.sr_solve_woodbury(O[[0, 40]].contiguous(), E[:1].contiguous(), eps=1e-3)
    assert torch.count_nonzero(d1).item() == 0
    for bad in (0.0, -1.0, float('nan')):
        with pytest.raises(nqs.NQSError) as ei:
            ctx.sr_solve_woodbury(O, E, eps=bad)
        assert ei.value.code == -1
    for bad in (-1, 9):
        with pytest.raises(nqs.NQSError) as ei:
            ctx.sr_solve_woodbury(O, E, eps=1e-3, refine_steps=bad)
        assert ei.value.code == -1


def test_woodbury_refinement_keeps_the_solution():
    """With 0, 1 and 2 refinement steps the delta stays within 1e-9 of the
    oracle and the residual does not grow (the direct solve is already at
    the FP64 floor of the residual's own evaluation here)."""
    lib()
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    dA, dPhi, e = _synthetic_sr(200, ctx.P, seed=76)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, _ = sr.solve_woodbury(dA, dPhi, e, 1e-4)
    res = []
    for k in (0, 1, 2):
        d, info = ctx.sr_solve_woodbury(O, E, eps=1e-4, refine_steps=k)
        assert np.linalg.norm(d.cpu().numpy() - want) <= 1e-9 * np.linalg.norm(want)
        res.append(info['resid'])
    assert res[1] <= max(res[0], 1e-12) * 1.5 and res[2] <= max(res[1], 1e-12) * 1.5
