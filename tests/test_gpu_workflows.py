"""Parallel initial-state selection and checkpoint / transfer across L."""

import numpy as np
import pytest
import torch

import nqs_synth
from oracle import cnn, eloc
from tests.gpu_common import WL, lib, make_ctx, oracle_of, problem_of

pytestmark = pytest.mark.gpu


def test_initial_state_selection_picks_the_lowest_energy():
    lib()
    from paper_2204_07816_gb300.workflows import select_initial_state
    w = WL['j1j2_10x10']
    over = {'L': 6, 'n_up': 18, 'n_down': 18, 'n_layers': 3}
    prob = problem_of(w, **over)
    cands = [nqs_synth.random_params(1, 16, 3, seed=200 + k, scale=s) for k, s in enumerate([0.3, 1.0, 1.6, 2.2])]
    best, energies, ctxs = select_initial_state(prob, cands, n_chains=64, samples_per_chain=4, precision='bf16')
    assert best == int(np.argmin([e.real for e in energies]))
    assert len(set(round(e.real, 9) for e in energies)) == 4
    # each energy is the mean of that candidate's own E_loc on its own samples
    spec, ham = oracle_of(w, **over)
    cfg, _ = ctxs[best].sample(64, 1, 1, 0, 'fp64')
    e64 = ctxs[best].local_energy(cfg, None, 'fp64').cpu().numpy()
    want = eloc.local_energy(cands[best], cfg.cpu().numpy(), spec, ham)
    assert np.allclose(e64[:, 0], want.real, rtol=1e-10, atol=1e-10)


def test_checkpoint_resume_reproduces_the_next_step(tmp_path):
    lib()
    from paper_2204_07816_gb300.workflows import load_checkpoint, save_checkpoint
    w = WL['j1j2_10x10']
    over = {'L': 6, 'n_up': 18, 'n_down': 18, 'n_layers': 3}
    ctx, params = make_ctx(w, seed=9, **over)
    ctx.sample(32, 2, 1, 5, 'fp64')
    path = str(tmp_path / 'ck.pt')
    save_checkpoint(path, ctx, 32, step_index=1)
    a, _ = ctx.sample(32, 3, 1, 0, 'fp64')
    ctx2, step_index = load_checkpoint(path, problem_of(w, **over), seed=9)
    b, _ = ctx2.sample(32, 3, 1, 0, 'fp64')
    assert step_index == 1 and torch.equal(a, b)


def test_parameters_transfer_to_a_larger_lattice(tmp_path):
    """Parameters saved at 6 x 6 start a 10 x 10 run: same vector, and the
    network at 10 x 10 is the oracle's network with those parameters."""
    lib()
    from paper_2204_07816_gb300.workflows import load_checkpoint, save_checkpoint
    w = WL['j1j2_10x10']
    small = {'L': 6, 'n_up': 18, 'n_down': 18, 'n_layers': 3}
    ctx, params = make_ctx(w, seed=3, **small)
    ctx.sample(16, 1, 1, 2, 'fp64')
    path = str(tmp_path / 'ck6.pt')
    save_checkpoint(path, ctx, 16)
    big = {'n_layers': 3}
    ctx10, _ = load_checkpoint(path, problem_of(w, **big), seed=3)
    assert torch.equal(ctx10.params.cpu(), torch.tensor(params))
    spec, _ = oracle_of(w, **big)
    cfg = nqs_synth.random_configs(100, 50, 50, 6, seed=5)
    got = ctx10.logpsi(torch.from_numpy(cfg).cuda(), 'fp64').cpu().numpy()
    a, phi = cnn.forward(params, cfg, spec)
    assert np.allclose(got[:, 0], a, rtol=1e-12, atol=1e-12)
