"""The VMC driver end to end: whole SR steps through the library against the
oracle's chain of the same steps (FP64), and a short optimisation of the
4x4 Heisenberg model against its exact ground-state energy."""

import json
import os

import numpy as np
import pytest
import torch

from oracle import cnn, eloc, sampler, sr
from tests.gpu_common import WL, lib, oracle_of, problem_of

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden', 'heisenberg_4x4.json')


@pytest.mark.parametrize('sr_method', ['cg', 'woodbury', 'auto'])
def test_fp64_sr_steps_match_the_oracle_chain(sr_method):
    """Two SR steps (sample, E_loc, O, SR solve, update) from the same seed:
    the samples and move counts bit for bit, energies, the solve and the
    updated parameters to FP64 rounding, with either SR solver."""
    lib()
    from paper_2204_07816_gb300.vmc import run_vmc
    import nqs_synth
    w = WL['j1j2_4x4']
    over = {'channels': 4, 'n_layers': 2}
    prob = problem_of(w, **over)
    spec, ham = oracle_of(w, **over)
    params = nqs_synth.random_params(1, 4, 2, seed=51, scale=0.8)
    n_ch, spc, burn, lr, eps, seed = 32, 4, 5, 0.05, 1e-3, 17
    final, recs = run_vmc(prob, params, 2, n_ch, spc, burn_in=burn, precision='fp64', eps=eps, rtol=1e-12,
                          lr=lr, seed=seed, sr_method=sr_method)
    p = np.array(params, dtype=np.float64)
    chains = sampler.init_chains(seed, n_ch, sampler.canonical_values(16, 8, 8))
    step = 0
    for k in range(2):
        counts = {}
        cfg, _, chains, _, _, step = sampler.metropolis(p, spec, chains, step, seed, spc, 1, burn if k == 0 else 0,
                                                        counts=counts)
        e = eloc.local_energy_batch(p, cfg, spec, ham)
        _, _, dA, dPhi = cnn.backward(p, cfg, spec)
        delta, em = sr.solve_dense(dA, dPhi, e, eps)
        r = recs[k]
        assert (r['moves'], r['accepted']) == (counts['moves'], counts['accepted'])
        assert abs(r['energy_per_site'] - em.real / 16) <= 1e-11 * abs(em.real / 16)
        assert abs(r['energy_imag_per_site'] - em.imag / 16) <= 1e-11
        # CG stops at rtol 1e-12; the sample-space solve's residual is the Cholesky's rounding, evaluated from O
        assert r['cg_converged'] and r['cg_residual'] <= (1e-12 if r['sr_method'] == 'cg' else 1e-10)
        assert r['sr_method'] == sr_method or (sr_method == 'auto' and (k > 0 or r['sr_method'] == 'cg'))
        assert abs(r['variance_per_site2'] - e.real.var() / 256) <= 1e-9 * e.real.var() / 256
        p = sr.update(p, delta, lr)
    assert np.linalg.norm(final - p) <= 1e-9 * np.linalg.norm(p - np.asarray(params))


def test_heisenberg_4x4_optimisation_approaches_exact_energy(tmp_path):
    """The paper's optimisation loop on its J2 = 0 special case (Eq. 2 with
    the Marshall sign rule), tensor-core path: after 150 SR steps the energy
    per site is within 1 % of exact diagonalisation and never below it by
    more than five error bars (the variational bound)."""
    lib()
    from paper_2204_07816_gb300.vmc import run_vmc
    import nqs_synth
    with open(GOLDEN) as f:
        e0 = json.load(f)['E0_per_site']
    w = WL['j1j2_4x4']
    over = {'J2': 0.0, 'sign_rule': True, 'channels': 16, 'n_layers': 3}
    prob = problem_of(w, **over)
    params = nqs_synth.random_params(1, 16, 3, seed=61, scale=0.3)
    log = str(tmp_path / 'vmc.jsonl')
    _, recs = run_vmc(prob, params, 150, 256, 4, burn_in=20, precision='bf16', eps=1e-3, lr=0.05, seed=62,
                      log=log)
    with open(log) as f:
        lines = [json.loads(s) for s in f]
    assert len(lines) == 150 and lines[-1]['step'] == 149
    for r in recs:
        assert np.isfinite(r['energy_per_site']) and 0.0 < r['acceptance'] <= 1.0
        assert r['energy_per_site'] >= e0 - 5 * r['error_per_site'] - 1e-9
    tail = np.mean([r['energy_per_site'] for r in recs[-20:]])
    assert recs[0]['energy_per_site'] > tail
    assert e0 - 0.01 <= tail <= 0.99 * e0
