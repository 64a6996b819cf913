"""Pins for oracle/philox.py, oracle/sampler.py and oracle/sr.py (CPU only)."""

import json
import os

import numpy as np
import pytest
from scipy import stats

import nqs_synth
from oracle import cnn, ed, eloc, hamiltonian, philox, sampler, sr
from tests import oracle_refs


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize('counter,key', [((0, 0, 0, 0), (0, 0)), ((5, 7, 0, 0), (11, 13)),
                                         ((2 ** 64 - 1, 2 ** 63 + 5, 9, 2 ** 40), (2 ** 64 - 3, 77)),
                                         ((123456789, 987654321, 0, 0), (42, 0))])
def test_philox_matches_numpy(counter, key):
    """numpy's Philox (a library routine) pre-increments its counter, so a
    generator started at counter - 1 returns the block for `counter`."""
    c = sum(v << (64 * k) for k, v in enumerate(counter))
    k_int = key[0] | (key[1] << 64)
    bg = np.random.Philox(counter=(c - 1) % (1 << 256), key=k_int)
    want = [int(v) for v in bg.random_raw(4)]
    assert list(philox.philox_block(counter, key)) == want
    vec = philox.philox_blocks(np.uint64(counter[0]), np.uint64(counter[1]), np.uint64(counter[2]),
                               np.uint64(counter[3]), key[0], key[1])
    assert [int(v) for v in vec] == want


def test_philox_vector_form_many_counters():
    rng = np.random.default_rng(0)
    c0 = rng.integers(0, 2 ** 63, 64, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    c1 = rng.integers(0, 2 ** 63, 64, dtype=np.uint64)
    out = philox.philox_blocks(c0, c1, 0, 0, 2 ** 64 - 1, 3)
    for n in range(64):
        ref = philox.philox_block((int(c0[n]), int(c1[n]), 0, 0), (2 ** 64 - 1, 3))
        assert tuple(int(o[n]) for o in out) == ref


def test_mulhi_and_unit_double():
    w = np.array([0, 1, 2 ** 63, 2 ** 64 - 1], dtype=np.uint64)
    for n in (1, 2, 100, 256, 144):
        assert [int(v) for v in philox.mulhi(w, n)] == [(int(x) * n) >> 64 for x in w]
    u = philox.unit_double(w)
    assert u[0] == 0.0 and u[2] == 0.5 and u[3] == 1.0 - 2.0 ** -53


# ---------------------------------------------------------------- sampler
def test_init_chains_are_permutations_of_the_multiset():
    vals = sampler.canonical_values(144, 63, 63)
    ch = sampler.init_chains(7, 32, vals)
    assert ch.shape == (32, 144)
    for row in ch:
        assert (row == 1).sum() == 63 and (row == -1).sum() == 63 and (row == 0).sum() == 18
    assert len({row.tobytes() for row in ch}) == 32


def test_init_chains_fisher_yates_by_hand():
    """Chain 3 of a 6-site multiset, shuffled step by step from the raw blocks."""
    vals = sampler.canonical_values(6, 2, 2)
    seed, c = 99, 3
    arr = list(vals)
    for k in range(5, 0, -1):
        b0 = philox.philox_block((c, k, 0, 0), (seed, 1))[0]
        j = (b0 * (k + 1)) >> 64
        arr[k], arr[j] = arr[j], arr[k]
    assert list(sampler.init_chains(seed, 4, vals)[c]) == arr


def test_sampler_conserves_sector_and_is_reproducible():
    spec = cnn.NetSpec(6, 3, 4, 2)
    params = nqs_synth.random_params(3, 4, 2, seed=2)
    ch0 = sampler.init_chains(5, 8, sampler.canonical_values(36, 14, 15))
    out1 = sampler.metropolis(params, spec, ch0, 0, 5, 3, 1, 2)
    out2 = sampler.metropolis(params, spec, ch0, 0, 5, 3, 1, 2)
    assert np.array_equal(out1[0], out2[0])
    s = out1[0]
    assert np.all((s == 1).sum(1) == 14) and np.all((s == -1).sum(1) == 15)
    a, phi = cnn.forward(params, s, spec)
    assert np.allclose(out1[1][:, 0], a, rtol=1e-13, atol=1e-13)
    assert np.allclose(out1[1][:, 1], phi, rtol=1e-13, atol=1e-13)
    # continuing from the returned state = one longer run
    first = sampler.metropolis(params, spec, ch0, 0, 5, 1, 1, 2)
    cont = sampler.metropolis(params, spec, first[2], first[5], 5, 2, 1, 0)
    assert np.array_equal(np.concatenate([first[0].reshape(8, 1, 36), cont[0].reshape(8, 2, 36)], 1),
                          out1[0].reshape(8, 3, 36))


@pytest.fixture(scope='module')
def exact_4x4():
    spec = cnn.NetSpec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=21, scale=0.8)
    basis = ed.sector_basis(16, 8, 8)
    a, _ = cnn.forward(params, basis, spec)
    p = np.exp(2 * (a - a.max()))
    p /= p.sum()
    return spec, params, basis, p


def _binned_counts(samples, basis, p, n_bins=32):
    keys = ed.config_keys(basis)
    idx = np.searchsorted(keys, ed.config_keys(samples))
    assert np.all(keys[idx] == ed.config_keys(samples))
    order = np.argsort(p)
    cum = np.cumsum(p[order])
    bin_of_rank = np.minimum((cum * n_bins).astype(int), n_bins - 1)
    bin_of_state = np.empty(p.size, dtype=int)
    bin_of_state[order] = bin_of_rank
    used = np.unique(bin_of_state)                # states heavier than 1/n_bins leave gaps
    bin_of_state = np.searchsorted(used, bin_of_state)
    expected = np.bincount(bin_of_state, weights=p, minlength=used.size)
    observed = np.bincount(bin_of_state[idx], minlength=used.size)
    return observed, expected, bin_of_state


@pytest.mark.parametrize('seed', [1, 2, 3])
def test_sampler_chi_square_against_enumeration(exact_4x4, seed):
    spec, params, basis, p = exact_4x4
    assert p.max() / p.min() > 100.0    # a distribution far from uniform
    assert p.max() < 0.01
    n_ch = 4096
    ch0 = sampler.init_chains(seed, n_ch, sampler.canonical_values(16, 8, 8))
    samples = sampler.metropolis(params, spec, ch0, 0, seed, 1, 1, 29)[0]
    obs, exp_p, bins = _binned_counts(samples, basis, p)
    chi2 = ((obs - n_ch * exp_p) ** 2 / (n_ch * exp_p)).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3
    # sensitivity: the same counts reject |psi|^1 (a sampler missing the factor 2)
    q = np.sqrt(p)
    q /= q.sum()
    exp_q = np.bincount(bins, weights=q, minlength=len(obs))
    chi2_q = ((obs - n_ch * exp_q) ** 2 / (n_ch * exp_q)).sum()
    assert stats.chi2.sf(chi2_q, len(obs) - 1) < 1e-6


def test_sampler_mixes_from_a_common_start(exact_4x4):
    """All 4,096 chains start from one striped state (rows alternately all up
    and all down), so the chi-square against |psi|^2 after burn-in also tests
    that the exchange moves connect the whole sector: a sampler that never
    moves spins between rows keeps every row's magnetisation and fails."""
    spec, params, basis, p = exact_4x4
    stripes = np.repeat(np.array([1, -1, 1, -1], dtype=np.int8), 4)
    n_ch = 4096
    samples = sampler.metropolis(params, spec, np.tile(stripes, (n_ch, 1)), 0, 4, 1, 1, 29)[0]
    obs, exp_p, _ = _binned_counts(samples, basis, p)
    chi2 = ((obs - n_ch * exp_p) ** 2 / (n_ch * exp_p)).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3


@pytest.mark.parametrize('start', ['uniform', 'packed'])
def test_sampler_chi_square_tj_sector(start):
    """t-J 4x4 with 2 up, 2 down and 12 holes (10,920 states): hops and
    exchanges sample the enumerated |psi|^2, and the same counts reject
    |psi|^1. 'uniform': independent uniform starts; 'packed': every chain
    starts with the four electrons on one 2x2 plaquette (up up / down down),
    so the chains must spread them over the lattice."""
    spec = cnn.NetSpec(4, 3, 4, 2)
    params = nqs_synth.random_params(3, 4, 2, seed=24, scale=2.0)
    basis = ed.sector_basis(16, 2, 2)
    assert basis.shape[0] == 10920
    a, _ = cnn.forward(params, basis, spec)
    p = np.exp(2 * (a - a.max()))
    p /= p.sum()
    assert p.max() / p.min() > 100.0
    n_ch = 4096
    if start == 'uniform':
        ch0 = sampler.init_chains(4, n_ch, sampler.canonical_values(16, 2, 2))
    else:
        packed = np.zeros(16, dtype=np.int8)
        packed[[0, 1]] = 1
        packed[[4, 5]] = -1
        ch0 = np.tile(packed, (n_ch, 1))
    samples = sampler.metropolis(params, spec, ch0, 0, 4, 1, 1, 40)[0]
    obs, exp_p, bins = _binned_counts(samples, basis, p)
    chi2 = ((obs - n_ch * exp_p) ** 2 / (n_ch * exp_p)).sum()
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3
    q = np.sqrt(p)
    q /= q.sum()
    exp_q = np.bincount(bins, weights=q, minlength=len(obs))
    chi2_q = ((obs - n_ch * exp_q) ** 2 / (n_ch * exp_q)).sum()
    assert stats.chi2.sf(chi2_q, len(obs) - 1) < 1e-6


# ---------------------------------------------------------------- SR
@pytest.fixture(scope='module')
def small_sr():
    spec = cnn.NetSpec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=31)
    cfg = nqs_synth.random_configs(16, 8, 8, 1024, seed=32)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    e = eloc.local_energy_batch(params, cfg, spec, hamiltonian.J1J2(4, 1.0, 0.5))
    return dA, dPhi, e


def test_s_matrix_symmetric_psd(small_sr):
    dA, dPhi, _ = small_sr
    S = sr.s_matrix(dA, dPhi)
    assert np.array_equal(S, S.T) or np.abs(S - S.T).max() < 1e-15
    assert np.linalg.eigvalsh(S).min() > -1e-12
    Oh = sr.centred_stack(dA, dPhi)
    assert np.allclose(Oh.T @ Oh / dA.shape[0], S, rtol=1e-12, atol=1e-14)


def test_cg_matches_dense_solve(small_sr):
    dA, dPhi, e = small_sr
    d_dense, em = sr.solve_dense(dA, dPhi, e, 1e-4)
    d_cg, it, res, em2 = sr.cg(dA, dPhi, e, 1e-4, 1e-12, 10000)
    assert res <= 1e-12 and it > 1
    assert np.linalg.norm(d_cg - d_dense) <= 1e-8 * np.linalg.norm(d_dense)
    assert em == em2


@pytest.mark.parametrize('n_s', [16, 64, 1024])
def test_woodbury_equals_dense_solve(small_sr, n_s):
    """The sample-space system gives the delta of the parameter-space one:
    fewer samples than parameters (2 N_s < P = 196), about equal, and more."""
    dA, dPhi, e = small_sr
    dA, dPhi, e = dA[:n_s], dPhi[:n_s], e[:n_s]
    for eps in (1e-4, 1e-2):
        d_dense, em = sr.solve_dense(dA, dPhi, e, eps)
        d_wb, em2 = sr.solve_woodbury(dA, dPhi, e, eps)
        assert np.linalg.norm(d_wb - d_dense) <= 1e-9 * np.linalg.norm(d_dense)
        assert abs(em - em2) <= 1e-14 * abs(em)


def test_large_shift_limit(small_sr):
    dA, dPhi, e = small_sr
    F, _ = sr.force(dA, dPhi, e)
    d, _ = sr.solve_dense(dA, dPhi, e, 1e8)
    assert np.linalg.norm(d * 1e8 - F) <= 1e-6 * np.linalg.norm(F)


@pytest.fixture(scope='module')
def exact_grad_setup():
    spec = cnn.NetSpec(4, 1, 2, 2)
    params = nqs_synth.random_params(1, 2, 2, seed=41, scale=1.2)
    basis = ed.sector_basis(16, 8, 8)
    Hf = oracle_refs.heisenberg_full(4, 1.0, 0.5)
    idx = np.array([oracle_refs.full_index(c) for c in basis])
    H = Hf[idx][:, idx].tocsr()
    return spec, params, basis, H


def _psi(params, basis, spec):
    a, phi = cnn.forward(params, basis, spec)
    return np.exp(a + 1j * phi)


def test_force_is_half_the_exact_energy_gradient(exact_grad_setup):
    """With |psi|^2 weights over the whole sector, F_k = (1/2) dE/dtheta_k for
    E = <psi|H|psi>/<psi|psi> (H from the Kronecker construction)."""
    spec, params, basis, H = exact_grad_setup
    _, _, dA, dPhi = cnn.backward(params, basis, spec)
    e = eloc.local_energy_batch(params, basis, spec, hamiltonian.J1J2(4, 1.0, 0.5))
    psi = _psi(params, basis, spec)
    F, e_mean = sr.force(dA, dPhi, e, weights=np.abs(psi) ** 2)

    def energy(th):
        v = _psi(th, basis, spec)
        return (np.vdot(v, H @ v) / np.vdot(v, v)).real

    assert abs(e_mean.real - energy(params)) < 1e-12
    h = 1e-5
    for k in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        g = (energy(pp) - energy(pm)) / (2 * h)
        assert abs(F[k] - 0.5 * g) <= 1e-6 * max(1.0, abs(g))


def test_s_matrix_is_the_fubini_study_metric(exact_grad_setup):
    """S_kl = Re[<d_k psi|d_l psi>/<psi|psi> - <d_k psi|psi><psi|d_l psi>/<psi|psi>^2]
    with d_k psi by central differences of the whole state vector."""
    spec, params, basis, _ = exact_grad_setup
    _, _, dA, dPhi = cnn.backward(params, basis, spec)
    psi = _psi(params, basis, spec)
    S = sr.s_matrix(dA, dPhi, weights=np.abs(psi) ** 2)
    h = 1e-5
    D = []
    for k in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        D.append((_psi(pp, basis, spec) - _psi(pm, basis, spec)) / (2 * h))
    D = np.array(D)
    nrm = np.vdot(psi, psi)
    G = (np.conj(D) @ D.T) / nrm - np.outer(np.conj(D) @ psi, np.conj(psi) @ D.T) / nrm ** 2
    assert np.abs(S - G.real).max() <= 1e-6 * np.abs(G.real).max()


def test_uniform_weights_equal_plain_means(small_sr):
    dA, dPhi, e = small_sr
    F1, e1 = sr.force(dA, dPhi, e)
    F2, e2 = sr.force(dA, dPhi, e, weights=np.full(e.size, 3.0))
    assert np.allclose(F1, F2, rtol=1e-13, atol=1e-16) and abs(e1 - e2) < 1e-13


def test_oracle_sampler_counts():
    """Move/acceptance counting in the oracle sampler: moves <= proposals,
    accepted <= moves; all-zero weights accept every move; the counts do not
    change the chains."""
    from oracle import cnn, sampler
    spec = cnn.NetSpec(L=4, c_in=1, channels=4, n_layers=2)
    rng = np.random.default_rng(5)
    params = 0.8 * rng.normal(size=cnn.param_count(spec))
    ch0 = sampler.init_chains(3, 32, sampler.canonical_values(16, 8, 8))
    counts = {}
    a = sampler.metropolis(params, spec, ch0, 0, 3, 2, 1, 2, counts=counts)
    b = sampler.metropolis(params, spec, ch0, 0, 3, 2, 1, 2)
    assert np.array_equal(a[0], b[0])
    assert 0 < counts['accepted'] <= counts['moves'] <= 32 * 4 * 16
    c0 = {}
    sampler.metropolis(np.zeros_like(params), spec, ch0, 0, 3, 2, 1, 2, counts=c0)
    assert c0['accepted'] == c0['moves'] > 0
    # a flat |psi| accepts every move, so the chains follow the proposals alone:
    # recount the moves one proposal at a time with Python integers
    moves = 0
    for c in range(32):
        s = [int(v) for v in ch0[c]]
        for step in range(4 * 16):
            b0, b1, _, _ = philox.philox_block((c, step, 0, 0), (3, 0))
            i = (b0 * 16) >> 64
            dx, dy = ((1, 0), (-1, 0), (0, 1), (0, -1))[b1 >> 62]
            j = ((i // 4 + dy) % 4) * 4 + (i % 4 + dx) % 4
            if s[i] != s[j]:
                moves += 1
                s[i], s[j] = s[j], s[i]
    assert c0['moves'] == moves


def test_exact_sr_descends_toward_the_ground_state():
    """Stochastic reconfiguration with exact |psi|^2 weights over the whole
    4x4 Sz=0 sector of the Heisenberg model (J2 = 0; the Sec. 3.2 update
    theta <- theta - eta (S + eps I)^-1 F): the energy falls at every step,
    never goes below the exact ground energy (variational bound), and moves
    most of the way from its start to it in 16 steps."""
    with open(os.path.join(os.path.dirname(__file__), 'golden', 'heisenberg_4x4.json')) as f:
        E0 = json.load(f)['E0']
    spec = cnn.NetSpec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=51, scale=1.5)
    basis = ed.sector_basis(16, 8, 8)
    H = ed.sparse_h(basis, hamiltonian.J1J2(4, 1.0, 0.0))
    energies = []
    for _ in range(16):
        a, phi = cnn.forward(params, basis, spec)
        psi = np.exp(a - a.max() + 1j * phi)
        _, _, dA, dPhi = cnn.backward(params, basis, spec)
        w = np.abs(psi) ** 2
        F, e_mean = sr.force(dA, dPhi, (H @ psi) / psi, weights=w)
        S = sr.s_matrix(dA, dPhi, weights=w)
        delta = np.linalg.solve(S + 1e-4 * np.eye(S.shape[0]), F)
        assert abs(e_mean.imag) < 1e-10
        energies.append(e_mean.real)
        params = sr.update(params, delta, 0.03)
    energies = np.array(energies)
    assert np.all(np.diff(energies) < 0)
    assert energies.min() >= E0 - 1e-9
    assert (energies[-1] - E0) < 0.2 * (energies[0] - E0)
