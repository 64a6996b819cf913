"""Pins for oracle/cnn.py and oracle/eloc.py (CPU only)."""

import numpy as np
import pytest

import nqs_synth
from oracle import cnn, ed, eloc, hamiltonian
from tests import oracle_refs


def _spec(L, c_in, C, n_l):
    return cnn.NetSpec(L=L, c_in=c_in, channels=C, n_layers=n_l)


@pytest.mark.parametrize('c_in,C,n_l,P', [(1, 4, 2, 196), (1, 16, 6, 11792), (1, 32, 8, 65120), (3, 32, 6, 47200)])
def test_param_counts(c_in, C, n_l, P):
    assert cnn.param_count(_spec(8, c_in, C, n_l)) == P
    assert nqs_synth.n_params(c_in, C, n_l) == P


def test_conv_matches_brute_force_loops():
    """Periodic cross-correlation with explicit index loops on a tiny case."""
    rng = np.random.default_rng(0)
    L, ci, co = 3, 2, 3
    h = rng.standard_normal((1, ci, L, L))
    W = rng.standard_normal((co, ci, 3, 3))
    b = rng.standard_normal(co)
    z = cnn.conv(h, W, b)
    for o in range(co):
        for y in range(L):
            for x in range(L):
                acc = b[o]
                for c in range(ci):
                    for ky in range(3):
                        for kx in range(3):
                            acc += W[o, c, ky, kx] * h[0, c, (y + ky - 1) % L, (x + kx - 1) % L]
                assert z[0, o, y, x] == pytest.approx(acc, abs=1e-13)


def test_silu_values():
    z = np.array([-3.0, -0.5, 0.0, 0.7, 4.0])
    assert np.allclose(cnn.silu(z), z / (1.0 + np.exp(-z)), rtol=0, atol=1e-16)
    h = 1e-6
    assert np.allclose(cnn.silu_grad(z), (cnn.silu(z + h) - cnn.silu(z - h)) / (2 * h), atol=1e-9)


@pytest.mark.parametrize('model', ['j1j2', 'tj'])
def test_translation_invariance(model):
    L = 6
    c_in = 1 if model == 'j1j2' else 3
    spec = _spec(L, c_in, 8, 3)
    params = nqs_synth.random_params(c_in, 8, 3, seed=1)
    nu, nd = (18, 18) if model == 'j1j2' else (15, 15)
    cfg = nqs_synth.random_configs(L * L, nu, nd, 4, seed=2)
    a0, p0 = cnn.forward(params, cfg, spec)
    grid = cfg.reshape(-1, L, L)
    for dy, dx in ((1, 0), (0, 1), (2, 3), (5, 5)):
        t = np.roll(grid, (dy, dx), axis=(1, 2)).reshape(-1, L * L)
        a1, p1 = cnn.forward(params, t, spec)
        assert np.allclose(a1, a0, rtol=1e-14, atol=1e-14)
        assert np.allclose(p1, p0, rtol=1e-14, atol=1e-14)
    # not invariant under an arbitrary permutation of sites
    perm = np.random.default_rng(9).permutation(L * L)
    a2, _ = cnn.forward(params, cfg[:, perm], spec)
    assert not np.allclose(a2, a0, rtol=1e-6)


def test_zero_head_gives_unit_amplitude():
    spec = _spec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=3)
    params[-8:] = 0.0
    a, phi = cnn.forward(params, nqs_synth.random_configs(16, 8, 8, 5, seed=4), spec)
    assert np.all(a == 0.0) and np.all(phi == 0.0)


@pytest.mark.parametrize('L,c_in,C,n_l,nu,nd', [(4, 1, 4, 2, 8, 8), (4, 3, 4, 2, 6, 7), (5, 1, 3, 3, 12, 13)])
def test_backward_matches_central_differences(L, c_in, C, n_l, nu, nd):
    """Every parameter, h = 1e-5, relative 1e-6."""
    spec = _spec(L, c_in, C, n_l)
    params = nqs_synth.random_params(c_in, C, n_l, seed=11)
    cfg = nqs_synth.random_configs(L * L, nu, nd, 3, seed=12)
    a, phi, dA, dPhi = cnn.backward(params, cfg, spec)
    h = 1e-5
    P = params.size
    fa = np.zeros((3, P))
    fp = np.zeros((3, P))
    for k in range(P):
        pp = params.copy()
        pm = params.copy()
        pp[k] += h
        pm[k] -= h
        ap, php = cnn.forward(pp, cfg, spec)
        am, phm = cnn.forward(pm, cfg, spec)
        fa[:, k] = (ap - am) / (2 * h)
        fp[:, k] = (php - phm) / (2 * h)
    scale = max(np.abs(fa).max(), np.abs(fp).max())
    assert np.abs(dA - fa).max() <= 1e-6 * scale
    assert np.abs(dPhi - fp).max() <= 1e-6 * scale
    # the head part is exactly the pooled features: d a / d w_a = hbar
    assert np.allclose(dA[:, P - 2 * C:P - C], dPhi[:, P - C:], rtol=0, atol=0)


def _blocks(c_in, C, n_l):
    """(offset, size) of every parameter block in the flat layout: per conv
    layer W[C_out][C_in][3][3] then b[C_out], then the head w_a[C], w_phi[C]."""
    out, off = [], 0
    for layer in range(n_l):
        cin = c_in if layer == 0 else C
        out += [(off, 9 * cin * C), (off + 9 * cin * C, C)]
        off += 9 * cin * C + C
    return out + [(off, C), (off + C, C)]


@pytest.mark.parametrize('L,c_in,C,n_l,nu,nd', [(10, 1, 16, 6, 50, 50), (12, 3, 32, 6, 63, 63)])
def test_backward_matches_central_differences_at_full_size(L, c_in, C, n_l, nu, nd):
    """The 10x10 J1-J2 and 12x12 t-J networks: a seeded random subset of
    parameters, at least eight from every weight, bias and head block,
    h = 1e-5, relative 1e-6."""
    spec = _spec(L, c_in, C, n_l)
    params = nqs_synth.random_params(c_in, C, n_l, seed=15)
    cfg = nqs_synth.random_configs(L * L, nu, nd, 2, seed=16)
    _, _, dA, dPhi = cnn.backward(params, cfg, spec)
    blocks = _blocks(c_in, C, n_l)
    assert blocks[-1][0] + blocks[-1][1] == params.size
    rng = np.random.default_rng(17)
    ks = np.concatenate([off + rng.choice(size, min(size, 8), replace=False) for off, size in blocks])
    h = 1e-5
    fa = np.zeros((2, ks.size))
    fp = np.zeros((2, ks.size))
    for n, k in enumerate(ks):
        pp = params.copy()
        pm = params.copy()
        pp[k] += h
        pm[k] -= h
        ap, php = cnn.forward(pp, cfg, spec)
        am, phm = cnn.forward(pm, cfg, spec)
        fa[:, n] = (ap - am) / (2 * h)
        fp[:, n] = (php - phm) / (2 * h)
    scale = max(np.abs(fa).max(), np.abs(fp).max())
    assert np.abs(dA[:, ks] - fa).max() <= 1e-6 * scale
    assert np.abs(dPhi[:, ks] - fp).max() <= 1e-6 * scale


@pytest.fixture(scope='module')
def enum_4x4():
    spec = _spec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=7, scale=1.5)
    basis = ed.sector_basis(16, 8, 8)
    return spec, params, basis


def test_local_energy_batch_equals_per_sample_form(enum_4x4):
    spec, params, basis = enum_4x4
    ham = hamiltonian.J1J2(4, 1.0, 0.5)
    pick = basis[::997]
    e1 = eloc.local_energy(params, pick, spec, ham)
    e2 = eloc.local_energy_batch(params, pick, spec, ham)
    assert np.allclose(e1, e2, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize('sign_rule', [False, True])
def test_full_enumeration_identity_j1j2(enum_4x4, sign_rule):
    """sum |psi|^2 E_loc / sum |psi|^2 = <psi|H|psi> / <psi|psi> with H from
    the independent Kronecker construction (sign rule: gauge-transformed)."""
    spec, params, basis = enum_4x4
    ham = hamiltonian.J1J2(4, 1.0, 0.5, sign_rule=sign_rule)
    e = eloc.local_energy_batch(params, basis, spec, ham)
    a, phi = cnn.forward(params, basis, spec)
    psi = np.exp(a + 1j * phi)
    w = np.abs(psi) ** 2
    Hf = oracle_refs.heisenberg_full(4, 1.0, 0.5)
    idx = np.array([oracle_refs.full_index(c) for c in basis])
    H = Hf[idx][:, idx]
    if sign_rule:
        even = np.array([(i % 4 + i // 4) % 2 == 0 for i in range(16)])
        d = np.where(((basis[:, even] == 1).sum(axis=1) % 2) == 0, 1.0, -1.0)
        H = H.multiply(np.outer(d, d)).tocsr()
    rayleigh = np.vdot(psi, H @ psi) / np.vdot(psi, psi)
    est = (w * e).sum() / w.sum()
    assert abs(est.real - rayleigh.real) <= 1e-12 * abs(rayleigh.real)
    assert abs(est.imag) <= 1e-12 * abs(rayleigh.real)
    assert abs(rayleigh.imag) <= 1e-12
    # a non-trivial state: E_loc varies from state to state
    assert np.std(e.real) > 1e-2


def test_full_enumeration_identity_tj():
    L, nu, nd = 4, 2, 2
    spec = _spec(L, 3, 4, 2)
    params = nqs_synth.random_params(3, 4, 2, seed=8, scale=1.5)
    basis = ed.sector_basis(16, nu, nd)
    ham = hamiltonian.TJ(L, 1.0, 0.4)
    e = eloc.local_energy_batch(params, basis, spec, ham)
    a, phi = cnn.forward(params, basis, spec)
    psi = np.exp(a + 1j * phi)
    H = ed.sparse_h(basis, ham)
    rayleigh = np.vdot(psi, H @ psi) / np.vdot(psi, psi)
    w = np.abs(psi) ** 2
    est = (w * e).sum() / w.sum()
    assert abs(est - rayleigh) <= 1e-12 * abs(rayleigh)


@pytest.mark.parametrize('L', [4, 6])
def test_zero_network_closed_form(L):
    """All parameters zero: psi is uniform on Sz = 0, the Sz = 0 member of the
    fully polarised multiplet, so E_loc = (J1 + J2) N / 4 * 2 / 2 = (J1+J2) N / 2
    for every configuration."""
    spec = _spec(L, 1, 4, 2)
    params = np.zeros(cnn.param_count(spec))
    N = L * L
    cfg = nqs_synth.random_configs(N, N // 2, N // 2, 6, seed=L)
    e = eloc.local_energy(params, cfg, spec, hamiltonian.J1J2(L, 1.0, 0.5))
    assert np.allclose(e.real, 0.75 * N, rtol=0, atol=1e-12)
    assert np.all(e.imag == 0.0)
