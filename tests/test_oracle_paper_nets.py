"""Pins of the oracle's CNN1 / CNN2 (the paper's network families, Sec. 5.2)
against things other than the vectorised code itself:

* an explicit-loop evaluation written from the formulas element by element;
* the amplitude as a direct float64 product of the output neurons against
  exp(a + i phi) (sign and magnitude of the product of neurons);
* central finite differences (Richardson-extrapolated) of a on every
  parameter (backward, max-pooling
  routes, transposed convolutions, the adjoint of the periodic padding,
  embedding rows);
* translation symmetries the reading implies (CNN1: shifts by an even number
  of columns and any number of rows; CNN2: any number of rows);
* a closed form: a constant network makes W uniform, so the J1-J2 local
  energy is (J1 + J2) N / 2 for every configuration;
* the full-enumeration identity sum |W|^2 E_loc / sum |W|^2 = <W|H|W>/<W|W>.
"""

import math

import numpy as np
import pytest

import nqs_synth
from oracle import cnn, cnn_paper, ed, eloc, hamiltonian
from tests import oracle_refs

KINDS = ['cnn1', 'cnn2']


def spec_of(kind, L=4, c_in=1, C=3, B=2):
    return cnn_paper.PaperSpec(kind, L, c_in, C, B)


def params_of(spec, seed, centre=False):
    p = nqs_synth.random_paper_params(spec.kind, spec.c_in, spec.channels, spec.n_layers, seed, scale=1.0)
    if centre:   # output neurons of both signs: the output bias (the last parameter) minus the median neuron
        _, _, (_, z) = cnn_paper.forward(p, configs_of(spec, 8, seed + 100), spec, return_cache=True)
        p[-1] -= np.median(z)
    return p


def configs_of(spec, count, seed):
    N = spec.L ** 2
    if spec.c_in == 1:
        return nqs_synth.random_configs(N, N // 2, N // 2, count, seed)
    return nqs_synth.random_configs(N, N // 2 - 1, N // 2 - 2, count, seed)


# ---------------------------------------------------------------- explicit loops
def loop_forward(params, sigma, spec):
    """The reading written out element by element (pure Python)."""
    L, N, C, B = spec.L, spec.L ** 2, spec.channels, spec.n_layers
    p = list(np.asarray(params, dtype=float))
    pos = 0

    def take(n):
        nonlocal pos
        out = p[pos:pos + n]
        pos += n
        return out

    ns = 2 if spec.c_in == 1 else 3

    def state(v):
        if spec.c_in == 1:
            return 1 if v > 0 else 0
        return {0: 0, 1: 1, -1: 2}[int(v)]

    if spec.kind == 'cnn2':
        E = take(ns * C)
        X = [[E[state(sigma[s]) * C + c] for s in range(N)] for c in range(C)]
    elif spec.c_in == 1:
        X = [[float(sigma[s]) for s in range(N)]]
    else:
        X = [[float(sigma[s] == v) for s in range(N)] for v in (0, 1, -1)]

    def conv3(X, cout):
        cin = len(X)
        W = take(9 * cout * cin)
        beta = take(cout)
        U = [[0.0] * N for _ in range(cout)]
        for o in range(cout):
            for y in range(L):
                for x in range(L):
                    acc = beta[o]
                    for c in range(cin):
                        for ky in range(3):
                            for kx in range(3):
                                yy, xx = (y + ky - 1) % L, (x + kx - 1) % L
                                acc += W[((o * cin + c) * 3 + ky) * 3 + kx] * X[c][yy * L + xx]
                    U[o][y * L + x] = acc
        return U

    for b in range(B):
        U = conv3(X, C)
        co = (1 if b == B - 1 else C) if spec.kind == 'cnn1' else C
        T = take(2 * C * co)
        gamma = take(co)
        if spec.kind == 'cnn1':
            V = [[max(U[c][2 * j], U[c][2 * j + 1]) for j in range(N // 2)] for c in range(C)]
            Y = [[gamma[o] + sum(T[(c * co + o) * 2 + (s % 2)] * V[c][s // 2] for c in range(C)) for s in range(N)]
                 for o in range(co)]
        else:
            V = [[max(U[c][s], U[c][(s + 1) % N]) for s in range(N)] for c in range(C)]
            Y = [[gamma[o] + sum(T[(c * co + o) * 2] * V[c][s] + T[(c * co + o) * 2 + 1] * V[c][(s - 1) % N]
                                 for c in range(C)) for s in range(N)] for o in range(co)]
        X = Y
    if spec.kind == 'cnn2':
        X = conv3(X, 1)
    assert pos == len(p)
    return X[0]


@pytest.mark.parametrize('kind', KINDS)
@pytest.mark.parametrize('c_in', [1, 3])
def test_forward_equals_explicit_loops_and_direct_product(kind, c_in):
    spec = spec_of(kind, c_in=c_in)
    params = params_of(spec, seed=5, centre=True)
    cfg = configs_of(spec, 8, seed=6)
    a, phi = cnn.forward(params, cfg, spec)
    signs = []
    for b in range(cfg.shape[0]):
        z = loop_forward(params, cfg[b], spec)
        w = math.prod(z)
        signs.append(w < 0)
        assert abs(np.exp(a[b] + 1j * phi[b]) - w) <= 1e-12 * abs(w)
    assert any(signs) and not all(signs)     # both signs of the product occur


# ---------------------------------------------------------------- finite differences
@pytest.mark.parametrize('kind', KINDS)
@pytest.mark.parametrize('c_in', [1, 3])
def test_backward_matches_central_differences(kind, c_in):
    # output neurons near 1 (not centred): with neurons near zero 1/z is large and the differences' own error
    # exceeds the bar; signs enter the derivative only through 1/z
    spec = spec_of(kind, c_in=c_in, C=3, B=3)
    params = params_of(spec, seed=7)
    cfg = configs_of(spec, 3, seed=8)
    _, phi, dA, dPhi = cnn.backward(params, cfg, spec)
    assert not dPhi.any()
    # central differences at h and h / 2 combined by Richardson extrapolation (error O(h^4)): an output neuron
    # near zero makes 1/z, and with it the h^2 term of a plain central difference, large
    h = 1e-5
    P = params.size

    def central(k, step):
        e = np.zeros(P)
        e[k] = step
        ap, php = cnn.forward(params + e, cfg, spec)
        am, phm = cnn.forward(params - e, cfg, spec)
        assert np.array_equal(php, phi) and np.array_equal(phm, phi)   # no sign change under the step
        return (ap - am) / (2 * step)

    num = np.zeros((cfg.shape[0], P))
    for k in range(P):
        num[:, k] = (4.0 * central(k, h / 2) - central(k, h)) / 3.0
    assert np.abs(num - dA).max() <= 1e-6 * max(1.0, np.abs(dA).max())


# ---------------------------------------------------------------- symmetries
def translate(cfg, L, dy, dx):
    return np.roll(cfg.reshape(-1, L, L), shift=(dy, dx), axis=(1, 2)).reshape(cfg.shape[0], -1)


def test_cnn1_invariant_under_even_column_and_any_row_shifts():
    spec = spec_of('cnn1', L=6, C=3, B=3)
    params = params_of(spec, seed=9, centre=True)
    cfg = configs_of(spec, 4, seed=10)
    a, phi = cnn.forward(params, cfg, spec)
    for dy, dx in ((1, 0), (0, 2), (3, 4), (5, 2)):
        a2, phi2 = cnn.forward(params, translate(cfg, 6, dy, dx), spec)
        assert np.abs(a2 - a).max() <= 1e-12 * np.abs(a).max() and np.array_equal(phi2, phi)
    a3, _ = cnn.forward(params, translate(cfg, 6, 0, 1), spec)   # pairs (2j, 2j+1) are not preserved
    assert np.abs(a3 - a).max() > 1e-6


def test_cnn2_invariant_under_row_shifts():
    spec = spec_of('cnn2', L=5, C=3, B=3)
    params = params_of(spec, seed=11, centre=True)
    cfg = nqs_synth.random_configs(25, 13, 12, 4, seed=12)
    a, phi = cnn.forward(params, cfg, spec)
    for dy in (1, 2, 4):
        a2, phi2 = cnn.forward(params, translate(cfg, 5, dy, 0), spec)
        assert np.abs(a2 - a).max() <= 1e-12 * np.abs(a).max() and np.array_equal(phi2, phi)
    a3, _ = cnn.forward(params, translate(cfg, 5, 0, 1), spec)   # the row-major window crosses row ends
    assert np.abs(a3 - a).max() > 1e-6


# ---------------------------------------------------------------- closed form and enumeration identity
@pytest.mark.parametrize('kind', KINDS)
def test_constant_network_gives_the_closed_form_local_energy(kind):
    spec = spec_of(kind)
    params = np.zeros(cnn_paper.param_count(spec))
    params[-1] = 0.7                               # every output neuron 0.7: W uniform
    ham = hamiltonian.J1J2(4, 1.0, 0.5)
    cfg = configs_of(spec, 10, seed=13)
    e = eloc.local_energy(params, cfg, spec, ham)
    assert np.allclose(e.real, 0.75 * 16, rtol=0, atol=1e-12) and np.abs(e.imag).max() <= 1e-12


@pytest.mark.parametrize('kind', KINDS)
def test_full_enumeration_identity_j1j2(kind):
    """H from the independent Kronecker construction of the spin Hamiltonian."""
    spec = spec_of(kind)
    params = params_of(spec, seed=14, centre=True)
    basis = ed.sector_basis(16, 8, 8)
    ham = hamiltonian.J1J2(4, 1.0, 0.5)
    e = eloc.local_energy_batch(params, basis, spec, ham)
    a, phi = cnn.forward(params, basis, spec)
    psi = np.exp((a - a.max()) + 1j * phi)
    Hf = oracle_refs.heisenberg_full(4, 1.0, 0.5)
    idx = np.array([oracle_refs.full_index(c) for c in basis])
    H = Hf[idx][:, idx]
    w = np.abs(psi) ** 2
    est = (w * e).sum() / w.sum()
    rayleigh = np.vdot(psi, H @ psi) / np.vdot(psi, psi)
    assert abs(est.real - rayleigh.real) <= 1e-12 * abs(rayleigh.real)
    assert abs(est.imag) <= 1e-12 * abs(rayleigh.real)
    assert np.any(phi != 0) and np.any(phi == 0)   # both signs take part
    assert np.std(e.real) > 1e-2


def test_full_enumeration_identity_tj_cnn2():
    spec = cnn_paper.PaperSpec('cnn2', 4, 3, 3, 2)
    params = params_of(spec, seed=15, centre=True)
    ham = hamiltonian.TJ(4, 1.0, 0.4)
    basis = ed.sector_basis(16, 2, 2)
    e = eloc.local_energy_batch(params, basis, spec, ham)
    a, phi = cnn.forward(params, basis, spec)
    psi = np.exp((a - a.max()) + 1j * phi)
    H = ed.sparse_h(basis, ham)
    w = np.abs(psi) ** 2
    est = (w * e).sum() / w.sum()
    rayleigh = np.vdot(psi, H @ psi) / np.vdot(psi, psi)
    assert abs(est - rayleigh) <= 1e-12 * abs(rayleigh)
