"""Sensitivity of the oracle's pins: each test plants one plausible mistake in
the oracle (on the CPU, through monkeypatch, undone after the test) and
checks that the pin meant to catch it fails. A pin that still passed with the
mistake in place would not be pinning that part."""

import numpy as np
import pytest

import nqs_synth
from oracle import cnn, ed, eloc, hamiltonian, lattice, philox, sampler, sr
from tests import oracle_refs
from tests import test_oracle_cnn_eloc as cnn_pins
from tests import test_oracle_hamiltonian as ham_pins
from tests import test_oracle_sampler_sr as sr_pins


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ------------------------------------------------------------ Hamiltonians
def test_nnn_bond_direction(monkeypatch):
    """Both next-nearest-neighbour bonds along x + y (the x - y diagonal
    lost): the Kronecker-product comparison at J2 = 0.5 fails."""
    basis = ed.sector_basis(16, 8, 8)
    ham_pins.test_j1j2_matrix_equals_kronecker_construction(basis, 0.5)
    monkeypatch.setattr(lattice, 'NNN_DIRS', ((1, 1), (1, 1)))
    _fails(ham_pins.test_j1j2_matrix_equals_kronecker_construction, basis, 0.5)


def test_exchange_without_half(monkeypatch):
    """Off-diagonal J instead of J/2: the Kronecker-product comparison fails."""
    basis = ed.sector_basis(16, 8, 8)
    dense = hamiltonian.J1J2.connected_dense
    monkeypatch.setattr(hamiltonian.J1J2, 'connected_dense', lambda self, c: (
        dense(self, c)[0], 2.0 * dense(self, c)[1]))
    _fails(ham_pins.test_j1j2_matrix_equals_kronecker_construction, basis, 0.0)


def test_sign_rule_on_every_bond(monkeypatch):
    """The sign rule flipping next-nearest-neighbour exchanges too (they keep
    the up count of each sublattice, so the gauge leaves them alone): the
    full-enumeration identity against the gauge-transformed Kronecker
    Hamiltonian fails."""
    setup = (cnn.NetSpec(4, 1, 4, 2), nqs_synth.random_params(1, 4, 2, seed=7, scale=1.5),
             ed.sector_basis(16, 8, 8))
    dense = hamiltonian.J1J2.connected_dense

    def every_bond(self, c):
        d, H = dense(self, c)
        if self.sign_rule:
            nnn = np.array([b[2] for b in self.bonds])
            H[:, nnn] = -H[:, nnn]
        return d, H
    monkeypatch.setattr(hamiltonian.J1J2, 'connected_dense', every_bond)
    _fails(cnn_pins.test_full_enumeration_identity_j1j2, setup, True)


def test_zero_doping_diagonal_without_quarter(monkeypatch):
    """t-J diagonal J s_i s_j / 4 without the - J n_i n_j / 4 term: the
    zero-doping identity with the shifted Heisenberg energy fails."""
    basis = ed.sector_basis(16, 8, 8)
    dense = hamiltonian.TJ.connected_dense

    def no_quarter(self, c):
        d, H = dense(self, c)
        cc = np.asarray(c, dtype=np.int64)
        pairs = sum(((cc[:, i] != 0) & (cc[:, j] != 0)).astype(float) for i, j, _ in self.bonds)
        return d + 0.25 * self.J * pairs, H
    monkeypatch.setattr(hamiltonian.TJ, 'connected_dense', no_quarter)
    _fails(ham_pins.test_tj_zero_doping_is_shifted_heisenberg, basis)


# ----------------------------------------------------------------- network
def test_convolution_instead_of_cross_correlation(monkeypatch):
    """Shifting by +d instead of -d (a true convolution): translation
    invariance still holds, the explicit-loop comparison does not."""
    monkeypatch.setattr(cnn, 'shifted', lambda h, dy, dx: np.roll(h, shift=(dy, dx), axis=(-2, -1)))
    cnn_pins.test_translation_invariance('j1j2')
    _fails(cnn_pins.test_conv_matches_brute_force_loops)


def test_silu_derivative_missing_term(monkeypatch):
    """silu'(z) taken as sigmoid(z): the finite-difference check of the
    backward fails."""
    monkeypatch.setattr(cnn, 'silu_grad', cnn.sigmoid)
    _fails(cnn_pins.test_backward_matches_central_differences, 4, 1, 4, 2, 8, 8)


def test_phase_head_reads_the_amplitude_weights(monkeypatch):
    """phi = w_a . hbar (the head's weight blocks mixed up): the
    finite-difference check finds d phi / d w_phi = 0 where the backward
    says hbar."""
    unpack = cnn.unpack

    def mixed(params, spec):
        layers, w_a, _ = unpack(params, spec)
        return layers, w_a, w_a
    monkeypatch.setattr(cnn, 'unpack', mixed)
    _fails(cnn_pins.test_backward_matches_central_differences, 4, 1, 4, 2, 8, 8)


# ---------------------------------------------------------- local energies
def test_local_energy_missing_diagonal(monkeypatch):
    """E_loc without H_SS: the zero-network closed form fails."""
    conn = hamiltonian.J1J2.connected
    monkeypatch.setattr(hamiltonian.J1J2, 'connected', lambda self, s: (0.0, conn(self, s)[1]))
    _fails(cnn_pins.test_zero_network_closed_form, 4)


def _eloc_inverted_ratio(params, configs, spec, ham):
    """local_energy_batch with the amplitude ratio turned over,
    W(S)/W(S') in place of W(S')/W(S)."""
    configs = np.asarray(configs)
    diag, H = ham.connected_dense(configs)
    a, phi = cnn.forward(params, configs, spec)
    e = diag.astype(np.complex128)
    for k, (i, j, _) in enumerate(ham.bonds):
        nz = np.nonzero(H[:, k])[0]
        if nz.size:
            a2, phi2 = cnn.forward(params, hamiltonian.swap(configs[nz], i, j), spec)
            e[nz] += H[nz, k] * np.exp((a[nz] - a2) + 1j * (phi[nz] - phi2))
    return e


def test_local_energy_inverted_ratio(monkeypatch):
    """The full-enumeration identity sum |psi|^2 E_loc = <psi|H|psi> fails."""
    setup = (cnn.NetSpec(4, 1, 4, 2), nqs_synth.random_params(1, 4, 2, seed=7, scale=1.5),
             ed.sector_basis(16, 8, 8))
    monkeypatch.setattr(eloc, 'local_energy_batch', _eloc_inverted_ratio)
    _fails(cnn_pins.test_full_enumeration_identity_j1j2, setup, False)


# ----------------------------------------------------------------- sampler
def test_sampler_horizontal_moves_only(monkeypatch):
    """Direction words decoded to +-x only, so no spin ever moves between
    rows. From independent uniform starts the chi-square test does not see
    it (each chain's rows already hold a uniform draw of magnetisations); from
    a common striped start the chains cannot reach the rest of the sector and
    the chi-square test fails."""
    spec = cnn.NetSpec(4, 1, 4, 2)
    params = nqs_synth.random_params(1, 4, 2, seed=21, scale=0.8)
    basis = ed.sector_basis(16, 8, 8)
    a, _ = cnn.forward(params, basis, spec)
    p = np.exp(2 * (a - a.max()))
    p /= p.sum()
    monkeypatch.setattr(sampler, 'NEIGHBOUR_DIRS', ((1, 0), (-1, 0), (1, 0), (-1, 0)))
    _fails(sr_pins.test_sampler_mixes_from_a_common_start, (spec, params, basis, p))


def test_philox_one_round_short(monkeypatch):
    """Nine rounds instead of ten: the comparison with numpy's Philox fails."""
    monkeypatch.setattr(philox, 'ROUNDS', 9)
    _fails(sr_pins.test_philox_matches_numpy, (5, 7, 0, 0), (11, 13))


# ---------------------------------------------------------------------- SR
def _exact_grad_setup():
    spec = cnn.NetSpec(4, 1, 2, 2)
    params = nqs_synth.random_params(1, 2, 2, seed=41, scale=1.2)
    basis = ed.sector_basis(16, 8, 8)
    Hf = oracle_refs.heisenberg_full(4, 1.0, 0.5)
    idx = np.array([oracle_refs.full_index(c) for c in basis])
    return spec, params, basis, Hf[idx][:, idx].tocsr()


def test_s_matrix_uncentred(monkeypatch):
    """S from the raw O instead of the centred O: the Fubini-Study metric
    check fails."""
    def uncentred(dA, dPhi, weights=None):
        w = sr._norm_weights(dA.shape[0], weights)
        return dA.T @ (w[:, None] * dA) + dPhi.T @ (w[:, None] * dPhi)
    monkeypatch.setattr(sr, 's_matrix', uncentred)
    _fails(sr_pins.test_s_matrix_is_the_fubini_study_metric, _exact_grad_setup())


def test_force_uncentred(monkeypatch):
    """F = Re <O* E> with neither O nor E centred: the check F = (1/2) dE/dtheta
    fails."""
    def uncentred(dA, dPhi, e, weights=None):
        e = np.asarray(e, dtype=np.complex128)
        w = sr._norm_weights(e.size, weights)
        return dA.T @ (w * e.real) + dPhi.T @ (w * e.imag), w @ e
    monkeypatch.setattr(sr, 'force', uncentred)
    _fails(sr_pins.test_force_is_half_the_exact_energy_gradient, _exact_grad_setup())


def test_update_with_the_wrong_sign(monkeypatch):
    """theta + eta delta: the exact SR run no longer lowers the energy."""
    monkeypatch.setattr(sr, 'update', lambda params, delta, lr: np.asarray(params) + lr * np.asarray(delta))
    _fails(sr_pins.test_exact_sr_descends_toward_the_ground_state)


# ------------------------------------------------------------ the paper's CNN1 / CNN2
from oracle import cnn_paper  # noqa: E402
from tests import test_oracle_paper_nets as paper_pins  # noqa: E402


def test_transposed_conv_taps_swapped(monkeypatch):
    """CNN1's transposed convolution writing tap 1 to the even site and tap 0
    to the odd one: the explicit-loop comparison fails."""
    real = cnn_paper.tconv

    def swapped(V, T, gamma, kind):
        return real(V, T[:, :, ::-1], gamma, kind) if kind == 'cnn1' else real(V, T, gamma, kind)
    monkeypatch.setattr(cnn_paper, 'tconv', swapped)
    _fails(paper_pins.test_forward_equals_explicit_loops_and_direct_product, 'cnn1', 1)


def test_stride_one_pool_looks_backwards(monkeypatch):
    """CNN2's stride-one pooling over (s - 1, s) instead of (s, s + 1): the
    explicit-loop comparison fails."""
    real = cnn_paper.pool

    def backwards(U, kind):
        if kind == 'cnn2':
            a, b = U, np.roll(U, 1, axis=-1)
            first = a >= b
            return np.where(first, a, b), first
        return real(U, kind)
    monkeypatch.setattr(cnn_paper, 'pool', backwards)
    _fails(paper_pins.test_forward_equals_explicit_loops_and_direct_product, 'cnn2', 1)


def test_product_sign_dropped(monkeypatch):
    """phi = 0 for every configuration (the sign of the product of neurons
    lost): the direct-product comparison fails, although the enumeration
    identity, which uses the same amplitudes on both sides, would not."""
    real = cnn_paper.forward

    def unsigned(params, configs, spec, return_cache=False):
        out = real(params, configs, spec, return_cache)
        return (out[0], np.zeros_like(out[1])) + tuple(out[2:])
    monkeypatch.setattr(cnn_paper, 'forward', unsigned)
    _fails(paper_pins.test_forward_equals_explicit_loops_and_direct_product, 'cnn1', 1)


def test_pool_gradient_to_both_elements(monkeypatch):
    """Max-pooling backward routing every window's gradient to its first
    element: the finite-difference comparison fails."""
    real = cnn_paper.pool

    def both(U, kind):
        V, first = real(U, kind)
        return V, np.ones_like(first) if kind == 'cnn1' else first
    monkeypatch.setattr(cnn_paper, 'pool', both)
    # forward unchanged (V is the max); the backward now routes every gV to the first element
    _fails(paper_pins.test_backward_matches_central_differences, 'cnn1', 1)


def test_embedding_rows_exchanged(monkeypatch):
    """CNN2's embedding reading up spins from the down row: the explicit-loop
    comparison fails."""
    real = cnn_paper.state_index
    monkeypatch.setattr(cnn_paper, 'state_index', lambda configs, spec: 1 - real(configs, spec)
                        if spec.c_in == 1 else real(configs, spec))
    _fails(paper_pins.test_forward_equals_explicit_loops_and_direct_product, 'cnn2', 1)


def test_padding_adjoint_without_wrap(monkeypatch):
    """The adjoint of the periodic padding dropping the wrapped contributions
    (the PBC gradient of Sec. 5.4.2 without its accumulation): the
    finite-difference comparison fails."""
    real = cnn_paper._conv_backward

    def open_boundary(gU, X, W):
        dW, db, dX = real(gU, X, W)
        L = X.shape[-1]
        dX_open = np.zeros_like(dX)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                sh = cnn.shifted(gU, -dy, -dx)
                mask = np.zeros((L, L))
                ys = slice(max(0, dy), L + min(0, dy))
                xs = slice(max(0, dx), L + min(0, dx))
                mask[ys, xs] = 1.0
                dX_open += np.einsum('oc,boyx->bcyx', W[:, :, dy + 1, dx + 1], sh) * mask
        return dW, db, dX_open
    monkeypatch.setattr(cnn_paper, '_conv_backward', open_boundary)
    _fails(paper_pins.test_backward_matches_central_differences, 'cnn2', 1)
