"""Pins for oracle/hamiltonian.py and oracle/ed.py (CPU only)."""

import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import ed, hamiltonian, lattice
from tests import oracle_refs

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def _heis_golden():
    with open(os.path.join(GOLDEN, 'heisenberg_4x4.json')) as f:
        return json.load(f)


@pytest.fixture(scope='module')
def basis_4x4_sz0():
    return ed.sector_basis(16, 8, 8)


def test_sector_size(basis_4x4_sz0):
    assert basis_4x4_sz0.shape == (12870, 16)
    assert np.all(basis_4x4_sz0.sum(axis=1) == 0)


@pytest.mark.parametrize('J2', [0.0, 0.5])
def test_j1j2_matrix_equals_kronecker_construction(basis_4x4_sz0, J2):
    """The enumeration's matrix elements equal the Kronecker-product spin
    Hamiltonian restricted to Sz = 0, entry by entry (exact: dyadic values)."""
    Hs = ed.sparse_h(basis_4x4_sz0, hamiltonian.J1J2(4, 1.0, J2))
    Hf = oracle_refs.heisenberg_full(4, 1.0, J2)
    idx = np.array([oracle_refs.full_index(c) for c in basis_4x4_sz0])
    Hr = Hf[idx][:, idx]
    diff = (Hs - Hr).tocsr()
    diff.eliminate_zeros()
    assert diff.nnz == 0
    # Sz = 0 block is closed: no weight of the sector rows leaves the sector
    assert abs(Hf[idx].sum() - Hr.sum()) < 1e-12


def test_heisenberg_4x4_ground_energy_textbook(basis_4x4_sz0):
    g = _heis_golden()
    H = ed.sparse_h(basis_4x4_sz0, hamiltonian.J1J2(4, 1.0, 0.0))
    e0 = ed.lanczos_ground(H)
    assert abs(e0 - g['E0']) < g['tolerance']
    e_ref = spla.eigsh(H, k=1, which='SA')[0][0]
    assert abs(e0 - e_ref) < 1e-9


def test_j1j2_4x4_ground_energy_lanczos_vs_eigsh(basis_4x4_sz0):
    H = ed.sparse_h(basis_4x4_sz0, hamiltonian.J1J2(4, 1.0, 0.5))
    assert abs(H - H.T).max() == 0.0
    e0 = ed.lanczos_ground(H)
    e_ref = spla.eigsh(H, k=1, which='SA')[0][0]
    assert abs(e0 - e_ref) < 1e-9
    # frustration raises the energy above the unfrustrated Heisenberg value
    assert -0.60 < e0 / 16 < -0.45


def test_j1j2_sign_rule_is_a_diagonal_gauge(basis_4x4_sz0):
    """With the sign rule the Hamiltonian is D H D for D = (-1)^(ups on the
    even sublattice): same spectrum, integer-exact gauge."""
    H0 = ed.sparse_h(basis_4x4_sz0, hamiltonian.J1J2(4, 1.0, 0.5))
    H1 = ed.sparse_h(basis_4x4_sz0, hamiltonian.J1J2(4, 1.0, 0.5, sign_rule=True))
    even = np.array([lattice.sublattice_a(i, 4) for i in range(16)])
    d = np.where(((basis_4x4_sz0[:, even] == 1).sum(axis=1) % 2) == 0, 1.0, -1.0)
    D = sp.diags(d)
    diff = (D @ H0 @ D - H1).tocsr()
    diff.eliminate_zeros()
    assert diff.nnz == 0


def test_connected_list_matches_dense_form():
    rng = np.random.default_rng(3)
    for ham, N, nu, nd in ((hamiltonian.J1J2(6, 1.0, 0.5), 36, 18, 18),
                           (hamiltonian.TJ(6, 1.0, 0.4), 36, 15, 16)):
        base = np.array([1] * nu + [-1] * nd + [0] * (N - nu - nd))
        for _ in range(5):
            s = rng.permutation(base)
            diag, conn = ham.connected(s)
            d2, H = ham.connected_dense(s[None])
            assert diag == pytest.approx(d2[0], abs=1e-15)
            nz = np.nonzero(H[0])[0]
            assert [(ham.bonds[k][0], ham.bonds[k][1], H[0, k]) for k in nz] == conn


def test_connected_configs_conserve_particle_numbers():
    rng = np.random.default_rng(5)
    ham = hamiltonian.TJ(8, 1.0, 0.4)
    base = np.array([1] * 28 + [-1] * 28 + [0] * 8)
    for _ in range(20):
        s = rng.permutation(base)
        _, conn = ham.connected(s)
        for i, j, _h in conn:
            s2 = hamiltonian.swap(s, i, j)
            assert (s2 == 1).sum() == 28 and (s2 == -1).sum() == 28
            assert s[i] != s[j]


@pytest.mark.parametrize('L,nu,nd', [(3, 2, 2), (3, 3, 3), (4, 2, 1), (4, 2, 2)])
def test_tj_fermion_signs_match_second_quantisation(L, nu, nd):
    """Snake-order hop signs equal brute-force fermion operator algebra under
    another mode ordering, up to a diagonal +-1 gauge (integer exact)."""
    basis = ed.sector_basis(L * L, nu, nd)
    Hs = ed.sparse_h(basis, hamiltonian.TJ(L, 1.0, 0.4))
    Hb = oracle_refs.tj_bruteforce(basis, L, 1.0, 0.4)
    assert oracle_refs.gauge_equivalent(Hb, Hs)


class _NoString(hamiltonian.TJ):
    """Planted mistake: hops without the fermion string sign."""
    def connected_dense(self, configs):
        d, H = super().connected_dense(configs)
        return d, np.where(np.abs(H) == self.t, -self.t, H)


class _SameSpinString(hamiltonian.TJ):
    """Planted mistake: the string counts only electrons of the hopping
    electron's spin (a spin-major ordering) while exchange stays unsigned."""
    def connected_dense(self, configs):
        d, H = super().connected_dense(configs)
        c = np.asarray(configs, dtype=np.int64)
        for k, (i, j, _) in enumerate(self.bonds):
            hop = (c[:, i] == 0) != (c[:, j] == 0)
            spin = c[:, i] + c[:, j]
            lo, hi = sorted((self.snake[i], self.snake[j]))
            mid = [q for q in range(c.shape[1]) if lo < self.snake[q] < hi]
            n = (c[:, mid] == spin[:, None]).sum(1)
            H[hop, k] = -self.t * (1.0 - 2.0 * (n[hop] % 2))
        return d, H


class _InclusiveString(hamiltonian.TJ):
    """Planted mistake: the string also counts the far end of the bond."""
    def connected_dense(self, configs):
        d, H = super().connected_dense(configs)
        c = np.asarray(configs, dtype=np.int64)
        for k, (i, j, _) in enumerate(self.bonds):
            hop = (c[:, i] == 0) != (c[:, j] == 0)
            lo, hi = sorted((self.snake[i], self.snake[j]))
            mid = [q for q in range(c.shape[1]) if lo < self.snake[q] <= hi]
            n = (c[:, mid] != 0).sum(1)
            H[hop, k] = -self.t * (1.0 - 2.0 * (n[hop] % 2))
        return d, H


@pytest.mark.parametrize('mistake', [_NoString, _SameSpinString, _InclusiveString])
@pytest.mark.parametrize('L,nu,nd', [(3, 3, 3), (4, 2, 2)])
def test_tj_sign_mistake_is_caught(mistake, L, nu, nd):
    """The gauge check is sensitive: each planted string-sign mistake breaks it."""
    basis = ed.sector_basis(L * L, nu, nd)
    Hs = ed.sparse_h(basis, mistake(L, 1.0, 0.4))
    Hb = oracle_refs.tj_bruteforce_vec(basis, L, 1.0, 0.4)
    assert not oracle_refs.gauge_equivalent(Hb, Hs)


@pytest.mark.parametrize('L,nu,nd', [(3, 3, 3), (4, 2, 1), (4, 2, 2)])
def test_vectorised_bruteforce_equals_per_state_form(L, nu, nd):
    """The array form of the operator algebra builds exactly the matrix of
    the per-state loop."""
    basis = ed.sector_basis(L * L, nu, nd)
    Hb = oracle_refs.tj_bruteforce(basis, L, 1.0, 0.4)
    Hv = oracle_refs.tj_bruteforce_vec(basis, L, 1.0, 0.4)
    assert (Hb != Hv).nnz == 0


def test_tj_fermion_signs_4x4_two_holes():
    """4x4 with 2 holes and 7 + 7 electrons (411,840 states): snake-order
    signs against the operator algebra, integer exact up to a +-1 gauge."""
    basis = ed.sector_basis(16, 7, 7)
    assert basis.shape == (411840, 16)
    Hs = ed.sparse_h(basis, hamiltonian.TJ(4, 1.0, 0.4))
    assert (Hs != Hs.T).nnz == 0
    Hb = oracle_refs.tj_bruteforce_vec(basis, 4, 1.0, 0.4)
    assert oracle_refs.gauge_equivalent(Hb, Hs)


def test_tj_zero_doping_is_shifted_heisenberg(basis_4x4_sz0):
    """No holes: H = J sum (s.s - 1/4), so E0 = J (E0_Heis - 2N/4)."""
    g = _heis_golden()
    H = ed.sparse_h(basis_4x4_sz0, hamiltonian.TJ(4, 1.0, 0.4))
    e0 = ed.lanczos_ground(H)
    assert abs(e0 - 0.4 * (g['E0'] - 8.0)) < 1e-6
