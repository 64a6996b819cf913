"""Independent constructions used only to pin the oracle.

Nothing here shares code with oracle/: the spin Hamiltonian is assembled from
Kronecker products of single-site spin matrices, and the t-J Hamiltonian from
fermion creation/annihilation operators acting on occupation bit strings
under a different mode ordering (all up modes, then all down modes, sites in
row-major order).
"""

import numpy as np
import scipy.sparse as sp


def lattice_pairs(L, nnn):
    """Bonds of the periodic square lattice from explicit coordinates."""
    nn, nnn_list = [], []
    for y in range(L):
        for x in range(L):
            i = y * L + x
            nn.append((i, y * L + (x + 1) % L))
            nn.append((i, ((y + 1) % L) * L + x))
            nnn_list.append((i, ((y + 1) % L) * L + (x + 1) % L))
            nnn_list.append((i, ((y - 1) % L) * L + (x + 1) % L))
    return nn, (nnn_list if nnn else [])


def _site_op(op, i, N):
    return sp.kron(sp.kron(sp.identity(2 ** i, format='csr'), op), sp.identity(2 ** (N - i - 1), format='csr'), format='csr')


def heisenberg_full(L, J1, J2):
    """Full 2^N J1-J2 Hamiltonian. Single-site basis index 0 = up, 1 = down;
    site 0 is the most significant factor of the Kronecker product."""
    N = L * L
    sz = sp.csr_matrix(np.array([[0.5, 0.0], [0.0, -0.5]]))
    splus = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    sminus = splus.T.tocsr()
    SZ = [_site_op(sz, i, N) for i in range(N)]
    SP = [_site_op(splus, i, N) for i in range(N)]
    SM = [_site_op(sminus, i, N) for i in range(N)]
    nn, nnn = lattice_pairs(L, nnn=True)
    H = sp.csr_matrix((2 ** N, 2 ** N))
    for J, pairs in ((J1, nn), (J2, nnn)):
        for i, j in pairs:
            H = H + J * (SZ[i] @ SZ[j] + 0.5 * (SP[i] @ SM[j] + SM[i] @ SP[j]))
    return H.tocsr()


def full_index(config):
    """Index in heisenberg_full's basis of a +-1 configuration."""
    N = len(config)
    return sum((1 if int(config[i]) == -1 else 0) << (N - 1 - i) for i in range(N))


def _count_below(state, m):
    return bin(state & ((1 << m) - 1)).count('1') & 1


def _annihilate(state, m):
    if not (state >> m) & 1:
        return None, 0
    return state & ~(1 << m), (-1 if _count_below(state, m) else 1)


def _create(state, m):
    if (state >> m) & 1:
        return None, 0
    return state | (1 << m), (-1 if _count_below(state, m) else 1)


def tj_bruteforce(basis, L, t, J):
    """t-J Hamiltonian (Eq. 3) on the given basis (rows of site values
    0/+1/-1) from second-quantised operators. Mode of (site, spin) is
    spin * N + site with spin 0 = up, 1 = down. Doubly occupied results are
    projected out."""
    N = L * L
    def to_state(c):
        s = 0
        for i, v in enumerate(c):
            if v == 1:
                s |= 1 << i
            elif v == -1:
                s |= 1 << (N + i)
        return s
    states = [to_state(c) for c in basis]
    index = {s: k for k, s in enumerate(states)}
    nn, _ = lattice_pairs(L, nnn=False)
    rows, cols, vals = [], [], []

    def add(src_k, st, coef):
        if st is None:
            return
        for i in range(N):
            if (st >> i) & 1 and (st >> (N + i)) & 1:
                return  # doubly occupied: outside the t-J space
        rows.append(index[st])
        cols.append(src_k)
        vals.append(coef)

    def apply(st, ops):
        """ops applied right to left: list of ('c'|'a', mode)."""
        sign = 1
        for kind, m in reversed(ops):
            st, s = (_create if kind == 'c' else _annihilate)(st, m)
            if st is None:
                return None, 0
            sign *= s
        return st, sign

    for k, st in enumerate(states):
        diag = 0.0
        for i, j in nn:
            for spin in (0, 1):
                for a, b in ((i, j), (j, i)):
                    res, sg = apply(st, [('c', spin * N + a), ('a', spin * N + b)])
                    if res is not None:
                        add(k, res, -t * sg)
            nu_i, nd_i = (st >> i) & 1, (st >> (N + i)) & 1
            nu_j, nd_j = (st >> j) & 1, (st >> (N + j)) & 1
            diag += J * ((nu_i - nd_i) * (nu_j - nd_j) / 4.0 - (nu_i + nd_i) * (nu_j + nd_j) / 4.0)
            # S+_i S-_j = c+_{i up} c_{i dn} c+_{j dn} c_{j up}, and its conjugate
            res, sg = apply(st, [('c', i), ('a', N + i), ('c', N + j), ('a', j)])
            if res is not None:
                add(k, res, 0.5 * J * sg)
            res, sg = apply(st, [('c', N + i), ('a', i), ('c', j), ('a', N + j)])
            if res is not None:
                add(k, res, 0.5 * J * sg)
        rows.append(k)
        cols.append(k)
        vals.append(diag)
    M = len(states)
    return sp.csr_matrix((vals, (rows, cols)), shape=(M, M))
