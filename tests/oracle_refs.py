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


def _apply_ops_vec(states, ops):
    """Operators ('c'|'a', mode) applied right to left to an array of
    occupation bit strings (uint64). Each operator on mode m carries the sign
    (-1)^(number of occupied modes below m). Returns the new strings, their
    signs and a mask of the strings the product does not annihilate."""
    one = np.uint64(1)
    st = states.copy()
    sign = np.ones(len(st), dtype=np.int64)
    alive = np.ones(len(st), dtype=bool)
    for kind, m in reversed(ops):
        bit = one << np.uint64(m)
        occ = (st & bit) != 0
        alive &= ~occ if kind == 'c' else occ
        sign = np.where(np.bitwise_count(st & (bit - one)) & 1, -sign, sign)
        st = (st | bit) if kind == 'c' else (st & ~bit)
    return st, sign, alive


def tj_bruteforce_vec(basis, L, t, J):
    """The same second-quantised construction as tj_bruteforce (mode of
    (site, spin) = spin * N + site), evaluated for all basis states at once
    with array bit operations; used where the per-state loop is too slow."""
    N = L * L
    b = np.asarray(basis)
    w = np.uint64(1) << np.arange(N, dtype=np.uint64)
    states = ((b == 1).astype(np.uint64) * w).sum(1, dtype=np.uint64) | \
        (((b == -1).astype(np.uint64) * w).sum(1, dtype=np.uint64) << np.uint64(N))
    order = np.argsort(states)
    sorted_states = states[order]
    low = (np.uint64(1) << np.uint64(N)) - np.uint64(1)
    M = len(states)
    src = np.arange(M)
    nn, _ = lattice_pairs(L, nnn=False)
    rows, cols, vals = [src], [src], []
    diag = np.zeros(M)

    def bit(m):
        return ((states >> np.uint64(m)) & np.uint64(1)).astype(np.int64)

    def add(ops, coef):
        st, sg, alive = _apply_ops_vec(states, ops)
        alive &= ((st & (st >> np.uint64(N))) & low) == 0     # no doubly occupied site
        st, sg, k = st[alive], sg[alive], src[alive]
        pos = np.searchsorted(sorted_states, st)
        assert np.all(sorted_states[pos] == st)
        rows.append(order[pos])
        cols.append(k)
        vals.append(coef * sg)

    for i, j in nn:
        for spin in (0, 1):
            for a, c in ((i, j), (j, i)):
                add([('c', spin * N + a), ('a', spin * N + c)], -t)
        nu_i, nd_i, nu_j, nd_j = bit(i), bit(N + i), bit(j), bit(N + j)
        diag += J * ((nu_i - nd_i) * (nu_j - nd_j) / 4.0 - (nu_i + nd_i) * (nu_j + nd_j) / 4.0)
        add([('c', i), ('a', N + i), ('c', N + j), ('a', j)], 0.5 * J)
        add([('c', N + i), ('a', i), ('c', j), ('a', N + j)], 0.5 * J)
    vals.insert(0, diag)
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(M, M))
    H.sum_duplicates()
    return H


def gauge_equivalent(A, B):
    """True iff A = D B D for a diagonal D of +-1 (A, B real sparse, same
    shape). D is propagated along a breadth-first tree of A's off-diagonal
    graph, then the identity is checked on every entry (exact for dyadic
    values)."""
    from scipy.sparse import csgraph
    A = sp.csr_matrix(A)
    B = sp.csr_matrix(B)
    if A.shape != B.shape or not np.array_equal(A.diagonal(), B.diagonal()):
        return False
    Ad = (A - sp.diags(A.diagonal())).tocsr()
    Bd = (B - sp.diags(B.diagonal())).tocsr()
    Ad.eliminate_zeros()
    Bd.eliminate_zeros()
    if (abs(Ad) != abs(Bd)).nnz:
        return False
    R = Ad.sign().multiply(Bd.sign()).tocsr()      # A_rc / B_rc on the common pattern
    M = A.shape[0]
    d = np.zeros(M)
    n_comp, labels = csgraph.connected_components(Ad, directed=False)
    for comp in range(n_comp):
        root = int(np.flatnonzero(labels == comp)[0])
        seq, pred = csgraph.breadth_first_order(Ad, root, directed=False, return_predecessors=True)
        d[root] = 1.0
        child = seq[1:]
        ratio = np.asarray(R[pred[child], child]).ravel()
        for c, p, r in zip(child.tolist(), pred[child].tolist(), ratio.tolist()):
            d[c] = r * d[p]
    D = sp.diags(d)
    diff = (D @ Bd @ D - Ad).tocsr()
    diff.eliminate_zeros()
    return diff.nnz == 0
