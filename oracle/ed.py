"""Exact diagonalisation on small lattices (the paper's Sec. 3.1 names ED as
the exact method limited to small systems).

sector_basis   every configuration with fixed numbers of up spins / up
               electrons and down spins / down electrons
sparse_h       the Hamiltonian restricted to that sector, assembled from
               hamiltonian.*.connected_dense (the same matrix elements
               E_loc uses)
lanczos_ground Lanczos with full reorthogonalisation for the lowest
               eigenvalue
"""

import itertools

import numpy as np
import scipy.sparse as sp

from .hamiltonian import swap


def sector_basis(N, n_up, n_down):
    """[M, N] int8 configurations, sorted by their base-3 key."""
    rows = []
    sites = range(N)
    for ups in itertools.combinations(sites, n_up):
        rest = [s for s in sites if s not in ups]
        for downs in itertools.combinations(rest, n_down):
            c = np.zeros(N, dtype=np.int8)
            c[list(ups)] = 1
            c[list(downs)] = -1
            rows.append(c)
    basis = np.array(rows, dtype=np.int8)
    keys = config_keys(basis)
    order = np.argsort(keys)
    return basis[order]


def config_keys(configs):
    """Injective integer key: base-3 digits (value + 1) of each site."""
    c = np.asarray(configs, dtype=np.int64) + 1
    w = 3 ** np.arange(c.shape[1], dtype=object)
    if c.shape[1] <= 39:  # 3^39 < 2^63
        w = (3 ** np.arange(c.shape[1])).astype(np.int64)
        return c @ w
    return np.array([int(sum(int(v) * int(x) for v, x in zip(row, w))) for row in c], dtype=object)


def sparse_h(basis, ham):
    """Sparse CSR Hamiltonian in the sector spanned by `basis` (sorted)."""
    keys = config_keys(basis)
    diag, H = ham.connected_dense(basis)
    M = basis.shape[0]
    rows, cols, vals = [np.arange(M)], [np.arange(M)], [diag]
    for k, (i, j, _) in enumerate(ham.bonds):
        nz = np.nonzero(H[:, k])[0]
        if nz.size == 0:
            continue
        target = swap(basis[nz], i, j)
        tk = config_keys(target)
        idx = np.searchsorted(keys, tk)
        assert np.all(keys[idx] == tk), "connected configuration left the sector"
        rows.append(nz)
        cols.append(idx)
        vals.append(H[nz, k])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(M, M))


def lanczos_ground(H, n_iter=200, seed=0, tol=1e-13):
    """Lowest eigenvalue by Lanczos with full reorthogonalisation."""
    M = H.shape[0]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(M)
    v /= np.linalg.norm(v)
    V = [v]
    alphas, betas = [], []
    prev = None
    w_prev_beta = 0.0
    for _ in range(min(n_iter, M)):
        w = H @ V[-1]
        alpha = V[-1] @ w
        w = w - alpha * V[-1] - (w_prev_beta * V[-2] if len(V) > 1 else 0.0)
        for u in V:                      # full reorthogonalisation
            w -= (u @ w) * u
        beta = np.linalg.norm(w)
        alphas.append(alpha)
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        e0 = np.linalg.eigvalsh(T)[0]
        if prev is not None and abs(e0 - prev) < tol * max(1.0, abs(e0)):
            return e0
        prev = e0
        if beta < 1e-14:
            return e0
        betas.append(beta)
        w_prev_beta = beta
        V.append(w / beta)
    return prev
