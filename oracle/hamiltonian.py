"""Hamiltonian matrix elements and connected configurations.

J1-J2 model, Eq. (2):  H = J1 sum_<ij> s_i.s_j + J2 sum_<<ij>> s_i.s_j
with spin-1/2 operators s = sigma/2, sigma_i = +1 (up) or -1 (down).
For a bond b = (i, j) with coupling J_b:
    diagonal      J_b * sigma_i * sigma_j / 4
    off-diagonal  J_b / 2 between sigma and swap(sigma, i, j), present only
                  when sigma_i != sigma_j.
Optional sign rule (Table 1 of the paper lists CNN1 with a sign rule): the
basis is multiplied by (-1)^(number of up spins on the (x+y)-even
sublattice). A nearest-neighbour exchange moves one up spin between the two
sublattices, so the rule flips the sign of the nearest-neighbour off-diagonal
elements only.

t-J model, Eq. (3):
    H = -t sum_<ij>,s (c+_is c_js + h.c.) + J sum_<ij> (s_i.s_j - n_i n_j / 4)
on nearest-neighbour bonds, site values 0 = hole, +1 = up, -1 = down. The
fermions are encoded by a Jordan-Wigner ordering of the modes: sites along
the snake path (lattice.snake_position), and the two spin modes of a site
next to each other. Then
    hop (one hole, one electron on the bond): -t * (-1)^(electrons at snake
        positions strictly between the two sites)
    exchange (up and down on the bond): +J/2, no string sign (it is a
        product of two on-site bilinears)
    diagonal per bond with two electrons: J * (sigma_i sigma_j / 4 - 1/4),
        i.e. -J/2 antiparallel, 0 parallel; bonds with a hole give 0.

Connected configurations of a configuration sigma are listed in bond order
(lattice.bonds); only bonds that change sigma are listed.
"""

import numpy as np

from . import lattice


class J1J2:
    def __init__(self, L, J1=1.0, J2=0.5, sign_rule=False):
        self.L, self.J1, self.J2, self.sign_rule = L, float(J1), float(J2), bool(sign_rule)
        self.bonds = lattice.bonds(L, with_nnn=True)

    def connected(self, sigma):
        """(diag, [(i, j, H_off), ...]) for one configuration, bond order."""
        sigma = [int(v) for v in sigma]
        diag = 0.0
        out = []
        for i, j, nnn in self.bonds:
            J = self.J2 if nnn else self.J1
            diag += J * sigma[i] * sigma[j] / 4.0
            if sigma[i] != sigma[j]:
                h = J / 2.0
                if self.sign_rule and not nnn:
                    h = -h
                out.append((i, j, h))
        return diag, out

    def connected_dense(self, configs):
        """Vectorised over configurations.

        Returns diag [B] and H [B, n_bonds]; H[b, k] is the off-diagonal
        element for bond k (0.0 where the bond does not change the
        configuration). The nonzero entries of a row, in column order, are
        exactly the list returned by ``connected``.
        """
        c = np.asarray(configs, dtype=np.int64)
        diag = np.zeros(c.shape[0])
        H = np.zeros((c.shape[0], len(self.bonds)))
        for k, (i, j, nnn) in enumerate(self.bonds):
            J = self.J2 if nnn else self.J1
            diag += J * c[:, i] * c[:, j] / 4.0
            h = J / 2.0
            if self.sign_rule and not nnn:
                h = -h
            H[:, k] = np.where(c[:, i] != c[:, j], h, 0.0)
        return diag, H


class TJ:
    def __init__(self, L, t=1.0, J=0.4):
        self.L, self.t, self.J = L, float(t), float(J)
        self.bonds = lattice.bonds(L, with_nnn=False)
        self.snake = [lattice.snake_position(i, L) for i in range(L * L)]

    def _electrons_between(self, sigma, i, j):
        lo, hi = sorted((self.snake[i], self.snake[j]))
        return sum(1 for k in range(len(sigma)) if sigma[k] != 0 and lo < self.snake[k] < hi)

    def connected(self, sigma):
        sigma = [int(v) for v in sigma]
        diag = 0.0
        out = []
        for i, j, _ in self.bonds:
            a, b = sigma[i], sigma[j]
            if a != 0 and b != 0:
                diag += self.J * (a * b / 4.0 - 0.25)
                if a != b:
                    out.append((i, j, self.J / 2.0))
            elif (a == 0) != (b == 0):
                n = self._electrons_between(sigma, i, j)
                out.append((i, j, -self.t * (-1.0) ** n))
        return diag, out

    def connected_dense(self, configs):
        c = np.asarray(configs, dtype=np.int64)
        B, N = c.shape
        order = np.argsort(self.snake)             # site at each snake position
        occ = (c[:, order] != 0).astype(np.int64)  # occupation along the snake
        cum = np.concatenate([np.zeros((B, 1), np.int64), np.cumsum(occ, axis=1)], axis=1)
        diag = np.zeros(B)
        H = np.zeros((B, len(self.bonds)))
        for k, (i, j, _) in enumerate(self.bonds):
            a, b = c[:, i], c[:, j]
            both = (a != 0) & (b != 0)
            diag += np.where(both, self.J * (a * b / 4.0 - 0.25), 0.0)
            lo, hi = sorted((self.snake[i], self.snake[j]))
            between = cum[:, hi] - cum[:, lo + 1]    # electrons at positions lo+1 .. hi-1
            hop = (a == 0) != (b == 0)
            H[:, k] = np.where(both & (a != b), self.J / 2.0,
                               np.where(hop, -self.t * (1.0 - 2.0 * (between % 2)), 0.0))
        return diag, H


def swap(sigma, i, j):
    s = np.array(sigma, copy=True)
    s[..., i], s[..., j] = sigma[..., j], sigma[..., i]
    return s
