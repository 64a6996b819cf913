"""Metropolis exchange sampler for |W(S)|^2 (Sec. 3.2 self-learning procedure:
MCMC performed according to |W(S)|^2; Sec. 5.4.1: many independent chains).

Random numbers come from Philox4x64-10 (philox.py), one 4-word block per use:

  initial state of chain c: the fixed multiset of site values in canonical
      order (up spins, then down spins, then holes) shuffled by Fisher-Yates:
      for k = N-1 down to 1, block B = philox((c, k, 0, 0), (seed, 1)),
      j = floor(B0 * (k+1) / 2^64), swap positions k and j.

  proposal number s (counted from 0 over the life of the chain) of chain c:
      block B = philox((c, s, 0, 0), (seed, 0))
      site i = floor(B0 * N / 2^64)
      direction d = B1 >> 62 selects the nearest neighbour j of i:
          0: x+1, 1: x-1, 2: y+1, 3: y-1 (periodic)
      u = (B2 >> 11) * 2^-53
      If S_i == S_j the proposal is rejected (no move). Otherwise the
      proposal S' = swap(S, i, j) is accepted iff 2(a' - a) >= 0 or
      u < exp(2(a' - a)), where a = log|W(S)|.

  The move exchanges the contents of two neighbouring sites, so it keeps
  the magnetisation (J1-J2) and the numbers of up and down electrons (t-J);
  it is symmetric, and adjacent transpositions connect the whole sector.

  One sweep is N proposals. After `burn_in` sweeps, a sample is recorded at
  the end of every `sweeps_between`-th sweep. Samples are ordered chain-major:
  row c * samples_per_chain + k holds sample k of chain c.
"""

import numpy as np

from . import cnn, lattice, philox

NEIGHBOUR_DIRS = ((1, 0), (-1, 0), (0, 1), (0, -1))


def canonical_values(N, n_up, n_down):
    n_h = N - n_up - n_down
    return np.array([1] * n_up + [-1] * n_down + [0] * n_h, dtype=np.int8)


def init_chains(seed, n_chains, values):
    """[n_chains, N] int8 initial states (Fisher-Yates, key (seed, 1))."""
    values = np.asarray(values, dtype=np.int8)
    N = values.size
    chains = np.tile(values, (n_chains, 1))
    rows = np.arange(n_chains)
    c = np.arange(n_chains, dtype=np.uint64)
    for k in range(N - 1, 0, -1):
        b0, _, _, _ = philox.philox_blocks(c, np.uint64(k), 0, 0, seed, 1)
        j = philox.mulhi(b0, k + 1).astype(np.int64)
        tk = chains[:, k].copy()
        chains[:, k] = chains[rows, j]
        chains[rows, j] = tk
    return chains


def neighbour(i, d, L):
    x, y = i % L, i // L
    dx = np.array([v[0] for v in NEIGHBOUR_DIRS])[d]
    dy = np.array([v[1] for v in NEIGHBOUR_DIRS])[d]
    return ((y + dy) % L) * L + (x + dx) % L


def metropolis(params, spec, chains, step0, seed, samples_per_chain, sweeps_between, burn_in, counts=None):
    """Run every chain; returns (samples, logpsi, chains, a, phi, step).

    counts (optional dict) accumulates 'moves' (proposals whose two sites
    differ) and 'accepted' (moves the Metropolis test accepts).

    chains [n_chains, N] int8 is the start state (not modified). step0 is the
    number of proposals the chains have already made. samples is
    [n_chains * samples_per_chain, N] int8 and logpsi the matching
    [n, 2] float64 (a, phi).
    """
    L = spec.L
    N = L * L
    chains = np.array(chains, dtype=np.int8, copy=True)
    nch = chains.shape[0]
    rows = np.arange(nch)
    cid = np.arange(nch, dtype=np.uint64)
    a, phi = cnn.forward(params, chains, spec)
    samples = np.zeros((nch, samples_per_chain, N), dtype=np.int8)
    logpsi = np.zeros((nch, samples_per_chain, 2))
    n_sweeps = burn_in + samples_per_chain * sweeps_between
    step = step0
    k = 0
    for sweep in range(n_sweeps):
        for _ in range(N):
            b0, b1, b2, _ = philox.philox_blocks(cid, np.uint64(step), 0, 0, seed, 0)
            step += 1
            i = philox.mulhi(b0, N).astype(np.int64)
            d = (b1 >> np.uint64(62)).astype(np.int64)
            u = philox.unit_double(b2)
            j = neighbour(i, d, L)
            differ = chains[rows, i] != chains[rows, j]
            idx = np.nonzero(differ)[0]
            if idx.size == 0:
                continue
            prop = chains[idx].copy()
            ti = prop[np.arange(idx.size), i[idx]].copy()
            prop[np.arange(idx.size), i[idx]] = prop[np.arange(idx.size), j[idx]]
            prop[np.arange(idx.size), j[idx]] = ti
            a_new, phi_new = cnn.forward(params, prop, spec)
            delta = 2.0 * (a_new - a[idx])
            with np.errstate(over='ignore'):
                acc = (delta >= 0.0) | (u[idx] < np.exp(np.minimum(delta, 0.0)))
            if counts is not None:
                counts['moves'] = counts.get('moves', 0) + int(idx.size)
                counts['accepted'] = counts.get('accepted', 0) + int(acc.sum())
            sel = idx[acc]
            chains[sel] = prop[acc]
            a[sel] = a_new[acc]
            phi[sel] = phi_new[acc]
        if sweep >= burn_in and (sweep - burn_in + 1) % sweeps_between == 0:
            samples[:, k] = chains
            logpsi[:, k, 0] = a
            logpsi[:, k, 1] = phi
            k += 1
    return (samples.reshape(-1, N), logpsi.reshape(-1, 2), chains, a, phi, step)
