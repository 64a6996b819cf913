"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).

State: a 4 x 64-bit counter X and a 2 x 64-bit key K. One block applies ten
rounds. Each round, with multipliers M0, M1:
    (hi0, lo0) = M0 * X0        (128-bit product split in halves)
    (hi1, lo1) = M1 * X2
    X <- (hi1 ^ X1 ^ K0,  lo1,  hi0 ^ X3 ^ K1,  lo0)
and between rounds the key is bumped by the Weyl constants
    K0 += W0,  K1 += W1   (mod 2^64).
The output block is the final X (four 64-bit words).

Uses by the method: the Metropolis sampler draws one block per proposal, and
the initial chain states are Fisher-Yates shuffles drawn from the same
generator under another key (sampler.py).
"""

import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15   # golden ratio
W1 = 0xBB67AE8584CAA73B   # sqrt(3) - 1
ROUNDS = 10
MASK64 = (1 << 64) - 1


def philox_block(counter, key):
    """Reference form on Python integers: counter (4 ints), key (2 ints)."""
    x0, x1, x2, x3 = [c & MASK64 for c in counter]
    k0, k1 = [k & MASK64 for k in key]
    for r in range(ROUNDS):
        p0 = M0 * x0
        p1 = M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        if r < ROUNDS - 1:
            k0 = (k0 + W0) & MASK64
            k1 = (k1 + W1) & MASK64
    return x0, x1, x2, x3


_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """Exact 64x64 -> 128-bit product of uint64 arrays, as (hi, lo)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.uint64(b)
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    cross = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (cross >> _S32)
    lo = (cross << _S32) | (ll & _LO32)
    return hi, lo


def philox_blocks(c0, c1, c2, c3, k0, k1):
    """Vectorised form: counter words are uint64 arrays (broadcast), key scalars.

    Returns four uint64 arrays. Must agree bit for bit with philox_block.
    """
    with np.errstate(over='ignore'):
        x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in np.broadcast_arrays(c0, c1, c2, c3))
        k0, k1 = np.uint64(k0 & MASK64), np.uint64(k1 & MASK64)
        for r in range(ROUNDS):
            hi0, lo0 = _mulhilo(x0, M0)
            hi1, lo1 = _mulhilo(x2, M1)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            if r < ROUNDS - 1:
                k0 = k0 + np.uint64(W0)
                k1 = k1 + np.uint64(W1)
    return x0, x1, x2, x3


def mulhi(w, n):
    """floor(w * n / 2^64) for uint64 w and a small positive integer n."""
    hi, _ = _mulhilo(w, n)
    return hi


def unit_double(w):
    """(w >> 11) * 2^-53: a double in [0, 1) using the top 53 bits."""
    return (np.asarray(w, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
