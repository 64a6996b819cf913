"""Seeded synthetic inputs shared by the tests, the benchmark and both
implementations (the CUDA library and the CPU oracle).

This module generates inputs only: random network parameters in the flat
layout both sides agree on, and random configurations uniform over a fixed
sector. It holds none of the method's arithmetic. All generators are numpy
Generator(Philox(seed)) streams.

Parameter layout (float64): for each conv layer W[C_out][C_in][3][3] then
b[C_out]; then the head vectors w_a[C] and w_phi[C]. Every entry is drawn
from N(0, (scale / sqrt(fan_in))^2) with fan_in = 9 * C_in for a conv layer
(weights and biases) and C for the head.
"""

import numpy as np


def layer_dims(c_in, channels, n_layers):
    return [(c_in if l == 0 else channels, channels) for l in range(n_layers)]


def n_params(c_in, channels, n_layers):
    return sum(9 * ci * co + co for ci, co in layer_dims(c_in, channels, n_layers)) + 2 * channels


def random_params(c_in, channels, n_layers, seed, scale=0.5):
    rng = np.random.Generator(np.random.Philox(seed))
    parts = []
    for ci, co in layer_dims(c_in, channels, n_layers):
        std = scale / np.sqrt(9.0 * ci)
        parts.append(rng.standard_normal(9 * ci * co) * std)
        parts.append(rng.standard_normal(co) * std)
    std = scale / np.sqrt(float(channels))
    parts.append(rng.standard_normal(2 * channels) * std)
    return np.concatenate(parts).astype(np.float64)


def paper_param_count(kind, c_in, channels, n_blocks):
    """Parameter count of the paper's CNN1 ('cnn1') / CNN2 ('cnn2') families in the flat layout
    CNN1: per block W[C][C_b][3][3], beta[C], T[C][C_o][2], gamma[C_o] (C_b = c_in first, C_o = 1 last);
    CNN2: E[n_states][C]; per block W[C][C][3][3], beta[C], T[C][C][2], gamma[C]; W_f[1][C][3][3], beta_f[1]."""
    C = channels
    if kind == 'cnn1':
        return sum(9 * C * (c_in if b == 0 else C) + C + 2 * C * (1 if b == n_blocks - 1 else C) +
                   (1 if b == n_blocks - 1 else C) for b in range(n_blocks))
    ns = 2 if c_in == 1 else 3
    return ns * C + n_blocks * (11 * C * C + 2 * C) + 9 * C + 1


def random_paper_params(kind, c_in, channels, n_blocks, seed, scale=0.5):
    """Parameters of CNN1 / CNN2 in their flat layout: every tensor N(0, (scale / sqrt(fan_in))^2) with fan_in
    = 9 C_in (convolutions), C_in (transposed convolutions, kernel 2: one input per output and channel for
    stride 2) or 1 (embedding); the bias of the one-channel output layer is shifted by +1 so that the neurons
    whose product is the amplitude start near 1."""
    rng = np.random.Generator(np.random.Philox(seed))
    C = channels
    parts = []

    def draw(n, fan_in, shift=0.0):
        parts.append(shift + rng.standard_normal(n) * (scale / np.sqrt(float(fan_in))))

    if kind == 'cnn2':
        draw((2 if c_in == 1 else 3) * C, 1)
    for b in range(n_blocks):
        cb = (c_in if b == 0 else C) if kind == 'cnn1' else C
        co = (1 if b == n_blocks - 1 else C) if kind == 'cnn1' else C
        draw(9 * C * cb, 9 * cb)
        draw(C, 9 * cb)
        draw(2 * C * co, C)
        draw(co, C, 1.0 if (kind == 'cnn1' and b == n_blocks - 1) else 0.0)
    if kind == 'cnn2':
        draw(9 * C, 9 * C)
        draw(1, 9 * C, 1.0)
    out = np.concatenate(parts).astype(np.float64)
    assert out.size == paper_param_count(kind, c_in, channels, n_blocks)
    return out


def random_configs(N, n_up, n_down, count, seed):
    """[count, N] int8, uniform over configurations with n_up (+1), n_down (-1)
    and N - n_up - n_down holes (0)."""
    rng = np.random.Generator(np.random.Philox(seed))
    base = np.array([1] * n_up + [-1] * n_down + [0] * (N - n_up - n_down), dtype=np.int8)
    return np.stack([rng.permutation(base) for _ in range(count)]).astype(np.int8)


# Workload shapes (lattice, Hamiltonian couplings, network, sample counts).
WORKLOADS = {
    "j1j2_4x4": dict(model="j1j2", L=4, J1=1.0, J2=0.5, n_up=8, n_down=8, c_in=1,
                     channels=4, n_layers=2, n_samples=1024, n_chains=16),
    "j1j2_10x10": dict(model="j1j2", L=10, J1=1.0, J2=0.5, n_up=50, n_down=50, c_in=1,
                       channels=16, n_layers=6, n_samples=8192, n_chains=256),
    "j1j2_16x16": dict(model="j1j2", L=16, J1=1.0, J2=0.5, n_up=128, n_down=128, c_in=1,
                       channels=32, n_layers=8, n_samples=16384, n_chains=256),
    "tj_12x12": dict(model="tj", L=12, t=1.0, J=0.4, n_up=63, n_down=63, c_in=3,
                     channels=32, n_layers=6, n_samples=8192, n_chains=256),
}
