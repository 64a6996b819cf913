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
