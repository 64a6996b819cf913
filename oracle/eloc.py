"""Local energy (Sec. 5.4.1, "Hotspot energy calculation").

E_loc(S) = sum_{S'} <S|H|S'> W(S') / W(S)
         = H_SS + sum_k H_k exp((a'_k - a) + i (phi'_k - phi))
where the sum runs over the connected configurations S'_k of S (listed by
hamiltonian.*.connected in bond order) and W = exp(a + i phi) comes from the
network (cnn.forward). The result is complex; the energy estimate is the mean
of the real part over samples drawn from |W|^2.
"""

import numpy as np

from . import cnn
from .hamiltonian import swap


def local_energy_one(params, sigma, spec, ham):
    """E_loc of one configuration as a complex number, summed in bond order."""
    sigma = np.asarray(sigma)
    diag, conn = ham.connected(sigma)
    if not conn:
        return complex(diag, 0.0)
    batch = np.stack([sigma] + [swap(sigma, i, j) for i, j, _ in conn])
    a, phi = cnn.forward(params, batch, spec)
    e = complex(diag, 0.0)
    for k, (_, _, h) in enumerate(conn):
        e += h * np.exp(complex(a[k + 1] - a[0], phi[k + 1] - phi[0]))
    return e


def local_energy(params, configs, spec, ham):
    """[B] complex local energies."""
    return np.array([local_energy_one(params, s, spec, ham) for s in np.asarray(configs)])


def local_energy_batch(params, configs, spec, ham):
    """Same values as local_energy, organised bond by bond over the whole batch
    (one network call per bond) so that full enumeration of a 4x4 sector is
    quick. Terms are added in bond order for every configuration."""
    configs = np.asarray(configs)
    diag, H = ham.connected_dense(configs)
    a, phi = cnn.forward(params, configs, spec)
    e = diag.astype(np.complex128)
    for k, (i, j, _) in enumerate(ham.bonds):
        nz = np.nonzero(H[:, k])[0]
        if nz.size == 0:
            continue
        a2, phi2 = cnn.forward(params, swap(configs[nz], i, j), spec)
        e[nz] += H[nz, k] * np.exp((a2 - a[nz]) + 1j * (phi2 - phi[nz]))
    return e
