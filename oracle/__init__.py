"""FP64 CPU oracle for the CNN-wavefunction variational Monte Carlo hot path.

This package is TEST INFRASTRUCTURE. Only the test suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it. The
product path (the CUDA library and its Python binding) never calls into it and
fails loudly when its compiled extension is missing.

It is a plain, slow, direct restatement of what the method computes
(arXiv 2204.07816): the wave function of Eq. (1), the J1-J2 Hamiltonian of
Eq. (2), the t-J Hamiltonian of Eq. (3), the local energy of Sec. 5.4.1
("Hotspot energy calculation"), MCMC importance sampling by |W(S)|^2 and the
local derivatives O_loc (Sec. 3.2, self-learning procedure), and the
stochastic-reconfiguration update (Sec. 3.2 and Sec. 5.4.1, "Distributed SR
computation"). Everything is float64 and written for a reader to check by eye.

Modules
-------
lattice      sites, bonds and the snake ordering used for fermion signs
hamiltonian  connected configurations and matrix elements (J1-J2, t-J)
cnn          the convolutional log-amplitude network, forward and backward
cnn_paper    the paper's CNN1 / CNN2 families (max-pooling, transposed
             convolutions, product of neurons), forward and backward
eloc         local energies
philox       Philox4x64-10 counter-based generator (Salmon et al., SC'11)
sampler      Metropolis exchange sampler
sr           stochastic reconfiguration (dense solve and conjugate gradient)
ed           sector bases, sparse Hamiltonians, Lanczos ground energy

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (exact diagonalisation, full enumeration, finite
differences, numpy's Philox, closed forms, brute-force operator algebra),
except where a module docstring says "parity unpinned".
"""
