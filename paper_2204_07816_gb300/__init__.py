"""GB300-native (sm_103a) hot path of CNN-wavefunction variational Monte
Carlo (arXiv 2204.07816): local energies, Metropolis sampling, local
derivatives and the stochastic-reconfiguration solve, behind the C ABI in
include/nqs.h.

Submodules: build (compiles libnqs.so in-tree), nqs (ctypes binding), vmc
(an optimisation loop of SR steps with per-step records), serving
(continuous batching of SR steps across independent lattices), workflows
(initial-state selection, checkpoints, transfer across lattice sizes),
autograd (log psi as a torch.autograd.Function)."""
