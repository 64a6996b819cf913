"""GB300-native (sm_103a) hot path of CNN-wavefunction variational Monte
Carlo (arXiv 2204.07816): local energies, Metropolis sampling, local
derivatives and the stochastic-reconfiguration solve, behind the C ABI in
include/nqs.h.

Submodules: build (compiles libnqs.so in-tree), nqs (ctypes binding),
sr_step (one SR step through the C ABI), serving (continuous batching of SR
steps across independent lattices)."""
