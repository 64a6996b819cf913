"""Two procedures of the paper built on the library's entry points.

select_initial_state (Sec. 5.3.2, "Parallel initial state selection"): many
randomly initialised networks, each with its own Markov chains, are sampled
and their energies estimated with one grouped local-energy launch; the
network (and chain state) with the lowest energy is kept as the starting
point of the optimisation.

Checkpoints and transfer across lattice sizes (Sec. 5.3.1, "Transfer
learning for large lattice"): the convolution stack has the same parameter
vector for every L (its length depends on the channel count and the number
of layers only), so parameters saved at L can start a run at L' > L.
save_checkpoint / load_checkpoint keep the parameters, the chain states and
the Philox step of a context; resuming reproduces the next SR step exactly.
"""

import numpy as np
import torch

from . import nqs


def select_initial_state(problem, param_sets, n_chains, samples_per_chain, burn_in=10, precision='bf16',
                         seed=0, device='cuda'):
    """Energies of every candidate network and the index of the lowest.

    problem: nqs_problem shared by the candidates; param_sets: list of float64
    host arrays (candidate initialisations). Candidate k samples with Philox
    key (seed + k). Returns (best_index, energies [complex], contexts)."""
    ctxs = []
    for k, p in enumerate(param_sets):
        t = torch.tensor(np.asarray(p, dtype=np.float64), device=device)
        ctxs.append(nqs.Context(problem, t, seed=seed + k))
    cfgs = []
    for c in ctxs:
        cfg, _ = c.sample(n_chains, samples_per_chain, 1, burn_in, precision)
        cfgs.append(cfg)
    outs = nqs.local_energy_multi(ctxs, cfgs, precision)
    torch.cuda.synchronize(device)
    energies = [complex(o[:, 0].mean().item(), o[:, 1].mean().item()) for o in outs]
    best = int(np.argmin([e.real for e in energies]))
    return best, energies, ctxs


def save_checkpoint(path, context, n_chains, step_index=0):
    """Parameters (float64), chain states, the Philox proposal counter and
    the SR step index of a context."""
    chains, step = context.get_chains(n_chains)
    torch.cuda.synchronize()
    torch.save({'params': context.params.detach().cpu(), 'chains': chains.cpu(), 'philox_step': int(step),
                'step_index': int(step_index), 'L': int(context.problem.L), 'channels': int(context.problem.channels),
                'n_layers': int(context.problem.n_layers)}, path)


def load_checkpoint(path, problem, seed, device='cuda', with_chains=True):
    """A new context for `problem` from a checkpoint. The parameters carry
    over to any lattice size with the same channels and layers; chains and
    the Philox counter are restored only for the same lattice size."""
    ck = torch.load(path)
    if ck['channels'] != problem.channels or ck['n_layers'] != problem.n_layers:
        raise ValueError('checkpoint network shape differs from the problem')
    params = ck['params'].to(device=device, dtype=torch.float64).contiguous()
    ctx = nqs.Context(problem, params, seed=seed)
    if with_chains and ck['L'] == problem.L:
        ctx.set_chains(ck['chains'].to(device).contiguous(), ck['philox_step'])
    return ctx, ck['step_index']
