"""Variational Monte Carlo driver: repeated stochastic-reconfiguration steps
(Sec. 3.2: sample by |W|^2, local energies, local derivatives, SR update)
through the library's entry points, with one JSON line per step.

Each record holds the step index, the energy per site <E>/N (real part), the
variance of the local energy per site^2 and the naive error bar
sqrt(var / n_samples) / N (no autocorrelation correction), the imaginary part
of <E>/N, the acceptance rate (accepted moves per proposed move, both counted
on the device by the sampler kernels), the SR solver used, its CG iterations
(0 for the sample-space solve), relative residual and convergence flag, and
the per-stage times (CUDA events on the context's stream, ms).

    python -m paper_2204_07816_gb300.vmc --model j1j2 --L 4 --J2 0 --sign-rule \
        --channels 16 --layers 3 --steps 100 --chains 128 --samples-per-chain 8 --log vmc.jsonl
"""

import argparse
import json
import sys
from dataclasses import dataclass

import numpy as np
import torch

from . import nqs


@dataclass
class SolverChoice:
    """Per-step choice between CG (nqs_sr_solve) and the sample-space
    Cholesky solve (nqs_sr_solve_woodbury) from measured times: CG costs
    its last iteration count times its last time per iteration; the
    sample-space solve its last measured time, or before any measurement
    its FP64 work at `fp64_flops` per second. Every `probe_every`-th step
    runs CG so its iteration count stays current."""
    n_samples: int
    n_params: int
    fp64_flops: float = 0.6e12
    probe_every: int = 10
    cg_iters: int = 0
    cg_ms_per_iter: float = 0.0
    woodbury_ms: float = 0.0

    def woodbury_estimate_ms(self):
        if self.woodbury_ms > 0.0:
            return self.woodbury_ms
        m = 2.0 * self.n_samples
        return (m * m * self.n_params + m ** 3 / 3.0) / self.fp64_flops * 1e3

    def pick(self, step):
        if self.cg_iters == 0 or step % self.probe_every == 0 or 2 * self.n_samples > 65536:
            return 'cg'
        return 'woodbury' if self.woodbury_estimate_ms() < self.cg_iters * self.cg_ms_per_iter else 'cg'

    def record(self, method, ms, iters=0):
        if method == 'cg':
            self.cg_iters = max(int(iters), 1)
            self.cg_ms_per_iter = ms / self.cg_iters
        else:
            self.woodbury_ms = ms


def run_vmc(problem, params, n_steps, n_chains, samples_per_chain, burn_in=10, sweeps_between=1,
            precision='bf16', eps=1e-4, rtol=1e-8, max_iter=10000, lr=0.02, seed=0, log=None, device='cuda',
            checkpoint=None, checkpoint_every=0, sr_method='cg'):
    """Run n_steps SR steps from `params` (float64, host or device). log: a
    path or a text file for the JSON lines (None: keep the records only).
    checkpoint / checkpoint_every: save parameters, chains and Philox step
    every so many steps (workflows.save_checkpoint). sr_method: 'cg',
    'woodbury' (sample-space Cholesky) or 'auto' (SolverChoice). Returns
    (final parameters as a float64 host array, list of records)."""
    from .workflows import save_checkpoint
    p = torch.as_tensor(np.asarray(params, dtype=np.float64) if not torch.is_tensor(params) else params,
                        dtype=torch.float64).to(device).contiguous()
    ctx = nqs.Context(problem, p, seed=seed)
    N = problem.L * problem.L
    n_samples = n_chains * samples_per_chain
    stream = torch.cuda.current_stream(device)
    O = torch.empty((2 * n_samples, ctx.P), dtype=torch.float64, device=device)
    out = open(log, 'a') if isinstance(log, str) else log
    records = []
    ctx.sampler_counts(reset=True)
    choice = SolverChoice(n_samples, ctx.P)
    try:
        for step in range(n_steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            burn = burn_in if step == 0 else 0
            ev[0].record(stream)
            cfg, _ = ctx.sample(n_chains, samples_per_chain, sweeps_between, burn, precision)
            ev[1].record(stream)
            e = ctx.local_energy(cfg, None, precision)
            ev[2].record(stream)
            ctx.logpsi_grad(cfg, precision, out=O)
            ev[3].record(stream)
            method = choice.pick(step) if sr_method == 'auto' else sr_method
            if method == 'cg':
                _, info = ctx.sr_solve(O, e, eps=eps, rtol=rtol, max_iter=max_iter, lr=lr, apply_update=True)
            else:
                _, info = ctx.sr_solve_woodbury(O, e, eps=eps, lr=lr, apply_update=True)
                info.update(iters=0, converged=True)
            ev[4].record(stream)
            moves, accepted = ctx.sampler_counts(reset=True)
            ev[4].synchronize()
            choice.record(method, ev[3].elapsed_time(ev[4]), info['iters'])
            eh = e.cpu().numpy()
            var = float(eh[:, 0].var())
            rec = {'step': step, 'energy_per_site': float(eh[:, 0].mean()) / N,
                   'energy_imag_per_site': float(eh[:, 1].mean()) / N,
                   'variance_per_site2': var / N ** 2, 'error_per_site': float(np.sqrt(var / n_samples)) / N,
                   'acceptance': accepted / max(moves, 1), 'moves': moves, 'accepted': accepted,
                   'cg_iters': int(info['iters']), 'cg_residual': float(info['resid']),
                   'cg_converged': bool(info['converged']), 'sr_method': method,
                   'stage_ms': {k: ev[i].elapsed_time(ev[i + 1])
                                for i, k in enumerate(('sample', 'eloc', 'grad', 'sr'))}}
            records.append(rec)
            if out is not None:
                out.write(json.dumps(rec) + '\n')
                out.flush()
            if checkpoint and checkpoint_every and (step + 1) % checkpoint_every == 0:
                save_checkpoint(checkpoint, ctx, n_chains, step_index=step + 1)
    finally:
        if isinstance(log, str) and out is not None:
            out.close()
    final = ctx.params.detach().cpu().numpy().copy()
    ctx.close()
    return final, records


def main(argv=None):
    import nqs_synth
    ap = argparse.ArgumentParser(description=__doc__.split('\n\n')[0])
    ap.add_argument('--model', choices=['j1j2', 'tj'], default='j1j2')
    ap.add_argument('--L', type=int, default=4)
    ap.add_argument('--J1', type=float, default=1.0)
    ap.add_argument('--J2', type=float, default=0.5)
    ap.add_argument('--t', type=float, default=1.0)
    ap.add_argument('--J', type=float, default=0.4)
    ap.add_argument('--holes', type=int, default=0)
    ap.add_argument('--sign-rule', action='store_true')
    ap.add_argument('--channels', type=int, default=16)
    ap.add_argument('--layers', type=int, default=3)
    ap.add_argument('--steps', type=int, default=50)
    ap.add_argument('--chains', type=int, default=128)
    ap.add_argument('--samples-per-chain', type=int, default=8)
    ap.add_argument('--precision', choices=['fp64', 'fp32', 'bf16'], default='bf16')
    ap.add_argument('--lr', type=float, default=0.02)
    ap.add_argument('--eps', type=float, default=1e-4)
    ap.add_argument('--seed', type=int, default=0)
    ap.add_argument('--init-scale', type=float, default=0.5)
    ap.add_argument('--sr-method', choices=['cg', 'woodbury', 'auto'], default='cg')
    ap.add_argument('--log', default=None, help='JSON lines file (default: stdout)')
    args = ap.parse_args(argv)
    N = args.L * args.L
    if args.model == 'j1j2':
        prob = nqs.make_problem('j1j2', args.L, J1=args.J1, J2=args.J2, sign_rule=args.sign_rule,
                                n_layers=args.layers, channels=args.channels)
        c_in = 1
    else:
        ne = N - args.holes
        prob = nqs.make_problem('tj', args.L, t=args.t, J=args.J, n_up=ne // 2, n_down=ne - ne // 2,
                                n_layers=args.layers, channels=args.channels)
        c_in = 3
    params = nqs_synth.random_params(c_in, args.channels, args.layers, seed=args.seed, scale=args.init_scale)
    run_vmc(prob, params, args.steps, args.chains, args.samples_per_chain, precision=args.precision, eps=args.eps,
            lr=args.lr, seed=args.seed, log=args.log or sys.stdout, sr_method=args.sr_method)


if __name__ == '__main__':
    main()
