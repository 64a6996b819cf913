"""Continuous batching of stochastic-reconfiguration steps for many
independent lattices (a J2 or doping scan at uneven L).

Every request asks for `n_steps` SR steps of its own problem (Sec. 3.2: MCMC
by |W|^2, local energies, local derivatives, SR update). The server admits
requests in arrival order while their device-memory footprint fits the
budget, keeps each admitted request's parameters and Markov chains resident
in its own context (one CUDA stream each), and runs ticks: in a tick every
active request advances by one SR step,

  1. sampling on each request's own stream,
  2. ONE grouped local-energy launch over all active requests
     (nqs_local_energy_multi: per channel count, blocks move from problem
     to problem), ordered after every request's samples by events,
  3. local derivatives and the SR solve of each request on its own stream,
     issued from one host thread per request so that the streams overlap.

Requests that arrive while others run join at the next tick as soon as the
memory of finished requests is returned. All reductions in the kernels run
in a fixed order and the per-configuration results do not depend on what
else shares a launch, so a request's trajectory is the same alone and in any
mix. Step latency = from the start of the tick to the end of the request's
SR solve; the summary reports p50 / p99 over every step of every request and
the throughput in SR steps and E_loc samples per second.
"""

import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import nqs


@dataclass
class Request:
    rid: int
    model: str = 'j1j2'
    L: int = 6
    J1: float = 1.0
    J2: float = 0.5
    t: float = 1.0
    J: float = 0.4
    n_up: int = None
    n_down: int = None
    n_layers: int = 4
    channels: int = 16
    n_samples: int = 1024
    n_chains: int = 64
    n_steps: int = 2
    seed: int = 0
    arrival: float = 0.0          # seconds after the server starts
    params: np.ndarray = None     # initial parameters (float64, host)
    burn_in: int = 10

    def problem(self):
        N = self.L * self.L
        n_up = self.n_up if self.n_up is not None else N // 2
        n_down = self.n_down if self.n_down is not None else N - n_up
        if self.model == 'j1j2':
            return nqs.make_problem('j1j2', self.L, J1=self.J1, J2=self.J2, n_up=n_up, n_down=n_down,
                                    n_layers=self.n_layers, channels=self.channels)
        return nqs.make_problem('tj', self.L, t=self.t, J=self.J, n_up=n_up, n_down=n_down,
                                n_layers=self.n_layers, channels=self.channels)


@dataclass
class RequestResult:
    rid: int
    energies: list = field(default_factory=list)      # complex <E> per step
    cg_iters: list = field(default_factory=list)
    latencies: list = field(default_factory=list)     # seconds per step
    admitted_at: float = 0.0
    finished_at: float = 0.0
    params: np.ndarray = None                         # final parameters (host)


def footprint_bytes(req):
    """Device memory one admitted request holds (parameters, packed images,
    chains, samples, E_loc, the [2 n, P] local-derivative matrix, SR and
    backward workspace)."""
    prob = req.problem()
    P = nqs.nqs_param_count(prob)
    N = req.L * req.L
    n = req.n_samples
    params = P * 8 * 3
    chains = req.n_chains * N
    samples = n * N + n * 16 * 2
    O = 2 * n * P * 8
    sr = (2 * n + 259 * P) * 8
    grad = 2 * req.n_layers * req.channels * N * 4 * 152 * 2
    return params + chains + samples + O + max(sr, grad) + (4 << 20)


class _Run:
    def __init__(self, req, device, precision, sr_args):
        self.req = req
        self.precision = precision
        self.sr_args = sr_args
        self.stream = torch.cuda.Stream(device)
        prob = req.problem()
        with torch.cuda.stream(self.stream):
            p0 = req.params
            if p0 is None:
                raise ValueError('request %d has no initial parameters' % req.rid)
            self.params = torch.tensor(p0, dtype=torch.float64, device=device)
            self.ctx = nqs.Context(prob, self.params, seed=req.seed, stream=self.stream)
            self.eloc = torch.empty((req.n_samples, 2), dtype=torch.float64, device=device)
            self.O = torch.empty((2 * req.n_samples, self.ctx.P), dtype=torch.float64, device=device)
            self.delta = torch.empty(self.ctx.P, dtype=torch.float64, device=device)
        self.spc = req.n_samples // req.n_chains
        self.steps_done = 0
        self.result = RequestResult(req.rid)
        self.sampled = torch.cuda.Event()
        self.cfg = None

    def sample(self, burn):
        with torch.cuda.stream(self.stream):
            self.cfg, _ = self.ctx.sample(self.req.n_chains, self.spc, 1, burn, self.precision)
        self.sampled.record(self.stream)

    def finish_step(self, eloc_done, tick_start, t0):
        """Backward, SR solve and update on this request's stream (runs in a worker thread)."""
        with torch.cuda.stream(self.stream):
            self.stream.wait_event(eloc_done)
            self.ctx.logpsi_grad(self.cfg, self.precision, out=self.O)
            _, info = self.ctx.sr_solve(self.O, self.eloc, delta=self.delta, apply_update=True, **self.sr_args)
        self.stream.synchronize()
        now = time.perf_counter()
        self.result.latencies.append(now - tick_start)
        self.result.energies.append(info['energy'])
        self.result.cg_iters.append(info['iters'])
        self.steps_done += 1
        if self.steps_done == self.req.n_steps:
            self.result.finished_at = now - t0
            self.result.params = self.params.detach().cpu().numpy().copy()

    def close(self):
        self.ctx.close()
        del self.O, self.eloc, self.delta, self.cfg


class Server:
    def __init__(self, device='cuda', hbm_budget_bytes=None, precision='bf16', eps=1e-4, rtol=1e-8,
                 max_iter=10000, lr=0.02):
        self.device = torch.device(device)
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget_bytes = int(free * 0.8)
        self.budget = hbm_budget_bytes
        self.precision = precision
        self.sr_args = dict(eps=eps, rtol=rtol, max_iter=max_iter, lr=lr)
        self.events = []          # (time, kind, rid) log: 'arrive', 'admit', 'retire'

    def run(self, requests):
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if footprint_bytes(r) > self.budget:
                raise ValueError('request %d needs more memory than the whole budget' % r.rid)
        active, results = [], {}
        used = 0
        t0 = time.perf_counter()
        ticks = 0
        eloc_samples = 0
        while pending or active:
            now = time.perf_counter() - t0
            # admission in arrival order while the footprint fits
            while pending and pending[0].arrival <= now and used + footprint_bytes(pending[0]) <= self.budget:
                req = pending.pop(0)
                run = _Run(req, self.device, self.precision, self.sr_args)
                run.result.admitted_at = now
                used += footprint_bytes(req)
                active.append(run)
                self.events.append((now, 'admit', req.rid))
            if not active:
                time.sleep(max(0.0, min(0.05, pending[0].arrival - now)))
                continue
            tick_start = time.perf_counter()
            for run in active:
                run.sample(run.req.burn_in if run.steps_done == 0 else 0)
            lead = active[0]
            for run in active:
                lead.stream.wait_event(run.sampled)
            with torch.cuda.stream(lead.stream):
                nqs.local_energy_multi([r.ctx for r in active], [r.cfg for r in active], self.precision,
                                       outs=[r.eloc for r in active])
            eloc_done = torch.cuda.Event()
            eloc_done.record(lead.stream)
            eloc_samples += sum(r.req.n_samples for r in active)
            threads = [threading.Thread(target=r.finish_step, args=(eloc_done, tick_start, t0)) for r in active]
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            ticks += 1
            still = []
            for run in active:
                if run.steps_done >= run.req.n_steps:
                    results[run.req.rid] = run.result
                    used -= footprint_bytes(run.req)
                    run.close()
                    self.events.append((time.perf_counter() - t0, 'retire', run.req.rid))
                else:
                    still.append(run)
            active = still
        wall = time.perf_counter() - t0
        lat = np.array([x for r in results.values() for x in r.latencies])
        steps = sum(len(r.latencies) for r in results.values())
        summary = {'requests': len(results), 'sr_steps': steps, 'ticks': ticks, 'wall_s': wall,
                   'sr_steps_per_s': steps / wall, 'eloc_samples_per_s': eloc_samples / wall,
                   'p50_ms': float(np.percentile(lat, 50) * 1e3), 'p99_ms': float(np.percentile(lat, 99) * 1e3)}
        return results, summary
