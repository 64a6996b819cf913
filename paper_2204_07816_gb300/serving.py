"""Continuous batching of stochastic-reconfiguration steps for many
independent lattices (a J2 or doping scan at uneven L).

Every request asks for `n_steps` SR steps of its own problem (Sec. 3.2: MCMC
by |W|^2, local energies, local derivatives, SR update). The server admits
requests in arrival order while their device-memory footprint fits the
budget and keeps each admitted request's parameters and Markov chains
resident in its own context, on its own CUDA stream. Each admitted request
runs its own loop of SR steps in a host thread:

  1. sampling on its stream,
  2. its local energies are submitted to a shared batcher, which groups
     every submission pending at that moment into grouped launches
     (nqs_local_energy_multi: blocks move from problem to problem), one per
     cost class (lattices up to 16 x 16, larger ones), each launch with a
     grid share of the SMs proportional to its work so the classes run side
     by side,
  3. local derivatives and the SR solve on its stream.

A request that arrives while others run is admitted as soon as memory is
returned by a finished one and joins the next grouped launch. Sampling is
issued as one launch per sample of every chain (the chains continue from
launch to launch, so the samples are those of one launch), and requests on
lattices up to 16 x 16 use high-priority streams: a large request's sampler
no longer holds every SM for the seconds of a whole step while a small
request waits to start.

Optional SM shares (`partition_sms=True`, `_Partition`): while requests of
both size classes run, the large class (lattices above 16 x 16) is held to
`large_frac` of the SMs and the small class keeps the rest; within a class
the budget is split evenly (at least 4 SMs a request), and a class running
alone gets the whole GPU. Every launch of a request is then sized for its
share (nqs_set_sm_limit; results do not change), and the grouped E_loc
launches of a class are capped at the class budget. On the measured mix
(up to 36 x 36) the shares made every step slower (p50 5.2-5.7 s against
1.6-2.3 s shared): the large requests' sampler and backward, held to fewer blocks,
keep their SMs proportionally longer, and the hardware scheduler already
interleaves the streams; sharing the whole GPU is the default. Every kernel
reduces in a fixed order and per-configuration results do not depend on
what else shares a launch, so a request's trajectory is the same alone and
in any mix. Step latency = from the start of a request's step (sampling) to
the end of its SR update; the summary reports p50 / p99 over every step of
every request and the throughput in SR steps and E_loc samples per second.
"""

import queue
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

    def eloc_cost(self):
        """Relative cost of one local-energy pass: samples x connected
        configurations x sites x per-site network work."""
        N = self.L * self.L
        bonds = (4 if self.model == 'j1j2' else 2) * N
        return float(self.n_samples) * bonds * N * self.channels ** 2 * self.n_layers


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


class _Partition:
    """SM budgets of the running requests (see the module notes)."""

    SMALL_SITES = 256

    def __init__(self, num_sms, large_frac=0.5, min_sms=4):
        self.num_sms = num_sms
        self.large_frac = large_frac
        self.min_sms = min_sms
        self.lock = threading.Lock()
        self.large = {}      # rid -> True for the large class

    @classmethod
    def is_large(cls, req):
        return req.L * req.L > cls.SMALL_SITES

    def add(self, req):
        with self.lock:
            self.large[req.rid] = self.is_large(req)

    def remove(self, rid):
        with self.lock:
            self.large.pop(rid, None)

    def class_budget(self, large):
        """SMs of a class; 0 if the class may use the whole GPU."""
        with self.lock:
            n_large = sum(1 for v in self.large.values() if v)
            n_small = len(self.large) - n_large
        if n_large == 0 or n_small == 0:
            return 0
        b_large = max(self.min_sms, int(round(self.num_sms * self.large_frac)))
        return b_large if large else self.num_sms - b_large

    def limit(self, rid):
        """SMs one request's launches are sized for (0 = whole GPU)."""
        with self.lock:
            large = self.large.get(rid, False)
            n_class = sum(1 for v in self.large.values() if v == large)
        budget = self.class_budget(large) or self.num_sms
        share = max(self.min_sms, budget // max(1, n_class))
        return 0 if share >= self.num_sms else share


class _Run:
    def __init__(self, req, device, precision, sr_args):
        self.req = req
        self.precision = precision
        self.sr_args = sr_args
        # lattices up to 16 x 16 run on high-priority streams: when a block of a large request's launch
        # retires, the block scheduler starts the small requests' pending blocks first
        self.stream = torch.cuda.Stream(device, priority=-1 if req.L * req.L <= _Batcher.SMALL_SITES else 0)
        self.device = device
        with torch.cuda.stream(self.stream):
            if req.params is None:
                raise ValueError('request %d has no initial parameters' % req.rid)
            self.params = torch.tensor(req.params, dtype=torch.float64, device=device)
            self.ctx = nqs.Context(req.problem(), self.params, seed=req.seed, stream=self.stream)
            self.eloc = torch.empty((req.n_samples, 2), dtype=torch.float64, device=device)
            self.O = torch.empty((2 * req.n_samples, self.ctx.P), dtype=torch.float64, device=device)
            self.delta = torch.empty(self.ctx.P, dtype=torch.float64, device=device)
            n_s = req.n_chains * (req.n_samples // req.n_chains)
            self.cfg_buf = torch.empty((n_s, req.L * req.L), dtype=torch.int8, device=device)
            self.lp_buf = torch.empty((n_s, 2), dtype=torch.float64, device=device)
        self.spc = req.n_samples // req.n_chains
        self.result = RequestResult(req.rid)
        self.sampled = torch.cuda.Event()
        self.eloc_done = None
        self.ready = threading.Event()
        self.cfg = None
        self.error = None

    def loop(self, batcher, t0, on_done, partition=None):
        try:
            torch.cuda.set_device(self.device)
            for step in range(self.req.n_steps):
                start = time.perf_counter()
                if partition is not None:
                    self.ctx.set_sm_limit(partition.limit(self.req.rid))
                with torch.cuda.stream(self.stream):
                    # one launch per sample of every chain (burn-in in the first): no request holds the SMs
                    # with a sampler launch of many sweeps while others wait to start theirs
                    nc = self.req.n_chains
                    for k in range(self.spc):
                        self.ctx.sample(nc, 1, 1, self.req.burn_in if (step == 0 and k == 0) else 0,
                                        self.precision, out=self.cfg_buf[k * nc:(k + 1) * nc],
                                        logpsi_out=self.lp_buf[k * nc:(k + 1) * nc])
                    self.cfg = self.cfg_buf
                self.sampled.record(self.stream)
                self.ready.clear()
                batcher.submit(self)
                self.ready.wait()
                if self.error:
                    raise self.error
                with torch.cuda.stream(self.stream):
                    self.stream.wait_event(self.eloc_done)
                    self.ctx.logpsi_grad(self.cfg, self.precision, out=self.O)
                    _, info = self.ctx.sr_solve(self.O, self.eloc, delta=self.delta, apply_update=True, **self.sr_args)
                self.stream.synchronize()
                self.result.latencies.append(time.perf_counter() - start)
                self.result.energies.append(info['energy'])
                self.result.cg_iters.append(info['iters'])
            self.result.finished_at = time.perf_counter() - t0
            self.result.params = self.params.detach().cpu().numpy().copy()
        except Exception as e:      # reported by the server
            self.error = e
        finally:
            on_done(self)

    def close(self):
        self.ctx.close()
        del self.O, self.eloc, self.delta, self.cfg, self.cfg_buf, self.lp_buf


class _Batcher:
    """Groups pending local-energy submissions into grouped launches."""

    SMALL_SITES = 256

    def __init__(self, device, precision, num_sms, window_s=0.0005, partition=None):
        self.q = queue.Queue()
        self.partition = partition
        self.device = device
        self.precision = precision
        self.num_sms = num_sms
        self.window = window_s
        self.samples = 0
        self.launches = 0
        self.stop = False
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def submit(self, run):
        self.q.put(run)

    def _loop(self):
        torch.cuda.set_device(self.device)
        while not self.stop:
            try:
                first = self.q.get(timeout=0.05)
            except queue.Empty:
                continue
            batch = [first]
            time.sleep(self.window)
            while True:
                try:
                    batch.append(self.q.get_nowait())
                except queue.Empty:
                    break
            classes = {}
            for r in batch:
                key = (r.req.L * r.req.L > self.SMALL_SITES, r.req.channels)
                classes.setdefault(key, []).append(r)
            total = sum(r.req.eloc_cost() for r in batch)
            for key, group in classes.items():
                if self.partition is not None:
                    # the class budget, split among the channel groups of that class in this batch
                    budget = self.partition.class_budget(key[0])
                    n_groups = sum(1 for k in classes if k[0] == key[0])
                    blocks = max(8, budget // n_groups) if budget else (self.num_sms // n_groups if n_groups > 1 else 0)
                else:
                    share = sum(r.req.eloc_cost() for r in group) / total
                    blocks = max(8, int(round(self.num_sms * share))) if len(classes) > 1 else 0
                lead = group[0]
                try:
                    for r in group:
                        lead.stream.wait_event(r.sampled)
                    with torch.cuda.stream(lead.stream):
                        nqs.local_energy_multi([r.ctx for r in group], [r.cfg for r in group], self.precision,
                                               outs=[r.eloc for r in group], max_blocks=blocks)
                    done = torch.cuda.Event()
                    done.record(lead.stream)
                    self.launches += 1
                    self.samples += sum(r.req.n_samples for r in group)
                    for r in group:
                        r.eloc_done = done
                except Exception as e:
                    for r in group:
                        r.error = e
                for r in group:
                    r.ready.set()


class Server:
    def __init__(self, device='cuda', hbm_budget_bytes=None, precision='bf16', eps=1e-4, rtol=1e-8,
                 max_iter=10000, lr=0.02, partition_sms=False, large_frac=0.5):
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device('cuda', torch.cuda.current_device())
        if hbm_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget_bytes = int(free * 0.8)
        self.budget = hbm_budget_bytes
        self.precision = precision
        self.sr_args = dict(eps=eps, rtol=rtol, max_iter=max_iter, lr=lr)
        self.partition_sms = partition_sms
        self.large_frac = large_frac
        self.events = []          # (time, kind, rid) log: 'admit', 'retire'

    def run(self, requests):
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in pending:
            if footprint_bytes(r) > self.budget:
                raise ValueError('request %d needs more memory than the whole budget' % r.rid)
        num_sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        partition = _Partition(num_sms, self.large_frac) if self.partition_sms else None
        batcher = _Batcher(self.device, self.precision, num_sms, partition=partition)
        lock = threading.Lock()
        finished = []
        results = {}
        running = {}
        used = 0
        t0 = time.perf_counter()

        def on_done(run):
            with lock:
                finished.append(run)

        try:
            while pending or running:
                now = time.perf_counter() - t0
                with lock:
                    done_now, finished[:] = list(finished), []
                for run in done_now:
                    running.pop(run.req.rid).join()
                    if run.error:
                        raise run.error
                    results[run.req.rid] = run.result
                    if partition is not None:
                        partition.remove(run.req.rid)
                    used -= footprint_bytes(run.req)
                    run.close()
                    self.events.append((time.perf_counter() - t0, 'retire', run.req.rid))
                now = time.perf_counter() - t0
                while pending and pending[0].arrival <= now and used + footprint_bytes(pending[0]) <= self.budget:
                    req = pending.pop(0)
                    run = _Run(req, self.device, self.precision, self.sr_args)
                    run.result.admitted_at = now
                    used += footprint_bytes(req)
                    if partition is not None:
                        partition.add(req)
                    th = threading.Thread(target=run.loop, args=(batcher, t0, on_done, partition), daemon=True)
                    running[req.rid] = th
                    self.events.append((now, 'admit', req.rid))
                    th.start()
                time.sleep(0.001)
        finally:
            batcher.stop = True
            batcher.thread.join(timeout=5)
        wall = time.perf_counter() - t0
        lat = np.array([x for r in results.values() for x in r.latencies])
        steps = sum(len(r.latencies) for r in results.values())
        summary = {'requests': len(results), 'sr_steps': steps, 'grouped_launches': batcher.launches,
                   'wall_s': wall, 'sr_steps_per_s': steps / wall, 'eloc_samples_per_s': batcher.samples / wall,
                   'p50_ms': float(np.percentile(lat, 50) * 1e3), 'p99_ms': float(np.percentile(lat, 99) * 1e3)}
        return results, summary
