#!/usr/bin/env python
"""Benchmark of one stochastic-reconfiguration step of CNN-wavefunction VMC.

A step is one pass of the whole hot path on one batch of synthetic input:
Metropolis sampling (one sample per sweep per chain), local energies of every
sample (connected-configuration enumeration, CNN forwards of all connected
configurations, FP64 reduction), local derivatives O_k, the SR conjugate
gradient to rtol 1e-8 and the parameter update.

Default workload: J1-J2, 10x10 periodic lattice, J2 = 0.5, 6 conv layers of
16 channels, 8192 samples over 256 chains (random-init parameters, synthetic
data). value = E_loc samples/s of the tensor-core path; the plain FP32 path
is measured in the same run for comparison.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = 'E_loc samples/s & SR steps/s vs plain FP32 path, same GB300; p50/p99 step latency'


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=5)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='ours', choices=['ours', 'reference'])
    ap.add_argument('--precision', default='bf16', choices=['bf16', 'fp32', 'fp64', 'fp8'],
                    help='fp8 (local energies only) with --profile-eloc; the SR step reports its FP8 form under "fp8"')
    ap.add_argument('--workload', default='j1j2_10x10')
    ap.add_argument('--compare-steps', type=int, default=2, help='steps of the plain FP32 path')
    ap.add_argument('--oracle-samples', type=int, default=256, help='bounded sample for the CPU oracle')
    ap.add_argument('--profile-eloc', type=int, default=0, metavar='S',
                    help='profiling mode: only run --steps E_loc passes over S uniform random samples')
    ap.add_argument('--serve', type=int, default=0, metavar='R',
                    help='serving mode: R Poisson-arriving SR-step requests of mixed lattices (continuous batching)')
    ap.add_argument('--profile-sample', type=int, default=0, metavar='CHAINS',
                    help='small sampler-only run for profilers: CHAINS chains, 2 samples each')
    ap.add_argument('--profile-grad', type=int, default=0, metavar='S',
                    help='small O_k-only run for profilers: S uniform random samples')
    ap.add_argument('--profile-sr', type=int, default=0, metavar='S',
                    help='small SR-only run for profilers: O and E_loc of S uniform random samples, then --steps '
                         'solves of 8 CG iterations each')
    ap.add_argument('--no-extra', action='store_true',
                    help='skip the other workloads (16x16 SR step, t-J 12x12 E_loc, serving mix) after the main line')
    ap.add_argument('--sr-compare', action='store_true',
                    help='time the CG and the sample-space (Woodbury) SR solves on the same O and E_loc')
    ap.add_argument('--sampler-overlap', action='store_true',
                    help='serving: requests\' sampler launches on their own streams against one launch over the union '
                         'of their chains, and against the same launches back to back')
    ap.add_argument('--serve-partition', action='store_true',
                    help='serving mode with per-class SM shares (default: every request sized for the whole GPU)')
    args = ap.parse_args()
    if args.precision == 'fp8' and not args.profile_eloc:
        ap.error('--precision fp8 runs local energies only: use it with --profile-eloc')
    return args


def serve_mix(n_req, seed=0, mean_gap_s=0.3, steps=2, lattices=(6, 8, 10, 12, 16, 24, 36)):
    """Seeded request mix: J1-J2 at L in `lattices` (default {6, 8, 10, 12, 16, 24, 36}) with J2 ~ U[0.4, 0.6]
    and t-J 12 x 12 at hole doping 1/16 .. 1/8; 6-8 conv layers, 16 or 32 channels (16 at L = 36, where 32 does
    not fit on chip), 2,048-8,192 samples (2,048 for L >= 24); Poisson arrivals."""
    import numpy as np
    import nqs_synth
    from paper_2204_07816_gb300.serving import Request
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(n_req):
        t += rng.exponential(mean_gap_s)
        n_layers = int(rng.integers(6, 9))
        if rng.random() < 0.25:
            n_h = int(rng.choice([10, 12, 14, 16, 18]))
            ch = int(rng.choice([16, 32]))
            ns = int(rng.choice([2048, 4096, 8192]))
            kw = dict(model='tj', L=12, n_up=(144 - n_h) // 2, n_down=(144 - n_h) // 2, n_layers=n_layers, channels=ch)
            c_in = 3
        else:
            L = int(rng.choice(list(lattices)))
            ch = 16 if L == 36 else int(rng.choice([16, 32]))
            ns = 2048 if L >= 24 else int(rng.choice([2048, 4096, 8192]))
            kw = dict(model='j1j2', L=L, J2=float(rng.uniform(0.4, 0.6)), n_layers=n_layers, channels=ch)
            c_in = 1
        params = nqs_synth.random_params(c_in, ch, n_layers, seed=1000 + i)
        reqs.append(Request(rid=i, n_samples=ns, n_chains=256, n_steps=steps, seed=i, arrival=t, params=params, **kw))
    return reqs


def run_serve(args):
    import torch
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300.serving import Server
    nbuild.build()
    reqs = serve_mix(args.serve)
    server = Server(device='cuda', precision='bf16', partition_sms=args.serve_partition)
    results, summary = server.run(reqs)
    summary['sm_partition'] = bool(args.serve_partition)
    per = [{'rid': r.rid, 'model': r.model, 'L': r.L, 'channels': r.channels, 'n_layers': r.n_layers,
            'samples': r.n_samples, 'arrival_s': round(r.arrival, 3),
            'step_ms': [round(x * 1e3, 1) for x in results[r.rid].latencies],
            'cg_iters': results[r.rid].cg_iters} for r in reqs]
    print(json.dumps({'mode': 'serve', 'metric': 'SR-step latency p50/p99 and throughput, continuous batching',
                      'summary': summary, 'requests': per, 'dtype': 'bf16', 'data': 'synthetic'}), flush=True)


def profile_eloc(args):
    """Small, self-contained E_loc run for profilers (no sampler, no SR)."""
    import numpy as np
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs
    nbuild.build()
    w = nqs_synth.WORKLOADS[args.workload]
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    prob = (nqs.make_problem('j1j2', w['L'], J1=w['J1'], J2=w['J2'], n_layers=w['n_layers'], channels=w['channels'])
            if w['model'] == 'j1j2' else
            nqs.make_problem('tj', w['L'], t=w['t'], J=w['J'], n_up=w['n_up'], n_down=w['n_down'],
                             n_layers=w['n_layers'], channels=w['channels']))
    ctx = nqs.Context(prob, torch.tensor(params, dtype=torch.float64, device='cuda'), seed=1)
    cfg = torch.from_numpy(nqs_synth.random_configs(w['L'] ** 2, w['n_up'], w['n_down'], args.profile_eloc, 3)).cuda()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.local_energy(cfg, None, args.precision)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.sync()
    print(json.dumps({'mode': 'profile-eloc', 'workload': args.workload, 'samples': args.profile_eloc,
                      'precision': args.precision, 'ms': times, 'samples_per_s': args.profile_eloc / (min(times) / 1e3)}))


def sampler_overlap(args):
    """Sampling in serving, where each request samples on its own stream: K
    requests of one shape (256 chains each, different parameters) launched
    concurrently on their streams, against one context sampling the union of
    their K x 256 chains (what a grouped sampler launch would do, with the plan
    the launcher picks for that many chains), and against the same K launches
    back to back; then one request of each shape, concurrent against back to
    back. Serving's pattern: one launch per sample of every chain, --steps
    samples. Prints one JSON line per case (best of three, CUDA events)."""
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs
    nbuild.build()
    spc = max(1, args.steps)
    nc = 256
    shapes = [('j1j2_10x10_c16', 'j1j2', 10, 16, 6), ('tj_12x12_c16', 'tj', 12, 16, 7),
              ('j1j2_6x6_c32', 'j1j2', 6, 32, 7), ('j1j2_16x16_c32', 'j1j2', 16, 32, 7)]

    def problem(model, L, C, layers):
        N = L * L
        if model == 'j1j2':
            return nqs.make_problem('j1j2', L, J1=1.0, J2=0.5, n_up=N // 2, n_down=N - N // 2, n_layers=layers,
                                    channels=C)
        holes = N // 16
        return nqs.make_problem('tj', L, t=1.0, J=0.4, n_up=(N - holes) // 2, n_down=N - holes - (N - holes) // 2,
                                n_layers=layers, channels=C)

    def ctx_of(shape, seed, stream):
        _, model, L, C, layers = shape
        params = nqs_synth.random_params(1 if model == 'j1j2' else 3, C, layers, seed)
        return nqs.Context(problem(model, L, C, layers), torch.tensor(params, dtype=torch.float64, device='cuda'),
                           seed=seed, stream=stream)

    def run(ctxs, chains, serial):
        """Each context's spc launches on its own stream; serial: each stream waits for the previous one."""
        cur = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        prev = e0
        ends = []
        for ctx, n in zip(ctxs, chains):
            ctx.stream.wait_event(prev if serial else e0)
            with torch.cuda.stream(ctx.stream):
                for _ in range(spc):
                    ctx.sample(n, 1, 1, 0, 'bf16')
            ev = torch.cuda.Event()
            ev.record(ctx.stream)
            ends.append(ev)
            prev = ev
        for ev in ends:
            cur.wait_event(ev)
        e1.record(cur)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def best(ctxs, chains, serial):
        run(ctxs, chains, serial)    # warm-up (first launch of each plan)
        return min(run(ctxs, chains, serial) for _ in range(3))

    for shape in shapes:
        for K in (2, 4):
            streams = [torch.cuda.Stream() for _ in range(K)]
            ctxs = [ctx_of(shape, 11 + k, streams[k]) for k in range(K)]
            union = ctx_of(shape, 11, torch.cuda.Stream())
            t_conc = best(ctxs, [nc] * K, False)
            t_seq = best(ctxs, [nc] * K, True)
            t_union = best([union], [K * nc], False)
            t_one = best(ctxs[:1], [nc], False)
            plan1 = nqs.tc_plan(ctxs[0].problem, 'sample', nc)
            planK = nqs.tc_plan(ctxs[0].problem, 'sample', K * nc)
            print(json.dumps({'case': shape[0], 'requests': K, 'chains_each': nc, 'samples_per_chain': spc,
                              'one_request_ms': round(t_one, 3), 'concurrent_streams_ms': round(t_conc, 3),
                              'back_to_back_ms': round(t_seq, 3), 'union_launch_ms': round(t_union, 3),
                              'union_over_streams': round(t_union / t_conc, 3),
                              'plan_one': {k: plan1[k] for k in ('G', 'blocks_per_sm', 'grid')},
                              'plan_union': {k: planK[k] for k in ('G', 'blocks_per_sm', 'grid')}}), flush=True)
            for c in ctxs + [union]:
                c.close()
    streams = [torch.cuda.Stream() for _ in shapes]
    ctxs = [ctx_of(sh, 21 + k, streams[k]) for k, sh in enumerate(shapes)]
    t_conc = best(ctxs, [nc] * len(ctxs), False)
    t_seq = best(ctxs, [nc] * len(ctxs), True)
    alone = [best([c], [nc], False) for c in ctxs]
    print(json.dumps({'case': 'mixed: ' + ', '.join(sh[0] for sh in shapes), 'chains_each': nc,
                      'samples_per_chain': spc, 'alone_ms': [round(t, 3) for t in alone],
                      'concurrent_streams_ms': round(t_conc, 3), 'back_to_back_ms': round(t_seq, 3)}), flush=True)
    for c in ctxs:
        c.close()


def sr_compare(args):
    """CG (parameter space) against the sample-space Cholesky solve on the
    same O and E_loc: time, CG iterations, and the difference of the deltas."""
    import numpy as np
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs
    from paper_2204_07816_gb300.vmc import run_vmc
    nbuild.build()
    out = []

    def timed(fn):
        best, res = None, None
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            res = fn()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best, res

    def case(name, prob, params, n, cfg_source, eps=1e-4):
        ctx = nqs.Context(prob, torch.tensor(params, dtype=torch.float64, device='cuda'), seed=5)
        N = prob.L * prob.L
        if cfg_source == 'sampled':
            cfg, _ = ctx.sample(n // 4, 4, 1, 20, 'bf16')
        else:
            cfg = torch.from_numpy(nqs_synth.random_configs(N, prob.n_up, prob.n_down, n, seed=9)).cuda()
        E = ctx.local_energy(cfg, None, 'bf16')
        O = ctx.logpsi_grad(cfg, 'bf16')
        t_cg, (d_cg, info) = timed(lambda: ctx.sr_solve(O, E, eps=eps, rtol=1e-8))
        t_w0, (_, iw0) = timed(lambda: ctx.sr_solve_woodbury(O, E, eps=eps, refine_steps=0))
        t_wb, (d_wb, iw) = timed(lambda: ctx.sr_solve_woodbury(O, E, eps=eps, refine_steps=1))
        m, P = 2 * n, ctx.P
        fl = 2.0 * m * m * P / 2 + m ** 3 / 3.0      # lower-triangle Gram + Cholesky (FLOP)
        rel = float(torch.linalg.norm(d_cg - d_wb) / torch.linalg.norm(d_wb))
        out.append({'case': name, 'P': P, 'samples': n, 'eps': eps, 'cg_ms': round(t_cg, 2), 'cg_iters': info['iters'],
                    'cg_resid': info['resid'], 'woodbury_ms': round(t_wb, 2), 'woodbury_resid': iw['resid'],
                    'woodbury_norefine_ms': round(t_w0, 2), 'woodbury_norefine_resid': iw0['resid'],
                    'woodbury_fp64_tflops': round(fl / (t_w0 * 1e-3) / 1e12, 3), 'delta_rel_diff': rel})
        ctx.close()

    # 4x4 Heisenberg after 60 SR steps (the late-training spectrum that makes CG slow)
    prob4 = nqs.make_problem('j1j2', 4, J1=1.0, J2=0.0, sign_rule=True, n_layers=3, channels=16)
    p4 = nqs_synth.random_params(1, 16, 3, seed=61, scale=0.3)
    p4, _ = run_vmc(prob4, p4, 60, 256, 4, burn_in=20, precision='bf16', eps=1e-3, lr=0.05, seed=62)
    case('heisenberg_4x4_C16_after_60_steps', prob4, p4, 1024, 'sampled', eps=1e-3)
    case('heisenberg_4x4_C16_after_60_steps', prob4, p4, 1024, 'sampled', eps=1e-4)
    w = nqs_synth.WORKLOADS['j1j2_10x10']
    prob10 = nqs.make_problem('j1j2', 10, J1=1.0, J2=0.5, n_layers=6, channels=16)
    p10 = nqs_synth.random_params(1, 16, 6, seed=1)
    for n in (256, 1024, 4096):
        case('j1j2_10x10_C16_L6', prob10, p10, n, 'uniform')
    prob16 = nqs.make_problem('j1j2', 16, J1=1.0, J2=0.5, n_layers=8, channels=32)
    p16 = nqs_synth.random_params(1, 32, 8, seed=1)
    for n in (256, 1024):
        case('j1j2_16x16_C32_L8', prob16, p16, n, 'uniform')
    print(json.dumps({'mode': 'sr-compare', 'cases': out, 'dtype': 'f64', 'data': 'synthetic'}), flush=True)


def profile_stage(args):
    """Small sampler-only or O_k-only run for profilers (bf16 path of the workload)."""
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs
    nbuild.build()
    w = nqs_synth.WORKLOADS[args.workload]
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    prob = (nqs.make_problem('j1j2', w['L'], J1=w['J1'], J2=w['J2'], n_layers=w['n_layers'], channels=w['channels'])
            if w['model'] == 'j1j2' else
            nqs.make_problem('tj', w['L'], t=w['t'], J=w['J'], n_up=w['n_up'], n_down=w['n_down'],
                             n_layers=w['n_layers'], channels=w['channels']))
    ctx = nqs.Context(prob, torch.tensor(params, dtype=torch.float64, device='cuda'), seed=1)
    if args.profile_sample:
        ctx.sample(args.profile_sample, 1, 1, 5, args.precision)      # burn-in outside the timed launches
    else:
        cfg = torch.from_numpy(nqs_synth.random_configs(w['L'] ** 2, w['n_up'], w['n_down'], args.profile_grad,
                                                        3)).cuda()
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if args.profile_sample:
            ctx.sample(args.profile_sample, 2, 1, 0, args.precision)
        else:
            ctx.logpsi_grad(cfg, args.precision)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.sync()
    print(json.dumps({'mode': 'profile-sample' if args.profile_sample else 'profile-grad', 'workload': args.workload,
                      'chains' if args.profile_sample else 'samples': args.profile_sample or args.profile_grad,
                      'precision': args.precision, 'ms': times}))


def _problem_of(nqs, w):
    if w['model'] == 'j1j2':
        return nqs.make_problem('j1j2', w['L'], J1=w['J1'], J2=w['J2'], n_layers=w['n_layers'], channels=w['channels'])
    return nqs.make_problem('tj', w['L'], t=w['t'], J=w['J'], n_up=w['n_up'], n_down=w['n_down'],
                            n_layers=w['n_layers'], channels=w['channels'])


def sx_iteration(ctx, O, e, iters=(4, 12)):
    """Device time of one CG iteration (two passes over O and the P-vector kernels): solves of exactly iters[0]
    and iters[1] iterations (rtol 0), timed with CUDA events on the context's stream; the difference divided by
    the iteration difference."""
    import torch
    times = []
    for k in iters:
        best = None
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = ctx.sr_solve(O, e, eps=1e-4, rtol=0.0, max_iter=k, lr=0.0)
            e1.record()
            torch.cuda.synchronize()
            assert info['iters'] == k, info
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        times.append(best)
    return (times[1] - times[0]) / (iters[1] - iters[0])


def float_exact(O):
    """True when every element of the float64 O is a float (the float32 and bf16 local derivatives are): the CG
    then reads only the float plane of its split of O, 4 bytes an element."""
    import torch
    return bool((O.to(torch.float32).to(torch.float64) == O).all().item())


def sx_roofline(n_samples, P, iter_ms, peaks, narrow):
    """Roofline entry of the S x products: algorithmic bytes per CG iteration = 2 passes x 2 n_samples x P x the
    bytes the passes read an element (4 from the float plane when O is made of floats, else 8 from the two planes),
    against the measured copy bandwidth. The passes multiply-add in double-float arithmetic on the float32 pipes;
    the float64 FLOP rate they stand in for (4 x 2 n_samples x P per iteration) is reported beside the nominal FP64
    rate that a float64 FMA per element would be bound by."""
    bpe = 4 if narrow else 8
    bytes_it = 2.0 * 2 * n_samples * P * bpe
    flop_it = 4.0 * 2 * n_samples * P
    gbs = bytes_it / (iter_ms / 1e3) / 1e9
    tfs = flop_it / (iter_ms / 1e3) / 1e12
    return {'kernels': 'gemv_rows_df_kernel + gemv_cols_df_kernel (+ P-vector kernels)', 'ms_per_cg_iteration': iter_ms,
            'planes': 'float plane only (O made of floats)' if narrow else 'float and low planes',
            'bytes_per_iteration': bytes_it, 'flop_per_iteration': flop_it,
            'hbm': {'achieved': gbs, 'peak': peaks['hbm_gbs'], 'unit': 'GB/s', 'frac': gbs / peaks['hbm_gbs']},
            'fp64_equivalent': {'achieved': tfs, 'nominal_fp64_peak': 1.25, 'unit': 'TFLOP/s',
                                'what': 'float64 multiply-adds done in double-float on the FP32 pipes'}}


def profile_sr(args):
    """Small SR-only run for profilers: O and E_loc of S uniform random samples (bf16 path), then --steps solves
    of exactly 8 CG iterations each."""
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs
    nbuild.build()
    w = nqs_synth.WORKLOADS[args.workload]
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    ctx = nqs.Context(_problem_of(nqs, w), torch.tensor(params, dtype=torch.float64, device='cuda'), seed=1)
    cfg = torch.from_numpy(nqs_synth.random_configs(w['L'] ** 2, w['n_up'], w['n_down'], args.profile_sr, 3)).cuda()
    e = ctx.local_energy(cfg, None, args.precision)
    O = ctx.logpsi_grad(cfg, args.precision)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.sr_solve(O, e, eps=1e-4, rtol=0.0, max_iter=8, lr=0.0)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.sync()
    print(json.dumps({'mode': 'profile-sr', 'workload': args.workload, 'samples': args.profile_sr,
                      'P': ctx.P, 'ms_per_8_iterations': times}))


class UtilSampler:
    """GPU utilisation (the share of time a kernel was running) sampled by nvidia-smi while a region runs."""

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix='.csv')
        os.close(fd)
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '--query-gpu=uuid,utilization.gpu', '--format=csv,noheader,nounits',
                                          '-lms', '100', '-f', self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        vals = []
        with open(self.path) as f:
            for line in f:
                parts = [q.strip() for q in line.split(',')]
                if len(parts) == 2 and (not self.uuid or self.uuid in parts[0]) and parts[1].isdigit():
                    vals.append(float(parts[1]))
        os.unlink(self.path)
        return {'mean_pct': statistics.mean(vals), 'samples': len(vals)} if vals else None


def extra_workloads(args, peaks, uuid, pool, cores):
    """The metric's other workloads on the same GPU, after the main line: the 16x16 SR step (32 channels,
    8 layers, 16,384 samples), t-J 12x12 E_loc (32 channels, 8,192 samples) with its energy checks, and a short
    serving mix of lattices up to 16x16 (continuous batching; p50/p99, throughput, GPU-busy share)."""
    import numpy as np
    import torch

    import nqs_synth
    from paper_2204_07816_gb300 import nqs
    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    def tc_roofline(w, ctx, cfg, eloc_ms):
        n = cfg.shape[0]
        n_conn, pairs, _, _ = ctx.connected(cfg)
        flops, flops_dense = eloc_algorithmic_flops(w, n, pairs, n_conn)
        peak = peaks.get('bf16_tflops_sustained') or peaks['bf16_tflops']
        ach = flops / (eloc_ms / 1e3) / 1e12
        ach_d = flops_dense / (eloc_ms / 1e3) / 1e12
        return {'bound': 'tensor', 'achieved': ach, 'peak': peak, 'unit': 'TFLOP/s', 'frac': ach / peak,
                'dense_form': {'achieved': ach_d, 'frac': ach_d / peak},
                'flops': 'cone form %.4g, dense form %.4g per launch' % (flops, flops_dense)}

    # ---- 16 x 16 J1-J2, 32 channels, 8 layers: one SR step = sample + E_loc + O_k + CG + update
    w = nqs_synth.WORKLOADS['j1j2_16x16']
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    ctx = nqs.Context(_problem_of(nqs, w), torch.tensor(params, dtype=torch.float64, device='cuda'), seed=11)
    P = ctx.P
    spc = w['n_samples'] // w['n_chains']
    stages = []
    infos = []
    for k in range(3):   # one warm-up step (with burn-in), two timed
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        cfg, _ = ctx.sample(w['n_chains'], spc, 1, 10 if k == 0 else 0, 'bf16')
        ev[1].record(stream)
        e = ctx.local_energy(cfg, None, 'bf16')
        ev[2].record(stream)
        O = ctx.logpsi_grad(cfg, 'bf16')
        ev[3].record(stream)
        _, info = ctx.sr_solve(O, e, eps=1e-4, rtol=1e-8, max_iter=min(P, 10000), lr=0.02, apply_update=True)
        ev[4].record(stream)
        torch.cuda.synchronize()
        if k > 0:
            stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
            infos.append(info)
    st = np.array(stages)
    eloc_ms = float(st[:, 1].mean())
    it_ms = sx_iteration(ctx, O, e)
    sub = cfg[:32].contiguous()
    e64 = ctx.local_energy(sub, None, 'fp64').cpu().numpy()
    e16 = ctx.local_energy(sub, None, 'bf16').cpu().numpy()
    out['j1j2_16x16'] = {
        'workload': 'J1-J2 16x16, 8 conv layers x 32 channels (P = %d), %d samples / %d chains' % (
            P, w['n_samples'], w['n_chains']),
        'sr_steps_per_s': 1000.0 / float(st.sum(axis=1).mean()),
        'stage_ms': {k: float(st[:, i].mean()) for i, k in enumerate(['sample', 'eloc', 'grad', 'sr'])},
        'cg_iters': [int(i['iters']) for i in infos],
        'eloc_samples_per_s': w['n_samples'] / (eloc_ms / 1e3),
        'roofline_eloc': tc_roofline(w, ctx, cfg, eloc_ms),
        'sx': sx_roofline(w['n_samples'], P, it_ms, peaks, float_exact(O)),
        'energy_per_site_vs_fp64_gpu': abs(e16[:, 0].mean() - e64[:, 0].mean()) / w['L'] ** 2,
        'fp64_check_samples': int(sub.shape[0])}
    del O
    ctx.close()
    torch.cuda.empty_cache()

    # ---- t-J 12 x 12, 32 channels, 6 layers: E_loc of 8,192 sampled configurations
    w = nqs_synth.WORKLOADS['tj_12x12']
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    ctx = nqs.Context(_problem_of(nqs, w), torch.tensor(params, dtype=torch.float64, device='cuda'), seed=12)
    cfg, _ = ctx.sample(w['n_chains'], w['n_samples'] // w['n_chains'], 1, 10, 'bf16')
    ctx.local_energy(cfg, None, 'bf16')
    times = []
    for _ in range(3):
        e, t = timed(lambda: ctx.local_energy(cfg, None, 'bf16'))
        times.append(t)
    eloc_ms = float(np.mean(times))
    sub = cfg[:256].contiguous()
    e64 = ctx.local_energy(sub, None, 'fp64').cpu().numpy()
    e16 = e[:256].cpu().numpy()
    N = w['L'] ** 2
    osub = cfg[:min(args.oracle_samples, 32)].cpu().numpy()
    e_or, _ = oracle_eloc('tj_12x12', params, osub, pool, cores)
    out['tj_12x12'] = {
        'workload': 't-J 12x12 (t=1, J=0.4, 18 holes), 6 conv layers x 32 channels, %d sampled configurations' %
                    w['n_samples'],
        'eloc_samples_per_s': w['n_samples'] / (eloc_ms / 1e3), 'eloc_ms': eloc_ms,
        'roofline_eloc': tc_roofline(w, ctx, cfg, eloc_ms),
        'energy_per_site_vs_fp64_gpu': abs(e16[:, 0].mean() - e64[:, 0].mean()) / N,
        'fp64_check_samples': int(sub.shape[0]),
        'energy_per_site_vs_oracle_subset': abs(e16[:osub.shape[0], 0].mean() - e_or.real.mean()) / N,
        'oracle_subset_samples': int(osub.shape[0])}
    ctx.close()
    torch.cuda.empty_cache()

    # ---- serving: a seeded mix of lattices up to 16 x 16 arriving faster than they run
    from paper_2204_07816_gb300.serving import Server
    reqs = serve_mix(10, seed=3, mean_gap_s=0.02, steps=2, lattices=(6, 8, 10, 12, 16))
    util = UtilSampler(uuid)
    util.start()
    server = Server(device='cuda', precision='bf16')
    _, summary = server.run(reqs)
    busy = util.stop()
    summary['gpu_busy'] = busy
    summary['mix'] = '10 requests x 2 SR steps: J1-J2 L in {6..16} and t-J 12x12, 16/32 channels, 2,048-8,192 ' \
                     'samples, Poisson arrivals 20 ms apart on average (seed 3)'
    out['serving'] = summary
    return out


def dense_forward_flops(w):
    N = w['L'] ** 2
    fl = 0
    for l in range(w['n_layers']):
        cin = w['c_in'] if l == 0 else w['channels']
        fl += 2 * 9 * cin * w['channels'] * N
    return fl


def cone_sites(L, l, nnn):
    """Sites of layer l's output (l = 1 .. n_layers) that differ between a
    configuration and one with two sites swapped: the union of the two
    (2l+1)^2 squares around the swapped sites on the periodic L x L lattice
    (exact while the squares do not wrap onto themselves, else all sites)."""
    s = 2 * l + 1
    if s + 1 > L:
        return L * L
    return 4 * l * l + 8 * l + 2 if nnn else s * (s + 1)


def cone_forward_flops(w, nnn):
    """FLOPs of the layers' outputs that change for one connected
    configuration (the incremental forward)."""
    fl = 0
    for l in range(w['n_layers']):
        cin = w['c_in'] if l == 0 else w['channels']
        fl += 2 * 9 * cin * w['channels'] * cone_sites(w['L'], l + 1, nnn)
    return fl


def eloc_algorithmic_flops(w, n_samples, pairs, n_conn):
    """(cone form, dense form) FLOPs of one E_loc launch: each sample's own
    dense forward (it is recomputed) plus, per connected configuration, the
    cone (incremental) or the full (dense) forward."""
    import torch
    L = w['L']
    k = torch.arange(pairs.shape[1], device=pairs.device)[None, :] < n_conn[:, None].to(torch.int64)
    i, j = pairs[..., 0].to(torch.int64), pairs[..., 1].to(torch.int64)
    dx = (i % L - j % L).abs()
    dy = (i // L - j // L).abs()
    dx = torch.minimum(dx, L - dx)
    dy = torch.minimum(dy, L - dy)
    nnn = ((dx + dy) == 2) & k
    n_nnn = int(nnn.sum().item())
    n_nn = int(k.sum().item()) - n_nnn
    dense = dense_forward_flops(w)
    cone = n_samples * dense + n_nn * cone_forward_flops(w, False) + n_nnn * cone_forward_flops(w, True)
    return float(cone), float((n_samples + n_nn + n_nnn) * dense)


TRAFFIC_SOURCES = ('tc.cu', 'tc_ptx.cuh', 'common.cuh', 'internal.h')
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one E_loc launch captured by ncu under
# `bench.py --profile-eloc 2048`, with the hash of the kernel sources it was taken on
TRAFFIC_RECORD = {'kernel': 'eloc_rows_kernel', 'samples': 2048, 'dram_bytes': 741632,
                  'source_sha256': '0fd012c4aa373536d53f1a8048253b0b3e102dd888ca0e442bd0a904243f6ae1'}


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, 'paper_2204_07816_gb300', 'csrc', name), 'rb') as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(n_samples, kernel):
    """DRAM bytes (read + write) of one E_loc launch of n_samples, scaled
    linearly from TRAFFIC_RECORD, or None if the record is of another kernel or
    the kernel sources differ from the ones it was taken on."""
    if TRAFFIC_RECORD['kernel'] != kernel or TRAFFIC_RECORD['source_sha256'] != kernel_source_hash():
        return None
    return float(TRAFFIC_RECORD['dram_bytes']) * n_samples / float(TRAFFIC_RECORD['samples'])


def load_peaks():
    path = os.path.join(ROOT, 'MEASURED_PEAKS.json')
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), 'measured'
    return {'hbm_gbs': 6800.0, 'bf16_tflops': 1900.0, 'bf16_tflops_sustained': 1700.0, 'sm_max_mhz': 2070.0}, 'fallback'


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ('index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
              'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
              'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix='.csv')
        os.close(fd)
        try:
            self.proc = subprocess.Popen(['nvidia-smi', '--query-gpu=' + self.FIELDS, '--format=csv,noheader,nounits',
                                          '-lms', '200', '-f', self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(',')]
                if len(parts) < 10:
                    continue
                if self.uuid and self.uuid not in parts[1]:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace('.', '').isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace('.', '').isdigit()]
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == 'active'})
        return {'sm_mhz': statistics.median(sm) if sm else None, 'sm_max_mhz': max(mx) if mx else None,
                'reasons': reasons, 'samples': len(rows)}


# ------------------------------------------------------------------ oracle (CPU baseline, reference arm)
def _oracle_chunk(args):
    wname, params, cfg = args
    import nqs_synth
    from oracle import cnn, eloc, hamiltonian
    w = nqs_synth.WORKLOADS[wname]
    spec = cnn.NetSpec(w['L'], w['c_in'], w['channels'], w['n_layers'])
    ham = (hamiltonian.J1J2(w['L'], w['J1'], w['J2']) if w['model'] == 'j1j2'
           else hamiltonian.TJ(w['L'], w['t'], w['J']))
    return eloc.local_energy(params, cfg, spec, ham)


def oracle_eloc(wname, params, cfg, pool, cores):
    chunks = [(wname, params, c) for c in _split(cfg, cores * 2)]
    t0 = time.perf_counter()
    parts = pool.map(_oracle_chunk, chunks)
    dt = time.perf_counter() - t0
    import numpy as np
    return np.concatenate(parts), dt


def _split(a, k):
    n = a.shape[0]
    step = max(1, (n + k - 1) // k)
    return [a[i:i + step] for i in range(0, n, step)]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    """The reference arm: the FP64 oracle on this machine's host cores, each step a
    bounded sample of the same workload's E_loc."""
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    import numpy as np
    import nqs_synth
    w = nqs_synth.WORKLOADS[args.workload]
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    cores = host_cores()
    per_step = min(args.oracle_samples, 64)
    ctx = mp.get_context('spawn')
    with ctx.Pool(cores) as pool:
        times = []
        for k in range(args.warmup + args.steps):
            cfg = nqs_synth.random_configs(w['L'] ** 2, w['n_up'], w['n_down'], per_step, seed=100 + k)
            _, dt = oracle_eloc(args.workload, params, cfg, pool, cores)
            if k >= args.warmup:
                times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    line = {'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 'samples/s', 'n_gpus': 0,
            'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': 1000 * total / len(times),
            'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
            'data': 'synthetic', 'config': _config(w, args.workload),
            'cpu_baseline': {'value': value, 'unit': 'samples/s', 'cores': cores, 'kind': 'oracle',
                             'sample': '%d uniform random sector configurations per step, E_loc only' % per_step},
            'e2e': {'value': value, 'unit': 'samples/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0}}
    print(json.dumps(line), flush=True)


def _config(w, wname):
    """The workload, identical on both arms (the arithmetic type is the line's dtype)."""
    return {'workload': '%s: %s %dx%d, %d conv layers x %d channels, %d samples / %d chains' % (
        wname, 'J1-J2 (J2=0.5)' if w['model'] == 'j1j2' else 't-J (t=1, J=0.4)', w['L'], w['L'], w['n_layers'],
        w['channels'], w['n_samples'], w['n_chains']),
        'n_samples': w['n_samples'], 'n_chains': w['n_chains'],
        'lattice': '%dx%d' % (w['L'], w['L']), 'sr': {'eps': 1e-4, 'rtol': 1e-8, 'lr': 0.02},
        'l2': 'flushed (256 MB write) before every timed step', 'parallelism': 'replicas'}


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == 'reference':
        run_reference(args)
        return
    if args.profile_eloc:
        profile_eloc(args)
        return
    if args.profile_sample or args.profile_grad:
        profile_stage(args)
        return
    if args.profile_sr:
        profile_sr(args)
        return
    if args.serve:
        run_serve(args)
        return
    if args.sr_compare:
        sr_compare(args)
        return
    if args.sampler_overlap:
        sampler_overlap(args)
        return
    # the oracle's process pool is started before the first GPU call
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local_rank = int(os.environ.get('LOCAL_RANK', '0'))
    cores = host_cores()
    pool = mp.get_context('spawn').Pool(cores) if rank == 0 else None

    import numpy as np
    import torch
    import torch.distributed as dist

    import nqs_synth
    from paper_2204_07816_gb300 import build as nbuild
    from paper_2204_07816_gb300 import nqs

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group('nccl', device_id=torch.device('cuda', local_rank))
    if rank == 0:
        nbuild.build()
    if world > 1:
        dist.barrier()
    nqs.load()

    w = nqs_synth.WORKLOADS[args.workload]
    dev = torch.device('cuda', local_rank)
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    if w['model'] == 'j1j2':
        prob = nqs.make_problem('j1j2', w['L'], J1=w['J1'], J2=w['J2'], n_layers=w['n_layers'],
                                channels=w['channels'])
    else:
        prob = nqs.make_problem('tj', w['L'], t=w['t'], J=w['J'], n_up=w['n_up'], n_down=w['n_down'],
                                n_layers=w['n_layers'], channels=w['channels'])
    n_chains, n_samples = w['n_chains'], w['n_samples']
    spc = n_samples // n_chains
    P = nqs.nqs_param_count(prob)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def new_ctx(seed):
        tp = torch.tensor(params, dtype=torch.float64, device=dev)
        return nqs.Context(prob, tp, seed=seed + 1000 * rank)

    def sr_step(ctx, prec, ev, burn=0):
        ev[0].record(stream)
        cfg, lp = ctx.sample(n_chains, spc, 1, burn, prec)
        ev[1].record(stream)
        e = ctx.local_energy(cfg, None, prec)
        ev[2].record(stream)
        O = ctx.logpsi_grad(cfg, prec)
        ev[3].record(stream)
        _, info = ctx.sr_solve(O, e, eps=1e-4, rtol=1e-8, max_iter=min(P, 10000), lr=0.02, apply_update=True)
        ev[4].record(stream)
        return cfg, e, info

    def run(prec, steps, warmup, sampler_clock=None):
        ctx = new_ctx(7)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(steps)]
        wev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        sr_step(ctx, prec, wev, burn=10)
        for _ in range(max(0, warmup - 1)):
            sr_step(ctx, prec, wev)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler_clock:
            sampler_clock.start()
        l0 = ctx.kernel_launches()
        infos = []
        last = None
        for k in range(steps):
            flush.zero_()
            last = sr_step(ctx, prec, evs[k])
            infos.append(last[2])
        torch.cuda.synchronize()
        launches = ctx.kernel_launches() - l0
        clocks = sampler_clock.stop() if sampler_clock else None
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        stage = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(steps)])
        return ctx, stage, infos, launches, clocks, last

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clock = ClockSampler(uuid)
    ctx, stage, infos, launches, clocks, last = run(args.precision, args.steps, args.warmup, clock)
    step_ms = stage.sum(axis=1)
    eloc_ms = stage[:, 1]
    # max over ranks of the timed totals; whole-job throughput
    eloc_total_ms, step_total_ms = max_over_ranks([eloc_ms.sum(), step_ms.sum()], dev)
    value = job_throughput(n_samples * args.steps, world, eloc_total_ms)
    sr_steps_per_s = job_throughput(args.steps, world, step_total_ms)

    # algorithmic FLOPs of one E_loc launch: the sample's forward plus the
    # changed cone of every connected configuration (the dense form, n_c + 1
    # full forwards per sample, is reported beside it)
    cfg_last, e_last, _ = last
    n_conn_s, pairs, _, _ = ctx.connected(cfg_last)
    flops, flops_dense = eloc_algorithmic_flops(w, n_samples, pairs, n_conn_s)
    del pairs

    # E_loc through the public API with host buffers (copies inside the timed region)
    cfg_host = cfg_last.cpu().pin_memory()
    out_host = torch.empty((n_samples, 2), dtype=torch.float64).pin_memory()
    cfg_dev = torch.empty_like(cfg_last)
    for _ in range(2):
        cfg_dev.copy_(cfg_host, non_blocking=True)
        out_host.copy_(ctx.local_energy(cfg_dev, None, args.precision), non_blocking=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        cfg_dev.copy_(cfg_host, non_blocking=True)
        out_host.copy_(ctx.local_energy(cfg_dev, None, args.precision), non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value = n_samples * args.steps * world / (e0.elapsed_time(e1) / 1000.0)

    # energy check: this path against the FP64 GPU path (all samples) and the oracle (bounded subset)
    e_fp64 = ctx.local_energy(cfg_last, None, 'fp64').cpu().numpy()
    e_this = ctx.local_energy(cfg_last, None, args.precision).cpu().numpy()
    N = w['L'] ** 2
    check = {'energy_per_site_vs_fp64_gpu': abs(e_this[:, 0].mean() - e_fp64[:, 0].mean()) / N,
             'max_abs_eloc_diff_vs_fp64_gpu': float(np.abs(e_this[:, 0] - e_fp64[:, 0]).max())}

    # the FP8 form of the same local energies (row-form plans with 16 channels): the step's last samples, L2
    # flushed before each launch, CUDA events on the context's stream
    fp8 = None
    if args.precision == 'bf16' and w['channels'] == 16 and nqs.tc_plan(prob, 'local_energy', n_samples)['row_form']:
        ctx.local_energy(cfg_last, None, 'fp8')
        torch.cuda.synchronize()
        t8 = []
        for _ in range(args.steps):
            flush.zero_()
            a8, b8 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a8.record(stream)
            e8 = ctx.local_energy(cfg_last, None, 'fp8')
            b8.record(stream)
            torch.cuda.synchronize()
            t8.append(a8.elapsed_time(b8))
        e8 = e8.cpu().numpy()
        ms8 = float(np.mean(t8))
        fp8 = {'eloc_ms': ms8, 'eloc_samples_per_s': n_samples / (ms8 / 1e3),
               'energy_per_site_vs_fp64_gpu': abs(e8[:, 0].mean() - e_fp64[:, 0].mean()) / N,
               'max_abs_eloc_diff_per_site_vs_fp64_gpu': float(np.abs(e8[:, 0] - e_fp64[:, 0]).max()) / N,
               'what': 'layer 0 bf16, layers >= 1 e4m3 operands with per-output-channel weight scales, fp32 '
                       'accumulation, float64 ratios and sums (eloc_rows_kernel, e4m3)'}

    # plain FP32 path on the same workload
    cmp = None
    if args.compare_steps > 0 and args.precision != 'fp32':
        ctx32, st32, inf32, _, _, _ = run('fp32', args.compare_steps, 1)
        cmp = {'eloc_samples_per_s': n_samples * args.compare_steps / (st32[:, 1].sum() / 1000.0),
               'sr_steps_per_s': args.compare_steps / (st32.sum() / 1000.0),
               'ms_per_step': float(st32.sum(axis=1).mean()), 'eloc_ms': float(st32[:, 1].mean())}
        # the baseline's own roofline: the same cone-form FLOPs against the FP32 CUDA-core peak at the clock seen
        mhz32 = (clocks or {}).get('sm_mhz') or 2070.0
        fp32_peak = 152 * 128 * 2 * mhz32 * 1e6 / 1e12
        cmp['eloc_tflops'] = flops / (cmp['eloc_ms'] / 1e3) / 1e12
        cmp['eloc_frac_of_fp32_cuda_core_peak'] = cmp['eloc_tflops'] / fp32_peak
        cmp['fp32_cuda_core_peak_tflops'] = fp32_peak
        ctx32.close()

    line = None
    if rank == 0:
        peaks, peak_kind = load_peaks()
        eloc_launch_s = float(eloc_ms.mean()) / 1000.0
        achieved = flops / eloc_launch_s / 1e12
        if args.precision == 'bf16':
            eloc_kernel = ('eloc_rows_kernel' if nqs.tc_plan(prob, 'local_energy', n_samples)['row_form']
                           else 'eloc_tc_kernel')
            peak = peaks.get('bf16_tflops_sustained') or peaks['bf16_tflops']
            roof = {'bound': 'tensor', 'achieved': achieved, 'peak': peak, 'unit': 'TFLOP/s',
                    'frac': achieved / peak, 'traffic': recorded_traffic(n_samples, eloc_kernel),
                    'kernel': eloc_kernel,
                    'peak_source': '%s bf16 dense (sustained)' % peak_kind,
                    'flops': 'cone form (changed sites only) %.4g per launch' % flops,
                    'dense_form': {'achieved': flops_dense / eloc_launch_s / 1e12,
                                   'frac': flops_dense / eloc_launch_s / 1e12 / peak}}
            if w['channels'] == 16:
                # context: the rate of back-to-back M128 N16 K16 MMAs (39.1 cycles each, bound by the shared-memory
                # operand path, measured with a clock64 probe on GB300) at the clock seen: the ceiling of one MMA
                # per 3x3 tap with 16 channels
                mhz = (clocks or {}).get('sm_mhz') or peaks.get('sm_max_mhz', 2070.0)
                n16 = 152 * (2.0 * 128 * 16 * 16 / 39.1) * mhz * 1e6 / 1e12
                roof['mma_n16_ceiling'] = {'peak': n16, 'frac': achieved / n16,
                                           'dense_form_frac': flops_dense / eloc_launch_s / 1e12 / n16}
        else:
            mhz = (clocks or {}).get('sm_mhz') or peaks.get('sm_max_mhz', 2070.0)
            lanes = 128 if args.precision == 'fp32' else 2
            peak = 152 * lanes * 2 * mhz * 1e6 / 1e12
            roof = {'bound': 'alu', 'achieved': achieved, 'peak': peak, 'unit': 'TFLOP/s', 'frac': achieved / peak,
                    'traffic': None, 'kernel': 'eloc_plain_kernel',
                    'peak_source': '152 SMs x %d lanes x 2 FLOP x %.0f MHz' % (lanes, mhz),
                    'flops': 'cone form (changed sites only) %.4g per launch' % flops,
                    'dense_form': {'achieved': flops_dense / eloc_launch_s / 1e12,
                                   'frac': flops_dense / eloc_launch_s / 1e12 / peak}}
        # S x products of the main workload: one CG iteration timed alone
        O_last = ctx.logpsi_grad(cfg_last, args.precision)
        sx = sx_roofline(n_samples, P, sx_iteration(ctx, O_last, e_last), peaks, float_exact(O_last))
        # the same iteration with the float64 passes (nqs_set_sx_arithmetic NQS_SX_FP64), for comparison
        ctx.set_sx_arithmetic('fp64')
        ms64 = sx_iteration(ctx, O_last, e_last)
        ctx.set_sx_arithmetic('double_float')
        sx['fp64_passes'] = {'ms_per_cg_iteration': ms64,
                             'fp64_tflops': 4.0 * 2 * n_samples * P / (ms64 / 1e3) / 1e12,
                             'fp64_frac_of_nominal': 4.0 * 2 * n_samples * P / (ms64 / 1e3) / 1e12 / 1.25}
        del O_last
        # CPU oracle on a bounded sample of the same workload
        sub = cfg_last[:args.oracle_samples].cpu().numpy()
        e_or, dt_or = oracle_eloc(args.workload, params_at_step(ctx), sub, pool, cores)
        e_sub = ctx.local_energy(cfg_last[:args.oracle_samples], None, args.precision).cpu().numpy()
        check['energy_per_site_vs_oracle_subset'] = abs(e_sub[:, 0].mean() - e_or.real.mean()) / N
        check['oracle_subset_samples'] = int(sub.shape[0])
        if fp8 is not None:
            fp8['energy_per_site_vs_oracle_subset'] = abs(e8[:sub.shape[0], 0].mean() - e_or.real.mean()) / N
            peak8 = 2.0 * (peaks.get('bf16_tflops_sustained') or peaks['bf16_tflops'])
            ach8 = flops / (ms8 / 1e3) / 1e12
            fp8['roofline'] = {'bound': 'tensor', 'achieved': ach8, 'peak': peak8, 'unit': 'TFLOP/s',
                               'frac': ach8 / peak8, 'kernel': 'eloc_rows_kernel (e4m3)',
                               'peak_source': '%s bf16 dense (sustained) x 2, the nominal e4m3 / bf16 ratio' % peak_kind,
                               'flops': 'cone form, as the main line',
                               'dense_form': {'achieved': flops_dense / (ms8 / 1e3) / 1e12,
                                              'frac': flops_dense / (ms8 / 1e3) / 1e12 / peak8}}
        line = {
            'metric': METRIC, 'value': value, 'unit': 'samples/s', 'n_gpus': world, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': float(step_total_ms / args.steps), 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': args.precision, 'data': 'synthetic',
            'config': _config(w, args.workload),
            'sr_steps_per_s': sr_steps_per_s,
            'latency_ms': {'p50': float(np.percentile(step_ms, 50)), 'p99': float(np.percentile(step_ms, 99))},
            'stage_ms': {k: float(stage[:, i].mean()) for i, k in enumerate(['sample', 'eloc', 'grad', 'sr'])},
            'cg_iters': [int(i['iters']) for i in infos],
            'energy_per_site': float(e_last[:, 0].mean().item()) / N,
            'vs_plain_fp32': cmp,
            'energy_check': check,
            'roofline': roof,
            'roofline_sx': sx,
            'fp8': fp8,
            'cpu_baseline': {'value': sub.shape[0] / dt_or, 'unit': 'samples/s', 'cores': cores, 'kind': 'oracle',
                             'sample': '%d of the step\'s samples, E_loc only (FP64 numpy oracle, spawn pool)' %
                                       sub.shape[0]},
            'e2e': {'value': e2e_value, 'unit': 'samples/s', 'h2d_bytes_per_step': int(cfg_host.numel()),
                    'd2h_bytes_per_step': int(out_host.numel() * 8),
                    'what': 'nqs_local_energy on host configs: H2D copy + E_loc + D2H of E_loc per step'},
            'gpu_launches': int(launches),
            'clocks': clocks,
        }
        if not args.no_extra and world == 1:
            line['extra'] = extra_workloads(args, peaks, uuid, pool, cores)
        print(json.dumps(line), flush=True)
    ctx.close()
    if pool is not None:
        pool.close()
    if world > 1:
        dist.destroy_process_group()


def max_over_ranks(values, device=None):
    """Element-wise maximum over the ranks of the default process group
    (identity when there is none)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank, world, max_ms):
    """Units all ranks processed (each rank the same share) per second of the slowest rank."""
    return units_per_rank * world / (max_ms / 1000.0)


def params_at_step(ctx):
    return ctx.params.detach().cpu().numpy().copy()


if __name__ == '__main__':
    main()
