"""The sharded SR solve of the multi-GPU design, simulated with two gloo
ranks on the CPU: each rank holds half of the samples (rows of the local
derivatives and local energies); the sample means, the force and every CG
matrix-vector product are completed by one all-reduce of a P-vector (or of a
few scalars), and the dot products run on replicated P-vectors. The result
must equal the unsharded conjugate gradient of the oracle to 1e-12 (Sec. 3.2
SR; Sec. 5.4.1 distributed SR, here as matrix-free CG)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import sr


def _free_port():
    with socket.socket() as s:
        s.bind(('127.0.0.1', 0))
        return s.getsockname()[1]


def _inputs(ns=96, P=40, seed=7):
    rng = np.random.default_rng(seed)
    dA = rng.normal(size=(ns, P))
    dPhi = 0.5 * rng.normal(size=(ns, P))
    eloc = rng.normal(size=ns) + 0.1j * rng.normal(size=ns)
    return dA, dPhi, eloc


def _allreduce(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def sharded_cg(dA_loc, dPhi_loc, e_loc, n_total, eps, rtol, max_iter):
    """CG on (S + eps I) delta = F with the samples split across ranks."""
    # sample means: one all-reduce of [sum dA | sum dPhi | sum E]
    sums = _allreduce(np.concatenate([dA_loc.sum(0), dPhi_loc.sum(0), [e_loc.real.sum(), e_loc.imag.sum()]]))
    P = dA_loc.shape[1]
    mA, mPhi = sums[:P] / n_total, sums[P:2 * P] / n_total
    e_mean = complex(sums[2 * P], sums[2 * P + 1]) / n_total
    oc = np.concatenate([dA_loc - mA, dPhi_loc - mPhi], axis=0)          # local rows of Ohat
    de = e_loc - e_mean
    F = _allreduce(oc.T @ np.concatenate([de.real, de.imag])) / n_total

    def apply(p):   # (S + eps I) p: local rows, then one P-vector all-reduce
        return _allreduce(oc.T @ (oc @ p)) / n_total + eps * p

    x = np.zeros(P)
    r = F.copy()
    p = r.copy()
    rs = r @ r
    fnorm = np.sqrt(F @ F)
    it = 0
    while it < max_iter and np.sqrt(rs) > rtol * fnorm:
        Ap = apply(p)
        alpha = rs / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rs_new = r @ r
        p = r + (rs_new / rs) * p
        rs = rs_new
        it += 1
    return x, it, e_mean


def _worker(rank, world, port, q):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    dA, dPhi, eloc = _inputs()
    ns = dA.shape[0]
    rows = np.array_split(np.arange(ns), world)[rank]
    x, it, e_mean = sharded_cg(dA[rows], dPhi[rows], eloc[rows], ns, 1e-3, 1e-10, 500)
    q.put((rank, x, it, e_mean))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_cg_equals_unsharded_cg():
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    dA, dPhi, eloc = _inputs()
    x_ref, it_ref, _, e_ref = sr.cg(dA, dPhi, eloc, 1e-3, 1e-10, 500)
    for rank, x, it, e_mean in out:
        assert np.abs(x - x_ref).max() <= 1e-12 * np.abs(x_ref).max()
        assert abs(it - it_ref) <= 1
        assert abs(e_mean - e_ref) <= 1e-14
    # both ranks hold the same (replicated) delta
    assert np.array_equal(out[0][1], out[1][1])
    # and CG reaches the dense solve
    x_dense, _ = sr.solve_dense(dA, dPhi, eloc, 1e-3)
    assert np.abs(out[0][1] - x_dense).max() <= 1e-8 * np.abs(x_dense).max()


def _dying_worker(rank, world, port, q):
    """Rank 1 exits after the first collective (a dead rank); rank 0 must get
    an error from its next collective instead of waiting for ever."""
    import datetime
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    dA, dPhi, eloc = _inputs()
    ns = dA.shape[0]
    rows = np.array_split(np.arange(ns), world)[rank]
    _allreduce(dA[rows].sum(0))
    if rank == 1:
        os._exit(0)
    try:
        sharded_cg(dA[rows], dPhi[rows], eloc[rows], ns, 1e-3, 1e-10, 500)
        q.put((rank, 'finished'))
    except Exception as e:    # the failure is reported, the process stays usable
        q.put((rank, 'error:' + type(e).__name__))


def test_dead_rank_is_reported_not_waited_for():
    import time
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for p in procs:
        p.start()
    rank, status = q.get(timeout=120)
    assert rank == 0 and status.startswith('error:')
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert time.time() - t0 < 100
