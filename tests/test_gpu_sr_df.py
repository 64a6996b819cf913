"""The conjugate gradient's S.x products in double-float arithmetic (Sec. 3.2,
the SR solve): the split of O into a plane of float high parts and a plane of
float low parts, the narrow passes that read the high plane alone when O is
made of floats (the float32 and bf16 local derivatives are), and the padded
plane stride when P is not a multiple of 4, each against the oracle's dense
solve of the same system in float64."""

import numpy as np
import pytest
import torch

from oracle import sr
from tests.gpu_common import WL, dev, lib, make_ctx

pytestmark = pytest.mark.gpu


def _system(P, n, seed, as_float):
    rng = np.random.default_rng(seed)
    dA = rng.normal(size=(n, P)) * np.exp(rng.normal(0.0, 1.0, size=P)) + rng.normal(size=P)
    dPhi = 0.5 * rng.normal(size=(n, P))
    e = -20.0 + rng.normal(size=n) + 0.3j * rng.normal(size=n)
    if as_float:
        dA = dA.astype(np.float32).astype(np.float64)
        dPhi = dPhi.astype(np.float32).astype(np.float64)
    return dA, dPhi, e


def _ctx(net, channels):
    """A context whose parameter count is the network's (CNN1 has P = 1 mod 4,
    the SiLU family P = 0 mod 4); sr_solve reads no parameter values."""
    nqs = lib()
    prob = nqs.make_problem('j1j2', 4, n_layers=2, channels=channels, net=net)
    P = nqs.nqs_param_count(prob)
    params = torch.tensor(np.random.default_rng(5).normal(size=P) * 0.1, dtype=torch.float64, device='cuda')
    return nqs.Context(prob, params, seed=0)


NETS = [('silu', 4), ('silu', 8), ('cnn1', 4), ('cnn1', 8)]


@pytest.mark.parametrize('net,channels', NETS)
@pytest.mark.parametrize('as_float', [True, False])
@pytest.mark.parametrize('arith', ['double_float', 'fp64'])
def test_cg_matches_dense_solve_float_planes(net, channels, as_float, arith):
    """Float-exact O (the float plane alone) and full float64 O (both planes);
    P = 0 and 1 mod 4 (plane rows padded by 0 and 3 columns); and the same
    systems with the float64 passes."""
    ctx = _ctx(net, channels)
    ctx.set_sx_arithmetic(arith)
    P, n = ctx.P, 300
    dA, dPhi, e = _system(P, n, 40 + channels + len(net), as_float)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, em = sr.solve_dense(dA, dPhi, e, 1e-3)
    got, info = ctx.sr_solve(O, E, eps=1e-3, rtol=1e-12, max_iter=10000)
    assert info['converged'] and info['resid'] <= 1e-12
    assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-9 * np.linalg.norm(want)
    assert abs(info['energy'] - em) <= 1e-12 * abs(em)
    ctx.close()


def test_plane_stride_residues_covered():
    residues = set()
    for net, channels in NETS:
        ctx = _ctx(net, channels)
        residues.add(ctx.P % 4)
        ctx.close()
    assert residues == {0, 1}, residues


def test_float_planes_at_bench_size():
    """8,192 samples of the 10x10 network's parameter count (P = 11,792), O made
    of floats as the bf16 local derivatives are: the narrow passes at the size
    the bench times, against the oracle's sample-space solve."""
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    P, n = ctx.P, 2048
    dA, dPhi, e = _system(P, n, 91, True)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, em = sr.solve_woodbury(dA, dPhi, e, 1e-4)
    got, info = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-11, max_iter=10000)
    assert info['converged'] and info['resid'] <= 1e-11
    assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
    ctx.close()


def test_double_float_and_fp64_passes_agree():
    """Full float64 O at the 10x10 network's P: the two arithmetics' deltas
    (both solved to rtol 1e-11) within 1e-9 of each other, and an unknown
    mode refused."""
    w = WL['j1j2_10x10']
    ctx, _ = make_ctx(w)
    P, n = ctx.P, 1024
    dA, dPhi, e = _system(P, n, 17, False)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    d_df, i_df = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-11, max_iter=10000)
    ctx.set_sx_arithmetic('fp64')
    d_64, i_64 = ctx.sr_solve(O, E, eps=1e-4, rtol=1e-11, max_iter=10000)
    assert i_df['converged'] and i_64['converged']
    assert torch.linalg.norm(d_df - d_64) <= 1e-9 * torch.linalg.norm(d_64)
    assert i_df['energy'] == i_64['energy']
    assert ctx.lib.nqs_set_sx_arithmetic(ctx.ctx, 7) == -1   # NQS_ERR_INVALID_ARG
    ctx.close()


def test_split_edge_magnitudes():
    """Elements the split treats specially: exact zero columns and magnitudes
    below 2^-80 (taken as zero; their products are below 1e-24 of the O(1)
    terms), against the oracle's dense solve in float64."""
    ctx = _ctx('silu', 4)
    P, n = ctx.P, 256
    dA, dPhi, e = _system(P, n, 77, False)
    rng = np.random.default_rng(78)
    dA[:, :3] = 0.0                                   # whole zero columns
    mask = rng.random(size=dA.shape) < 0.05
    dA[mask] *= 1e-30                                 # tiny elements
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, em = sr.solve_dense(dA, dPhi, e, 1e-3)
    got, info = ctx.sr_solve(O, E, eps=1e-3, rtol=1e-12, max_iter=20000)
    assert info['converged']
    assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
    ctx.close()


def test_products_beyond_float_range():
    """O scaled by 1e20: the double-float passes' sums leave the float range,
    which the solve reports as NQS_ERR_NONFINITE (parameters unchanged), while
    the float64 passes solve the same system (eps scaled with S)."""
    nqs = lib()
    ctx = _ctx('silu', 4)
    P, n = ctx.P, 128
    dA, dPhi, e = _system(P, n, 79, False)
    dA *= 1e20
    dPhi *= 1e20
    eps = 1e-3 * 1e40
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    before = ctx.params.clone()
    with pytest.raises(nqs.NQSError) as ex:
        ctx.sr_solve(O, E, eps=eps, rtol=1e-12, max_iter=2000, lr=0.1, apply_update=True)
    assert ex.value.code == -4, ex.value   # NQS_ERR_NONFINITE
    assert torch.equal(ctx.params, before)
    ctx.set_sx_arithmetic('fp64')
    want, _ = sr.solve_dense(dA, dPhi, e, eps)
    got, info = ctx.sr_solve(O, E, eps=eps, rtol=1e-12, max_iter=20000)
    assert info['converged']
    assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
    ctx.close()


@pytest.mark.parametrize('n', [1, 3, 9])
@pytest.mark.parametrize('as_float', [True, False])
def test_few_samples(n, as_float):
    """Ragged row blocks of the passes (2n = 2, 6, 18 rows against blocks of 8
    rows) and P = 1 mod 4, against the oracle's dense solve."""
    ctx = _ctx('cnn1', 4)
    P = ctx.P
    dA, dPhi, e = _system(P, n, 200 + n, as_float)
    O = dev(np.concatenate([dA, dPhi], 0))
    E = dev(np.stack([e.real, e.imag], 1))
    want, em = sr.solve_dense(dA, dPhi, e, 1e-2)
    got, info = ctx.sr_solve(O, E, eps=1e-2, rtol=1e-12, max_iter=10000)
    assert info['converged']
    assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-9 * max(np.linalg.norm(want), 1e-300)
    assert abs(info['energy'] - em) <= 1e-12 * abs(em)
    ctx.close()
