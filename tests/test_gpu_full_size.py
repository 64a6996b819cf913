"""Local energies at the full workload sizes, in the launch configuration the
benchmark uses (one bf16 launch over the whole batch): sampled rows against
the oracle one by one, and the batch energy against the FP64 GPU path."""

import numpy as np
import pytest
import torch

from oracle import eloc
from tests.gpu_common import WL, configs_for, dev, make_ctx, oracle_of

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('name,n,rows,fp64_rows', [('j1j2_10x10', 8192, 16, 8192), ('tj_12x12', 8192, 8, 1024),
                                                    ('j1j2_16x16', 16384, 2, 64)])
def test_local_energy_bf16_full_batch(name, n, rows, fp64_rows):
    w = WL[name]
    N = w['L'] ** 2
    ctx, params = make_ctx(w, param_seed=91)
    spec, ham = oracle_of(w)
    cfg = dev(configs_for(w, n, seed=92))
    e = ctx.local_energy(cfg, None, 'bf16')
    e_h = e.cpu().numpy()
    assert np.all(np.isfinite(e_h))
    # sampled rows, spread over the batch (first, last and in between), against the oracle
    pick = np.unique(np.linspace(0, n - 1, rows).astype(int))
    want = eloc.local_energy(params, cfg[pick].cpu().numpy(), spec, ham)
    assert np.abs(e_h[pick, 0] - want.real).max() / N <= 2e-4
    assert np.abs(e_h[pick, 1] - want.imag).max() / N <= 2e-4
    # batch energy per site against the FP64 GPU path (whole batch where it is affordable)
    e64 = ctx.local_energy(cfg[:fp64_rows], None, 'fp64').cpu().numpy()
    assert abs(e_h[:fp64_rows, 0].mean() - e64[:, 0].mean()) / N <= 1e-5
    # the same batch split in two launches gives bitwise the same rows
    half = n // 2
    e2 = torch.cat([ctx.local_energy(cfg[:half], None, 'bf16'), ctx.local_energy(cfg[half:], None, 'bf16')])
    assert torch.equal(e2, e)


def test_local_energy_fp8_full_batch():
    """The FP8 form at the 10x10 workload size in one launch over the whole
    batch: sampled rows against the oracle (per-sample bound of the e4m3
    form, 5e-3 per site), the batch energy per site against the FP64 GPU path
    within the 1e-4 validity condition, and bitwise-equal rows when the batch
    is split in two launches."""
    w = WL['j1j2_10x10']
    N = w['L'] ** 2
    n = 8192
    ctx, params = make_ctx(w, param_seed=91)
    spec, ham = oracle_of(w)
    cfg = dev(configs_for(w, n, seed=93))
    e = ctx.local_energy(cfg, None, 'fp8')
    e_h = e.cpu().numpy()
    assert np.all(np.isfinite(e_h))
    pick = np.unique(np.linspace(0, n - 1, 8).astype(int))
    want = eloc.local_energy(params, cfg[pick].cpu().numpy(), spec, ham)
    assert np.abs(e_h[pick, 0] - want.real).max() / N <= 5e-3
    e64 = ctx.local_energy(cfg, None, 'fp64').cpu().numpy()
    assert abs(e_h[:, 0].mean() - e64[:, 0].mean()) / N <= 1e-4
    half = n // 2
    e2 = torch.cat([ctx.local_energy(cfg[:half], None, 'fp8'), ctx.local_energy(cfg[half:], None, 'fp8')])
    assert torch.equal(e2, e)
