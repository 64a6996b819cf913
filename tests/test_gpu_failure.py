"""Failure detection without a GPU fault: the device-side waits are bounded,
a wait that runs out sets the timeout bit that the host reads at the next
sync (NQS_ERR_TIMEOUT), and the context stays usable afterwards."""

import numpy as np
import pytest
import torch

from tests.gpu_common import WL, configs_for, dev, lib, make_ctx

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_recovers():
    nqs = lib()
    w = WL['j1j2_10x10']
    over = {'L': 6, 'n_up': 18, 'n_down': 18, 'n_layers': 3}
    ctx, _ = make_ctx(w, **over)
    cfg = dev(configs_for(w, 12, seed=41, **over))
    before = ctx.local_energy(cfg, None, 'bf16')
    ctx.sync()
    ctx.probe_wait_timeout(2000)
    with pytest.raises(nqs.NQSError) as err:
        ctx.sync()
    assert err.value.code == -6          # NQS_ERR_TIMEOUT
    assert 'wait' in str(err.value)
    ctx.sync()                           # the latched bit was cleared
    after = ctx.local_energy(cfg, None, 'bf16')
    ctx.sync()
    assert torch.equal(before, after)


def test_probe_rejects_bad_counts():
    nqs = lib()
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w, channels=16, n_layers=2)
    for bad in (0, -5, 10 ** 7):
        with pytest.raises(nqs.NQSError):
            ctx.probe_wait_timeout(bad)
    ctx.sync()


def test_bounds_probe_is_reported_and_cleared():
    """The reporting path of the device-side index checks: a failed check
    makes the next sync raise NQS_ERR_BOUNDS, and the context stays usable."""
    nqs = lib()
    w = WL['j1j2_4x4']
    ctx, _ = make_ctx(w)
    cfg = dev(configs_for(w, 4, seed=3))
    before = ctx.local_energy(cfg, None, 'fp64').clone()
    ctx.probe_bounds()
    with pytest.raises(nqs.NQSError) as ei:
        ctx.sync()
    assert ei.value.code == -8
    ctx.sync()
    assert torch.equal(ctx.local_energy(cfg, None, 'fp64'), before)
