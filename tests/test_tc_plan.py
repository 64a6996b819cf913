"""CPU checks of the host-side tensor-core plan choice (nqs_tc_plan): every
plan the launchers would use fits the SM's shared memory, tensor memory and
tile limits, the measured choices hold, and the tuning overrides are
respected. No GPU work is issued."""

import pytest

import nqs_synth

SM_BYTES = 233472          # shared memory per SM (228 KB), 1 KB reserved per block
MAX_SMEM = 232448          # opt-in limit per block
NUM_SMS = 152


@pytest.fixture(scope='module')
def nqs():
    from paper_2204_07816_gb300 import build, nqs as mod
    build.build()
    return mod


def _problem(nqs, w, **over):
    kw = dict(w)
    kw.update(over)
    if kw['model'] == 'j1j2':
        return nqs.make_problem('j1j2', kw['L'], n_layers=kw['n_layers'], channels=kw['channels'])
    N = kw['L'] ** 2
    nu = kw.get('n_up', (N - N // 8) // 2)
    nd = kw.get('n_down', nu)
    return nqs.make_problem('tj', kw['L'], n_up=nu, n_down=nd, n_layers=kw['n_layers'], channels=kw['channels'])


def _check_fits(plan, channels):
    assert plan['blocks_per_sm'] in (1, 2, 3)
    assert plan['epilogue_warps'] % 4 == 0 and plan['epilogue_warps'] >= 4
    assert 1 <= plan['tiles'] <= 16
    assert plan['blocks_per_sm'] * (plan['smem_bytes'] + 1024) <= SM_BYTES
    assert plan['smem_bytes'] <= MAX_SMEM
    cols = plan['tmem_cols']
    assert cols >= 32 and cols & (cols - 1) == 0
    assert cols >= plan['slots'] * plan['tiles'] * channels
    # co-resident blocks (as many as shared memory allows) never ask for more than 512 columns
    assert cols * (SM_BYTES // (plan['smem_bytes'] + 1024)) <= 512
    assert plan['grid'] >= 1


@pytest.mark.parametrize('name', [k for k, w in nqs_synth.WORKLOADS.items() if w['channels'] in (16, 32)])
@pytest.mark.parametrize('kind,n', [('logpsi', 8192), ('local_energy', 8192), ('sample', 256)])
def test_every_workload_has_a_plan_that_fits(nqs, name, kind, n):
    w = nqs_synth.WORKLOADS[name]
    plan = nqs.tc_plan(_problem(nqs, w), kind, n, MAX_SMEM, NUM_SMS)
    assert plan is not None
    _check_fits(plan, w['channels'])


@pytest.mark.parametrize('L', [4, 6, 8, 10, 12, 16, 20, 24, 36])
@pytest.mark.parametrize('channels', [16, 32])
def test_plans_fit_across_lattice_sizes(nqs, L, channels):
    prob = nqs.make_problem('j1j2', L, n_layers=6, channels=channels)
    for kind, n in (('logpsi', 4096), ('local_energy', 4096), ('sample', 256), ('sample', 4096)):
        plan = nqs.tc_plan(prob, kind, n, MAX_SMEM, NUM_SMS)
        if plan is None:
            assert channels == 32 and L >= 24     # too large for one block's shared memory
            continue
        _check_fits(plan, channels)
        if kind == 'sample':   # one chain per block, every chain has a block (chains beyond one wave run in later waves)
            assert (plan['G'], plan['slots'], plan['grid']) == (1, 1, n)


def test_measured_choices(nqs):
    # 10x10, 16 channels: the row form, two blocks per SM with twelve configurations each (120 of the 128
    # accumulator rows); the log psi plan keeps the tap form
    p10 = nqs.make_problem('j1j2', 10, n_layers=6, channels=16)
    e = nqs.tc_plan(p10, 'local_energy', 8192, MAX_SMEM, NUM_SMS)
    assert (e['G'], e['slots'], e['blocks_per_sm'], e['grid'], e['row_form']) == (12, 1, 2, 2 * NUM_SMS, 1)
    assert e['tmem_cols'] == 256 and e['tiles'] == 1
    lp = nqs.tc_plan(p10, 'logpsi', 8192, MAX_SMEM, NUM_SMS)
    assert (lp['blocks_per_sm'], lp['row_form']) == (2, 0)
    # the row form covers J1-J2 with 16 channels up to 13x13; larger lattices and 32 channels keep the tap form
    for L, want in ((4, 1), (7, 1), (13, 1), (14, 0), (16, 0)):
        pl = nqs.tc_plan(nqs.make_problem('j1j2', L, n_up=L * L // 2, n_down=L * L - L * L // 2, n_layers=6,
                                          channels=16), 'local_energy', 4096, MAX_SMEM, NUM_SMS)
        assert pl['row_form'] == want, L
        assert pl['G'] == (min(16, 128 // L) if want else pl['G'])
    # sampler: one chain per block, three co-resident blocks where they fit; every chain has its block
    for n in (256, 4096):
        s = nqs.tc_plan(p10, 'sample', n, MAX_SMEM, NUM_SMS)
        assert (s['G'], s['slots'], s['blocks_per_sm'], s['grid'], s['epilogue_warps']) == (1, 1, 3, n, 4)
    p16c32 = nqs.make_problem('j1j2', 16, n_layers=8, channels=32)
    assert nqs.tc_plan(p16c32, 'sample', 256, MAX_SMEM, NUM_SMS)['blocks_per_sm'] == 2
    # t-J 12x12, 16 channels: two blocks of three configurations
    ptj = nqs.make_problem('tj', 12, n_up=63, n_down=63, n_layers=6, channels=16)
    t = nqs.tc_plan(ptj, 'local_energy', 8192, MAX_SMEM, NUM_SMS)
    assert (t['G'], t['blocks_per_sm']) == (3, 2)
    # 16x16, 16 channels: groups of at most 2 fit two blocks, so one block per SM
    p16 = nqs.make_problem('j1j2', 16, n_layers=8, channels=16)
    assert nqs.tc_plan(p16, 'local_energy', 8192, MAX_SMEM, NUM_SMS)['blocks_per_sm'] == 1
    # 32 channels: one block per SM for the local energy
    p32 = nqs.make_problem('j1j2', 10, n_layers=6, channels=32)
    assert nqs.tc_plan(p32, 'local_energy', 8192, MAX_SMEM, NUM_SMS)['blocks_per_sm'] == 1
    # a lattice too large for two sampler blocks falls back to one
    p36 = nqs.make_problem('j1j2', 36, n_layers=6, channels=16)
    assert nqs.tc_plan(p36, 'sample', 256, MAX_SMEM, NUM_SMS)['blocks_per_sm'] == 1


def test_overrides(nqs, monkeypatch):
    p10 = nqs.make_problem('j1j2', 10, n_layers=6, channels=16)
    monkeypatch.setenv('NQS_TC_ROWS', '0')               # the tap form for the local energy
    assert nqs.tc_plan(p10, 'local_energy', 8192, MAX_SMEM, NUM_SMS)['row_form'] == 0
    monkeypatch.setenv('NQS_TC_PLAN', '16,1,1')
    e = nqs.tc_plan(p10, 'local_energy', 8192, MAX_SMEM, NUM_SMS)
    assert (e['G'], e['slots'], e['blocks_per_sm']) == (16, 1, 1)
    monkeypatch.setenv('NQS_TC_PLAN', '40,1,1')          # infeasible: ignored
    assert nqs.tc_plan(p10, 'local_energy', 8192, MAX_SMEM, NUM_SMS)['G'] == 8
    monkeypatch.delenv('NQS_TC_PLAN')
    monkeypatch.delenv('NQS_TC_ROWS')
    monkeypatch.setenv('NQS_TC_SAMPLE', '2,1,1')
    s = nqs.tc_plan(p10, 'sample', 256, MAX_SMEM, NUM_SMS)
    assert (s['G'], s['blocks_per_sm'], s['grid']) == (2, 1, 128)


def test_unsupported_and_invalid(nqs):
    assert nqs.tc_plan(nqs.make_problem('j1j2', 4, n_layers=2, channels=4), 'local_energy', 8) is None
    bad = nqs.make_problem('j1j2', 4, n_up=3, n_down=3, n_layers=2, channels=16)   # n_up + n_down != N
    with pytest.raises(nqs.NQSError):
        nqs.tc_plan(bad, 'local_energy', 8)
    with pytest.raises(nqs.NQSError):
        nqs.tc_plan(nqs.make_problem('j1j2', 4, n_layers=2, channels=16), 'local_energy', 0)
