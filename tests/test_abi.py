"""CPU checks of the C ABI library: it builds, loads, exports every entry
point include/nqs.h declares, and agrees with the oracle on the parameter
count. No GPU work is issued."""

import ctypes
import os
import re

import pytest

import nqs_synth
from oracle import cnn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def nqs():
    from paper_2204_07816_gb300 import build, nqs as mod
    build.build()
    return mod


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, 'include')):
        if h.endswith('.h'):
            text = open(os.path.join(ROOT, 'include', h)).read()
            text = re.sub(r'/\*.*?\*/', '', text, flags=re.S)
            names |= set(re.findall(r'\b(nqs_[a-z0-9_]+)\s*\(', text))
    return names


def test_every_declared_symbol_is_exported(nqs):
    lib = ctypes.CDLL(nqs.LIB_PATH)
    declared = _declared()
    assert declared, 'no declarations found'
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(nqs.EXPORTS) | (declared - set(nqs.EXPORTS))
    for name in nqs.EXPORTS:
        assert name in declared, name


@pytest.mark.parametrize('name', list(nqs_synth.WORKLOADS))
def test_param_count_matches_oracle(nqs, name):
    w = nqs_synth.WORKLOADS[name]
    if w['model'] == 'j1j2':
        p = nqs.make_problem('j1j2', w['L'], n_layers=w['n_layers'], channels=w['channels'])
    else:
        p = nqs.make_problem('tj', w['L'], n_up=w['n_up'], n_down=w['n_down'], n_layers=w['n_layers'],
                             channels=w['channels'])
    assert nqs.nqs_param_count(p) == cnn.param_count(cnn.NetSpec(w['L'], w['c_in'], w['channels'], w['n_layers']))


@pytest.mark.parametrize('bad', [dict(L=3), dict(L=40), dict(channels=12), dict(n_layers=0),
                                 dict(n_up=7, n_down=8), dict(model=5), dict(sign_rule=2)])
def test_invalid_problems_rejected(nqs, bad):
    kw = dict(model='j1j2', L=4, n_layers=2, channels=4)
    kw.update(bad)
    p = nqs.make_problem(**{k: v for k, v in kw.items() if k not in ('sign_rule',)})
    if 'sign_rule' in bad:
        p.sign_rule = bad['sign_rule']
    assert nqs.nqs_param_count(p) == -1


def test_null_problem_rejected(nqs):
    assert nqs.load().nqs_param_count(None) == -1


def test_binding_rejects_host_and_misshaped_tensors(nqs):
    """Argument marshalling fails before any device work: parameters must be
    a float64 CUDA tensor of the problem's length (checked on the host)."""
    import torch
    prob = nqs.make_problem('j1j2', 4, n_layers=2, channels=4)
    P = nqs.nqs_param_count(prob)
    with pytest.raises(ValueError):
        nqs.Context(prob, torch.zeros(P + 1, dtype=torch.float64))
    with pytest.raises(TypeError):
        nqs.Context(prob, torch.zeros(P, dtype=torch.float64))          # a host tensor
    with pytest.raises(TypeError):
        nqs._ptr(torch.zeros(3, dtype=torch.float32), torch.float64, 'x')


def test_status_names_cover_the_header(nqs):
    """Every status code the header declares has a name in the binding."""
    header = open(os.path.join(ROOT, 'include', 'nqs.h')).read()
    codes = {int(v) for v in re.findall(r'NQS_(?:OK|ERR_[A-Z_]+) = (-?\d+)', header)}
    assert codes <= set(nqs.STATUS)


def test_checked_build_exports_the_same_entry_points(nqs):
    """The checked variant (device-side index checks, NQS_ERR_BOUNDS) builds
    from the same sources and exports every declared entry point."""
    from paper_2204_07816_gb300 import build
    path = build.build(checked=True)
    assert os.path.basename(path) != os.path.basename(nqs.LIB_PATH)
    lib = ctypes.CDLL(path)
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_param_count_of_the_paper_families_matches_the_oracle():
    from oracle import cnn_paper
    from paper_2204_07816_gb300 import build, nqs
    build.build()
    for kind in ('cnn1', 'cnn2'):
        for model, c_in in (('j1j2', 1), ('tj', 3)):
            for L, C, B in ((4, 4, 2), (10, 16, 6), (12, 32, 6)):
                N = L * L
                prob = (nqs.make_problem('j1j2', L, n_layers=B, channels=C, net=kind) if model == 'j1j2' else
                        nqs.make_problem('tj', L, n_up=N // 2 - 1, n_down=N // 2 - 1, n_layers=B, channels=C, net=kind))
                assert nqs.nqs_param_count(prob) == cnn_paper.param_count(cnn_paper.PaperSpec(kind, L, c_in, C, B))
    assert nqs.nqs_param_count(nqs.make_problem('j1j2', 5, n_up=13, n_down=12, net='cnn1')) == -1   # odd N
    assert nqs.nqs_param_count(nqs.make_problem('j1j2', 4, net=7)) == -1
