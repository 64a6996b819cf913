"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU: its JSON line carries the contract's keys, the same workload
config as the GPU arm, and only rank 0 prints."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, 'bench.py', '--impl', 'reference', '--steps', '2', '--warmup', '1',
                        '--oracle-samples', '4'], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return [l for l in r.stdout.splitlines() if l.startswith('{')]


def test_reference_line():
    lines = _run({'RANK': '0'})
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ('metric', 'value', 'unit', 'n_gpus', 'steps', 'warmup', 'ms_per_step', 'higher_is_better',
                'scaling', 'vs_baseline', 'dtype', 'data', 'config', 'cpu_baseline', 'e2e'):
        assert key in line, key
    assert line['impl'] == 'reference' and line['steps'] == 2 and line['warmup'] == 1
    assert line['value'] > 0 and line['higher_is_better'] is True and line['unit'] == 'samples/s'
    cb = line['cpu_baseline']
    assert cb['kind'] == 'oracle' and cb['value'] == line['value'] and cb['cores'] >= 1 and cb['sample']
    assert line['e2e'] == {'value': line['value'], 'unit': line['unit'], 'h2d_bytes_per_step': 0,
                           'd2h_bytes_per_step': 0}
    sys.path.insert(0, ROOT)
    import bench
    import nqs_synth
    assert line['config'] == bench._config(nqs_synth.WORKLOADS['j1j2_10x10'], 'j1j2_10x10')
    assert line['metric'] == bench.METRIC


def test_other_ranks_print_nothing():
    assert _run({'RANK': '1'}) == []
