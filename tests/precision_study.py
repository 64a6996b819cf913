"""Effect of the convolution operand format on log psi and on the energy per
site (the validity condition of the reduced-precision forms: within 1e-4 of
FP64 on the same samples), computed with the oracle's network and local
energy with every convolution's operands rounded first:

  bf16: weights and activations rounded to bfloat16 (8-bit mantissa);
  fp8:  e4m3 (4-bit mantissa, largest finite 448) with per-channel scales:
        each output channel's weights divided by max|W| / 448, each input
        channel's activations by its largest magnitude over the batch / 448.

Accumulation stays FP64, so this isolates the operand rounding.

    python -m tests.precision_study [samples]
"""

import sys

import numpy as np

import nqs_synth
from oracle import cnn, eloc, hamiltonian


def round_mantissa(x, bits, emin):
    """Round to nearest with `bits` explicit mantissa bits; exponents below
    emin are subnormal (fixed quantum 2^(emin - bits))."""
    x = np.asarray(x, dtype=np.float64)
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-300)))
    q = 2.0 ** (np.maximum(e, emin) - bits)
    return np.round(x / q) * q


def bf16(x):
    return round_mantissa(x, 7, -126)


def e4m3(x):
    return np.clip(round_mantissa(x, 3, -6), -448.0, 448.0)


def _conv_rounded(fmt, conv):
    def f(h, W, b):
        if fmt == 'bf16':
            return conv(bf16(h), bf16(W), b)
        sw = np.abs(W).reshape(W.shape[0], -1).max(1) / 448.0
        sw = np.where(sw > 0, sw, 1.0)[:, None, None, None]
        sh = np.abs(h).max(axis=(0, 2, 3)) / 448.0
        sh = np.where(sh > 0, sh, 1.0)[None, :, None, None]
        return conv(e4m3(h / sh) * sh, e4m3(W / sw) * sw, b)
    return f


def study(wname, n_samples, seed=3):
    w = nqs_synth.WORKLOADS[wname]
    spec = cnn.NetSpec(w['L'], w['c_in'], w['channels'], w['n_layers'])
    ham = (hamiltonian.J1J2(w['L'], w['J1'], w['J2']) if w['model'] == 'j1j2'
           else hamiltonian.TJ(w['L'], w['t'], w['J']))
    params = nqs_synth.random_params(w['c_in'], w['channels'], w['n_layers'], seed=1)
    N = w['L'] ** 2
    cfg = nqs_synth.random_configs(N, w['n_up'], w['n_down'], n_samples, seed=seed)
    plain = cnn.conv
    out = {}
    try:
        for fmt in (None, 'bf16', 'fp8'):
            cnn.conv = plain if fmt is None else _conv_rounded(fmt, plain)
            a, _ = cnn.forward(params, cfg, spec)
            e = eloc.local_energy_batch(params, cfg, spec, ham)
            out[fmt] = (a, e)
    finally:
        cnn.conv = plain
    a0, e0 = out[None]
    rows = []
    for fmt in ('bf16', 'fp8'):
        a, e = out[fmt]
        rows.append((wname, fmt, np.abs(a - a0).max(), abs(e.real.mean() - e0.real.mean()) / N,
                     np.abs(e.real - e0.real).max() / N))
    return rows


def main(argv):
    n = int(argv[0]) if argv else 8
    print('| workload | operands | max abs d log psi | energy/site diff | max per-sample E_loc/site diff |')
    print('|---|---|---|---|---|')
    for wname in ('j1j2_10x10', 'tj_12x12', 'j1j2_16x16'):
        for r in study(wname, n):
            print('| %s | %s | %.2e | %.2e | %.2e |' % r, flush=True)


if __name__ == '__main__':
    main(sys.argv[1:])
