"""Convolutional log-amplitude network, FP64, forward and analytic backward.

The wave function of Eq. (1) is |Psi> = sum_S W(S)|S> with W(S) given by a
network. Here W(S) = exp(a(S) + i phi(S)), so the network returns the pair
(a, phi) = (log|W|, arg W). The network is the translation-invariant
convolutional family of Sec. 5.2 ("Neural network innovations": convolutions
with periodic padding, Sec. 5.4.2 "PBC padding"), in the form fixed for this
build:

    input  J1-J2: one channel, the site value sigma = +-1
           t-J:   three one-hot channels in the order (hole, up, down)
    n_layers times:  z = conv3x3_periodic(h) + bias;  h = silu(z) = z / (1 + e^-z)
    head   hbar_c = sum over sites of h_c;  a = w_a . hbar;  phi = w_phi . hbar

The convolution is a cross-correlation with circular padding:
    z[o, y, x] = b[o] + sum_{c, dy, dx in -1..1} W[o, c, dy+1, dx+1] * h[c, (y+dy) mod L, (x+dx) mod L]

Flat parameter layout (float64): for each layer W[C_out][C_in][3][3] then
b[C_out]; then w_a[C] and w_phi[C]. The head has no bias.
"""

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class NetSpec:
    L: int
    c_in: int        # 1 for J1-J2, 3 for t-J
    channels: int
    n_layers: int


def layer_dims(spec):
    return [(spec.c_in if l == 0 else spec.channels, spec.channels) for l in range(spec.n_layers)]


def param_count(spec):
    if _paper(spec):
        return _paper(spec).param_count(spec)
    return sum(9 * ci * co + co for ci, co in layer_dims(spec)) + 2 * spec.channels


def unpack(params, spec):
    params = np.asarray(params, dtype=np.float64)
    assert params.shape == (param_count(spec),)
    layers, off = [], 0
    for ci, co in layer_dims(spec):
        W = params[off:off + 9 * ci * co].reshape(co, ci, 3, 3)
        off += 9 * ci * co
        b = params[off:off + co]
        off += co
        layers.append((W, b))
    C = spec.channels
    w_a = params[off:off + C]
    w_phi = params[off + C:off + 2 * C]
    return layers, w_a, w_phi


def encode(configs, spec):
    """[B, N] site values -> [B, c_in, L, L] network input."""
    c = np.asarray(configs, dtype=np.int64).reshape(-1, spec.L, spec.L)
    if spec.c_in == 1:
        return c[:, None, :, :].astype(np.float64)
    return np.stack([c == 0, c == 1, c == -1], axis=1).astype(np.float64)


def shifted(h, dy, dx):
    """h'[..., y, x] = h[..., (y+dy) mod L, (x+dx) mod L]."""
    return np.roll(h, shift=(-dy, -dx), axis=(-2, -1))


def conv(h, W, b):
    out = np.broadcast_to(b[None, :, None, None], (h.shape[0], W.shape[0]) + h.shape[2:]).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out += np.einsum('oc,bcyx->boyx', W[:, :, dy + 1, dx + 1], shifted(h, dy, dx))
    return out


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def _paper(spec):
    """The paper's CNN1 / CNN2 families live in cnn_paper (spec.kind)."""
    if getattr(spec, 'kind', None) in ('cnn1', 'cnn2'):
        from . import cnn_paper
        return cnn_paper
    return None


def forward(params, configs, spec, return_cache=False):
    if _paper(spec):
        return _paper(spec).forward(params, configs, spec, return_cache)
    layers, w_a, w_phi = unpack(params, spec)
    h = encode(configs, spec)
    cache = [h]
    zs = []
    for W, b in layers:
        z = conv(h, W, b)
        h = silu(z)
        zs.append(z)
        cache.append(h)
    hbar = h.sum(axis=(2, 3))
    a = hbar @ w_a
    phi = hbar @ w_phi
    if return_cache:
        return a, phi, (cache, zs, hbar)
    return a, phi


def _backprop(layers, cache, zs, g):
    """Gradient of sum_sites sum_c g[c]*h_n wrt every conv parameter, per sample."""
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        gz = g * silu_grad(zs[l])
        hin = cache[l]
        dW = np.zeros((gz.shape[0],) + W.shape)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                dW[:, :, :, dy + 1, dx + 1] = np.einsum('boyx,bcyx->boc', gz, shifted(hin, dy, dx))
        db = gz.sum(axis=(2, 3))
        grads.append((dW.reshape(gz.shape[0], -1), db))
        if l > 0:
            g = np.zeros_like(hin)
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    # z[y] uses h[y+d]; so dL/dh[y'] collects gz[y' - d]
                    g += np.einsum('oc,boyx->bcyx', W[:, :, dy + 1, dx + 1], shifted(gz, -dy, -dx))
    grads.reverse()
    return np.concatenate([np.concatenate([dW, db], axis=1) for dW, db in grads], axis=1)


def backward(params, configs, spec):
    """Per-sample log-derivatives.

    Returns (a, phi, dA, dPhi) with dA[b, k] = d a(S_b) / d theta_k and
    dPhi[b, k] = d phi(S_b) / d theta_k, so that the complex local derivative
    of the paper (O_loc, Sec. 3.2) is O_k = dA + i dPhi.
    """
    if _paper(spec):
        return _paper(spec).backward(params, configs, spec)
    layers, w_a, w_phi = unpack(params, spec)
    a, phi, (cache, zs, hbar) = forward(params, configs, spec, return_cache=True)
    B, C = hbar.shape
    hn = cache[-1]
    ones = np.ones_like(hn)
    conv_a = _backprop(layers, cache, zs, ones * w_a[None, :, None, None])
    conv_phi = _backprop(layers, cache, zs, ones * w_phi[None, :, None, None])
    zero = np.zeros((B, C))
    dA = np.concatenate([conv_a, hbar, zero], axis=1)
    dPhi = np.concatenate([conv_phi, zero, hbar], axis=1)
    return a, phi, dA, dPhi
