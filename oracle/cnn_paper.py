"""The paper's two network families (Sec. 5.2, "Neural network innovations"),
FP64, forward and analytic backward. Test infrastructure (see the package
docstring).

The paper describes them in words only (its figure is not available):

* CNN1 (spin models): a building block of a two-dimensional convolution, a
  one-dimensional max-pooling and a transposed convolution, stacked; periodic
  (PBC) padding on the lattice and between blocks; the wave-function
  coefficient is the product of the neurons of the last layer. Non-linearity
  comes from the max-pooling only.
* CNN2 (fermion models): CNN1 with an embedding layer on the input and a
  one-dimensional max-pooling of stride one, padded by copying the first
  neurons to the end; a final convolution reduces the channels to one and the
  coefficient is the product of its neurons.

Reading taken here (the paper gives no sizes; the operator table of
Sec. 5.4.2 shows activations as [batch, sites, channels] with a 10 x 10
lattice padded to 12 x 12, so the one-dimensional operators run over the
row-major site order s = y L + x):

    encode   CNN1: the input channels of the SiLU family (sigma = +-1, or the
             one-hot (hole, up, down) of t-J);
             CNN2: X[c, s] = E[v(s), c], v = 0/1 for down/up (J1-J2) and
             0/1/2 for hole/up/down (t-J)
    block b  U = conv3x3_periodic(X) + beta_b           (cross-correlation)
             CNN1: V[c, j] = max(U[c, 2j], U[c, 2j+1]),  j < N/2   (window 2, stride 2)
                   Y[o, 2j + t] = gamma_b[o] + sum_c T_b[c, o, t] V[c, j]   (transposed conv, kernel 2, stride 2)
             CNN2: V[c, s] = max(U[c, s], U[c, (s+1) mod N])          (window 2, stride 1, first neuron copied to the end)
                   Y[o, s] = gamma_b[o] + sum_c (T_b[c, o, 0] V[c, s] + T_b[c, o, 1] V[c, (s-1) mod N])
                                                                (transposed conv, kernel 2, stride 1, periodic)
    output   CNN1: the last block's transposed convolution has one output channel;
             CNN2: Z = conv3x3_periodic(Y_last) + beta_f with one output channel;
             W(S) = prod over sites of that channel, so
             a = sum_s log|z_s|,  phi = pi (number of negative z_s mod 2)

CNN1 needs an even number of sites. Max-pooling ties (equal values) route
the gradient to the first element of the window.

Flat parameter layout (float64), blocks b = 0 .. n_blocks-1:
    CNN1: per block W_b[C][C_b][3][3], beta_b[C], T_b[C][C_o][2], gamma_b[C_o]
          (C_b = c_in for b = 0 else C; C_o = 1 for the last block else C)
    CNN2: E[n_states][C]; per block W_b[C][C][3][3], beta_b[C], T_b[C][C][2],
          gamma_b[C]; then W_f[1][C][3][3], beta_f[1]

The local derivatives are real (phi is piecewise constant):
    d a / d theta = sum_s (1 / z_s) d z_s / d theta,   d phi / d theta = 0.
"""

from dataclasses import dataclass

import numpy as np

from .cnn import conv, shifted


@dataclass(frozen=True)
class PaperSpec:
    kind: str        # 'cnn1' or 'cnn2'
    L: int
    c_in: int        # 1 for J1-J2, 3 for t-J (CNN1 input channels; CNN2: 2 or 3 embedding rows)
    channels: int
    n_layers: int    # building blocks


def n_states(spec):
    return 2 if spec.c_in == 1 else 3


def param_count(spec):
    C, B = spec.channels, spec.n_layers
    if spec.kind == 'cnn1':
        total = 0
        for b in range(B):
            cb = spec.c_in if b == 0 else C
            co = 1 if b == B - 1 else C
            total += 9 * C * cb + C + 2 * C * co + co
        return total
    return n_states(spec) * C + B * (9 * C * C + C + 2 * C * C + C) + 9 * C + 1


def unpack(params, spec):
    """(embedding or None, [(W, beta, T, gamma)] per block, (W_f, beta_f) or None)."""
    params = np.asarray(params, dtype=np.float64)
    assert params.shape == (param_count(spec),)
    C, B = spec.channels, spec.n_layers
    off = 0

    def take(n, shape):
        nonlocal off
        out = params[off:off + n].reshape(shape)
        off += n
        return out

    emb = take(n_states(spec) * C, (n_states(spec), C)) if spec.kind == 'cnn2' else None
    blocks = []
    for b in range(B):
        cb = (spec.c_in if b == 0 else C) if spec.kind == 'cnn1' else C
        co = (1 if b == B - 1 else C) if spec.kind == 'cnn1' else C
        W = take(9 * C * cb, (C, cb, 3, 3))
        beta = take(C, (C,))
        T = take(2 * C * co, (C, co, 2))
        gamma = take(co, (co,))
        blocks.append((W, beta, T, gamma))
    final = (take(9 * C, (1, C, 3, 3)), take(1, (1,))) if spec.kind == 'cnn2' else None
    assert off == params.size
    return emb, blocks, final


def state_index(configs, spec):
    c = np.asarray(configs, dtype=np.int64)
    if spec.c_in == 1:
        return (c > 0).astype(np.int64)                         # down 0, up 1
    return np.where(c == 0, 0, np.where(c == 1, 1, 2))           # hole 0, up 1, down 2


def encode(configs, spec, emb):
    """[B, N] site values -> [B, channels, L, L] network input."""
    B = np.asarray(configs).shape[0]
    L = spec.L
    if spec.kind == 'cnn2':
        v = state_index(configs, spec)                           # [B, N]
        return emb[v].transpose(0, 2, 1).reshape(B, spec.channels, L, L)
    c = np.asarray(configs, dtype=np.int64).reshape(B, L, L)
    if spec.c_in == 1:
        return c[:, None, :, :].astype(np.float64)
    return np.stack([c == 0, c == 1, c == -1], axis=1).astype(np.float64)


# ---------------------------------------------------------------- one-dimensional operators on [B, C, N]
def pool(U, kind):
    """Max-pooling over the site order; returns (V, first) where first[...] is
    True where the window's first element is the maximum (ties included)."""
    if kind == 'cnn1':
        a, b = U[..., 0::2], U[..., 1::2]
    else:
        a, b = U, np.roll(U, -1, axis=-1)       # window s covers s and (s + 1) mod N
    first = a >= b
    return np.where(first, a, b), first


def tconv(V, T, gamma, kind):
    """Transposed convolution with kernel 2: stride 2 (CNN1), stride 1 with
    periodic wrap (CNN2)."""
    if kind == 'cnn1':
        B, _, M = V.shape
        Y = np.empty((B, T.shape[1], 2 * M))
        Y[..., 0::2] = np.einsum('co,bcj->boj', T[:, :, 0], V)
        Y[..., 1::2] = np.einsum('co,bcj->boj', T[:, :, 1], V)
    else:
        Y = np.einsum('co,bcs->bos', T[:, :, 0], V) + np.einsum('co,bcs->bos', T[:, :, 1], np.roll(V, 1, axis=-1))
    return Y + gamma[None, :, None]


def forward(params, configs, spec, return_cache=False):
    emb, blocks, final = unpack(params, spec)
    B = np.asarray(configs).shape[0]
    L, N = spec.L, spec.L * spec.L
    if spec.kind == 'cnn1':
        assert N % 2 == 0, 'CNN1 pairs sites: N must be even'
    X = encode(configs, spec, emb)                               # [B, c, L, L]
    cache = []
    for W, beta, T, gamma in blocks:
        U = conv(X, W, beta).reshape(B, W.shape[0], N)
        V, first = pool(U, spec.kind)
        Y = tconv(V, T, gamma, spec.kind)
        cache.append((X, V, first))
        X = Y.reshape(B, T.shape[1], L, L)
    if spec.kind == 'cnn2':
        Wf, bf = final
        cache.append((X, None, None))
        X = conv(X, Wf, bf)
    z = X.reshape(B, N)
    a = np.log(np.abs(z)).sum(axis=1)
    phi = np.pi * (np.sum(z < 0, axis=1) % 2)
    if return_cache:
        return a, phi, (cache, z)
    return a, phi


def _conv_backward(gU, X, W):
    """Given gU = dL/dU ([B, O, L, L]) of U = conv(X, W) + beta: per-sample dW
    [B, O, C, 3, 3], dbeta [B, O] and dX [B, C, L, L] (the adjoint of the
    periodic padding: each input site collects the gradients of every output
    that read it)."""
    dW = np.zeros((gU.shape[0],) + W.shape)
    dX = np.zeros_like(X)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            dW[:, :, :, dy + 1, dx + 1] = np.einsum('boyx,bcyx->boc', gU, shifted(X, dy, dx))
            dX += np.einsum('oc,boyx->bcyx', W[:, :, dy + 1, dx + 1], shifted(gU, -dy, -dx))
    return dW, gU.sum(axis=(2, 3)), dX


def backward(params, configs, spec):
    """(a, phi, dA, dPhi) with dA[b, k] = d a(S_b)/d theta_k and dPhi = 0."""
    emb, blocks, final = unpack(params, spec)
    a, phi, (cache, z) = forward(params, configs, spec, return_cache=True)
    B = z.shape[0]
    L, N = spec.L, spec.L * spec.L
    g = (1.0 / z).reshape(B, 1, L, L)                            # d a / d z
    grads = []
    if spec.kind == 'cnn2':
        Wf, _ = final
        Xf = cache[-1][0]
        dWf, dbf, g = _conv_backward(g, Xf, Wf)
        grads.append([dWf.reshape(B, -1), dbf])
    for bi in range(len(blocks) - 1, -1, -1):
        W, beta, T, gamma = blocks[bi]
        X, V, first = cache[bi]
        gY = g.reshape(B, T.shape[1], N)
        dgamma = gY.sum(axis=2)
        if spec.kind == 'cnn1':
            dT = np.stack([np.einsum('boj,bcj->bco', gY[..., 0::2], V),
                           np.einsum('boj,bcj->bco', gY[..., 1::2], V)], axis=-1)
            gV = np.einsum('co,boj->bcj', T[:, :, 0], gY[..., 0::2]) + np.einsum('co,boj->bcj', T[:, :, 1], gY[..., 1::2])
            gU = np.zeros((B, W.shape[0], N))
            gU[..., 0::2] = np.where(first, gV, 0.0)
            gU[..., 1::2] = np.where(first, 0.0, gV)
        else:
            Vm1 = np.roll(V, 1, axis=-1)                         # V[(s - 1) mod N]
            dT = np.stack([np.einsum('bos,bcs->bco', gY, V), np.einsum('bos,bcs->bco', gY, Vm1)], axis=-1)
            gV = np.einsum('co,bos->bcs', T[:, :, 0], gY) + np.einsum('co,bos->bcs', T[:, :, 1], np.roll(gY, -1, axis=-1))
            # window s sends gV[s] to s (first) or s + 1 (second)
            gU = np.where(first, gV, 0.0) + np.roll(np.where(first, 0.0, gV), 1, axis=-1)
        dW, dbeta, gX = _conv_backward(gU.reshape(B, W.shape[0], L, L), X, W)
        grads.append([dW.reshape(B, -1), dbeta, dT.reshape(B, -1), dgamma])
        g = gX
    grads.reverse()
    parts = []
    if spec.kind == 'cnn2':
        v = state_index(configs, spec)                           # [B, N]
        gX0 = g.reshape(B, spec.channels, N)
        dE = np.zeros((B, n_states(spec), spec.channels))
        for k in range(n_states(spec)):
            dE[:, k, :] = np.einsum('bcs,bs->bc', gX0, (v == k).astype(np.float64))
        parts.append(dE.reshape(B, -1))
    for gr in grads:
        parts.extend(gr)
    dA = np.concatenate(parts, axis=1)
    assert dA.shape[1] == param_count(spec)
    return a, phi, dA, np.zeros_like(dA)
