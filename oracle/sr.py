"""Stochastic reconfiguration (Sec. 3.2: gradients and covariance matrix of the
SR method, parameter update by delta; Sec. 5.4.1 "Distributed SR
computation": covariance matrix from the [samples x parameters] matrix, then a
linear solve, then the update).

Inputs per sample b: the complex local derivative O_bk = dA[b,k] + i dPhi[b,k]
(cnn.backward) and the complex local energy E_b (eloc.py). With real
parameters:

    <E>    = mean_b E_b
    Oc     = O - mean_b O                               (centred)
    S_kl   = Re( sum_b conj(Oc_bk) Oc_bl ) / N_s
    F_k    = Re( sum_b conj(Oc_bk) (E_b - <E>) ) / N_s
    (S + eps * I) delta = F                              (additive shift)
    theta <- theta - lr * delta

Real-stacked form used throughout: Ohat = [Re Oc; Im Oc] is [2 N_s, P] and
Ehat = [Re(E - <E>); Im(E - <E>)], so S = Ohat^T Ohat / N_s and
F = Ohat^T Ehat / N_s.

The paper forms S explicitly and factorises it; this oracle offers that
(dense solve) and conjugate gradient on the same system with the stopping
rule ||r||_2 <= rtol * ||F||_2 from x0 = 0, and the sample-space form
(solve_woodbury): since (Ohat^T Ohat / N_s + eps I)^-1 Ohat^T
= Ohat^T (Ohat Ohat^T / N_s + eps I)^-1, the same delta is
Ohat^T y with (Ohat Ohat^T / N_s + eps I) y = Ehat / N_s, a 2 N_s x 2 N_s
system in place of the P x P one.
"""

import numpy as np


def _norm_weights(ns, weights):
    if weights is None:
        return np.full(ns, 1.0 / ns)
    w = np.asarray(weights, dtype=np.float64)
    return w / w.sum()


def centred_stack(dA, dPhi):
    """Ohat = [Re Oc; Im Oc], [2 N_s, P], centred by the plain sample mean."""
    dA = np.asarray(dA, dtype=np.float64)
    dPhi = np.asarray(dPhi, dtype=np.float64)
    return np.concatenate([dA - dA.mean(axis=0), dPhi - dPhi.mean(axis=0)], axis=0)


def force(dA, dPhi, eloc, weights=None):
    """F and <E>. `weights` (default: every sample 1) turns the sample means
    into weighted means; with |psi|^2 weights over a whole sector it gives the
    exact expectation values."""
    dA = np.asarray(dA, dtype=np.float64)
    dPhi = np.asarray(dPhi, dtype=np.float64)
    eloc = np.asarray(eloc, dtype=np.complex128)
    w = _norm_weights(eloc.size, weights)
    e_mean = w @ eloc
    oc_re = dA - w @ dA
    oc_im = dPhi - w @ dPhi
    de = eloc - e_mean
    return oc_re.T @ (w * de.real) + oc_im.T @ (w * de.imag), e_mean


def s_matrix(dA, dPhi, weights=None):
    dA = np.asarray(dA, dtype=np.float64)
    dPhi = np.asarray(dPhi, dtype=np.float64)
    w = _norm_weights(dA.shape[0], weights)
    oc_re = dA - w @ dA
    oc_im = dPhi - w @ dPhi
    return oc_re.T @ (w[:, None] * oc_re) + oc_im.T @ (w[:, None] * oc_im)


def solve_dense(dA, dPhi, eloc, eps):
    F, e_mean = force(dA, dPhi, eloc)
    S = s_matrix(dA, dPhi)
    return np.linalg.solve(S + eps * np.eye(S.shape[0]), F), e_mean


def solve_woodbury(dA, dPhi, eloc, eps):
    """delta from the 2 N_s x 2 N_s sample-space system (eps > 0); returns
    (delta, <E>)."""
    eloc = np.asarray(eloc, dtype=np.complex128)
    e_mean = eloc.mean()
    Oh = centred_stack(dA, dPhi)
    ns = eloc.size
    eh = np.concatenate([(eloc - e_mean).real, (eloc - e_mean).imag])
    T = Oh @ Oh.T / ns
    y = np.linalg.solve(T + eps * np.eye(2 * ns), eh / ns)
    return Oh.T @ y, e_mean


def s_times(Oh, ns, eps, x):
    """Matrix-free (S + eps I) x = Ohat^T (Ohat x) / N_s + eps x."""
    return Oh.T @ (Oh @ x) / ns + eps * x


def cg(dA, dPhi, eloc, eps, rtol, max_iter):
    """Conjugate gradient on (S + eps I) delta = F from delta = 0.

    Returns (delta, iterations, relative residual, <E>).
    """
    F, e_mean = force(dA, dPhi, eloc)
    Oh = centred_stack(dA, dPhi)
    ns = Oh.shape[0] // 2
    x = np.zeros_like(F)
    r = F.copy()
    p = r.copy()
    rs = r @ r
    fnorm = np.sqrt(F @ F)
    if fnorm == 0.0:
        return x, 0, 0.0, e_mean
    it = 0
    while it < max_iter and np.sqrt(rs) > rtol * fnorm:
        Ap = s_times(Oh, ns, eps, p)
        alpha = rs / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rs_new = r @ r
        p = r + (rs_new / rs) * p
        rs = rs_new
        it += 1
    return x, it, np.sqrt(rs) / fnorm, e_mean


def update(params, delta, lr):
    return np.asarray(params, dtype=np.float64) - lr * np.asarray(delta)
