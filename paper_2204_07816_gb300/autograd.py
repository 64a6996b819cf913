"""log psi as a differentiable torch function backed by the C ABI.

LogPsi.apply(params, configs, context, precision) returns the [n, 2] float64
tensor (a, phi) of nqs_logpsi (Eq. 1: W(S) = exp(a + i phi)); its backward is
nqs_logpsi_vjp, the per-sample backward of the network (Sec. 3.2: the
backward gives O_loc) seeded with the incoming gradient:

    d L / d theta = sum_s  g_a[s] * d a(S_s)/d theta + g_phi[s] * d phi(S_s)/d theta

The backward kernel recomputes every activation from the configuration, so
nothing is stored between forward and backward, and it sums the samples'
vectors on the device without forming the [2 n, P] matrix of local
derivatives, so the product works whatever N_samples x P is.
"""

import torch


class LogPsi(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, configs, context, precision='fp64'):
        if params.data_ptr() != context.params.data_ptr():
            raise ValueError('params must be the tensor the context was created with')
        fctx.context = context
        fctx.precision = precision
        fctx.save_for_backward(configs)
        return context.logpsi(configs, precision)

    @staticmethod
    def backward(fctx, grad_out):
        (configs,) = fctx.saved_tensors
        g = grad_out.to(torch.float64).contiguous()
        return fctx.context.logpsi_vjp(configs, g, fctx.precision), None, None, None


def logpsi(params, configs, context, precision='fp64'):
    return LogPsi.apply(params, configs, context, precision)
