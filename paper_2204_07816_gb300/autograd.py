"""log psi as a differentiable torch function backed by the C ABI.

LogPsi.apply(params, configs, context, precision) returns the [n, 2] float64
tensor (a, phi) of nqs_logpsi (Eq. 1: W(S) = exp(a + i phi)); its backward
multiplies the incoming gradient by the per-sample local derivatives of
nqs_logpsi_grad (Sec. 3.2: the backward of the network gives O_loc):

    d L / d theta = sum_s  g_a[s] * d a(S_s)/d theta + g_phi[s] * d phi(S_s)/d theta

The per-sample backward kernel recomputes every activation from the
configuration, so nothing is stored between forward and backward. The
[2 n, P] matrix of local derivatives is produced in chunks of samples whose
size follows `max_bytes` (default: a quarter of the free device memory), so
the product works when N_samples x P does not fit in HBM.
"""

import torch


def _chunk_rows(P, max_bytes, device):
    if max_bytes is None:
        free, _ = torch.cuda.mem_get_info(device)
        max_bytes = free // 4
    return max(1, int(max_bytes // (2 * P * 8)))


class LogPsi(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, configs, context, precision='fp64', max_bytes=None):
        if params.data_ptr() != context.params.data_ptr():
            raise ValueError('params must be the tensor the context was created with')
        fctx.context = context
        fctx.precision = precision
        fctx.max_bytes = max_bytes
        fctx.save_for_backward(configs)
        return context.logpsi(configs, precision)

    @staticmethod
    def backward(fctx, grad_out):
        (configs,) = fctx.saved_tensors
        ctx = fctx.context
        n = configs.shape[0]
        grad = torch.zeros(ctx.P, dtype=torch.float64, device=configs.device)
        rows = _chunk_rows(ctx.P, fctx.max_bytes, configs.device)
        g = grad_out.to(torch.float64)
        for s0 in range(0, n, rows):
            s1 = min(n, s0 + rows)
            O = ctx.logpsi_grad(configs[s0:s1].contiguous(), fctx.precision)
            m = s1 - s0
            grad += g[s0:s1, 0] @ O[:m] + g[s0:s1, 1] @ O[m:]
        return grad, None, None, None, None


def logpsi(params, configs, context, precision='fp64', max_bytes=None):
    return LogPsi.apply(params, configs, context, precision, max_bytes)
