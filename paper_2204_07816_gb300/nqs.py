"""Python binding of libnqs (include/nqs.h): argument marshalling only.

Every function below forwards to the C entry point of the same name. Tensors
must be CUDA tensors on the context's device, contiguous, with the dtypes the
header states; the stream is taken from torch's current stream at init.
No computation happens here: if the compiled library is missing the import
fails, there is no fallback.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libnqs.so')

NQS_OK = 0
STATUS = {0: 'NQS_OK', -1: 'NQS_ERR_INVALID_ARG', -2: 'NQS_ERR_OOM', -3: 'NQS_ERR_CUDA', -4: 'NQS_ERR_NONFINITE',
          -5: 'NQS_ERR_NOT_CONVERGED', -6: 'NQS_ERR_TIMEOUT', -7: 'NQS_ERR_UNSUPPORTED', -8: 'NQS_ERR_BOUNDS'}
NQS_ERR_NOT_CONVERGED = -5
NQS_ERR_UNSUPPORTED = -7
PRECISION = {'fp64': 0, 'fp32': 1, 'bf16': 2, 'fp8': 3}
SX_ARITHMETIC = {'double_float': 0, 'fp64': 1}
MODEL = {'j1j2': 0, 'tj': 1}

EXPORTS = ('nqs_param_count', 'nqs_init', 'nqs_destroy', 'nqs_last_error', 'nqs_sync', 'nqs_kernel_launches',
           'nqs_logpsi',
           'nqs_connected', 'nqs_local_energy', 'nqs_local_energy_multi', 'nqs_sample', 'nqs_get_chains', 'nqs_set_chains',
           'nqs_logpsi_grad', 'nqs_logpsi_vjp', 'nqs_logpsi_grad_noalloc', 'nqs_noalloc_last_error', 'nqs_sr_solve',
           'nqs_sr_solve_woodbury', 'nqs_set_sx_arithmetic', 'nqs_tc_plan', 'nqs_probe_wait_timeout', 'nqs_probe_bounds', 'nqs_set_sm_limit',
           'nqs_sampler_counts')


class nqs_problem(ctypes.Structure):
    _fields_ = [('model', ctypes.c_int32), ('L', ctypes.c_int32), ('J1', ctypes.c_double), ('J2', ctypes.c_double),
                ('t', ctypes.c_double), ('J', ctypes.c_double), ('n_up', ctypes.c_int32),
                ('n_down', ctypes.c_int32), ('sign_rule', ctypes.c_int32), ('n_layers', ctypes.c_int32),
                ('channels', ctypes.c_int32), ('net', ctypes.c_int32)]


class NQSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (STATUS.get(code, code), msg))
        self.code = code


_lib = None


def load(path=None):
    """Load libnqs.so (raises OSError if it has not been built). path
    defaults to $NQS_LIBRARY (another build, for instance the checked
    libnqs_checked.so), else the in-tree libnqs.so."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get('NQS_LIBRARY') or LIB_PATH
    if not os.path.exists(path):
        raise OSError('libnqs.so not found at %s: run paper_2204_07816_gb300/build.py' % path)
    lib = ctypes.CDLL(path)
    P, I32, I64, U64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        'nqs_param_count': (I64, [ctypes.POINTER(nqs_problem)]),
        'nqs_tc_plan': (ctypes.c_int, [ctypes.POINTER(nqs_problem), I32, I64, I32, I32, ctypes.POINTER(I32)]),
        'nqs_init': (ctypes.c_int, [ctypes.POINTER(P), ctypes.POINTER(nqs_problem), P, U64, P]),
        'nqs_destroy': (ctypes.c_int, [P]),
        'nqs_last_error': (ctypes.c_char_p, [P]),
        'nqs_sync': (ctypes.c_int, [P]),
        'nqs_kernel_launches': (I64, [P]),
        'nqs_probe_wait_timeout': (ctypes.c_int, [P, I64]),
        'nqs_probe_bounds': (ctypes.c_int, [P]),
        'nqs_set_sm_limit': (ctypes.c_int, [P, I32]),
        'nqs_sampler_counts': (ctypes.c_int, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), I32]),
        'nqs_logpsi': (ctypes.c_int, [P, P, I64, P, I32]),
        'nqs_connected': (ctypes.c_int, [P, P, I64, I32, P, P, P, P]),
        'nqs_local_energy': (ctypes.c_int, [P, P, P, I64, P, I32]),
        'nqs_local_energy_multi': (ctypes.c_int, [P, I32, P, P, P, P, I32, I32]),
        'nqs_sample': (ctypes.c_int, [P, I32, I32, I32, I32, P, P, I32]),
        'nqs_get_chains': (ctypes.c_int, [P, I32, P, ctypes.POINTER(U64)]),
        'nqs_set_chains': (ctypes.c_int, [P, I32, P, U64]),
        'nqs_logpsi_grad': (ctypes.c_int, [P, P, I64, P, I32]),
        'nqs_logpsi_vjp': (ctypes.c_int, [P, P, I64, P, P, I32]),
        'nqs_logpsi_grad_noalloc': (ctypes.c_int, [ctypes.POINTER(nqs_problem), P, P, I64, P, I32, P]),
        'nqs_noalloc_last_error': (ctypes.c_char_p, []),
        'nqs_sr_solve': (ctypes.c_int, [P, P, P, I64, D, D, I32, D, P, ctypes.POINTER(I32), ctypes.POINTER(D),
                                        ctypes.POINTER(D), I32]),
        'nqs_sr_solve_woodbury': (ctypes.c_int, [P, P, P, I64, D, D, I32, P, ctypes.POINTER(D), ctypes.POINTER(D),
                                                 I32]),
        'nqs_set_sx_arithmetic': (ctypes.c_int, [P, I32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t, dtype, name):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError('%s must be a CUDA tensor' % name)
    if t.dtype != dtype:
        raise TypeError('%s must be %s, got %s' % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError('%s must be contiguous' % name)
    return ctypes.c_void_p(t.data_ptr())


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


NET = {'silu': 0, 'cnn1': 1, 'cnn2': 2}


def make_problem(model='j1j2', L=4, J1=1.0, J2=0.5, t=1.0, J=0.4, n_up=None, n_down=None, sign_rule=False,
                 n_layers=2, channels=4, net='silu'):
    N = L * L
    if n_up is None:
        n_up = N // 2
    if n_down is None:
        n_down = N - n_up
    return nqs_problem(MODEL[model] if isinstance(model, str) else int(model), L, J1, J2, t, J, n_up, n_down,
                       int(bool(sign_rule)), n_layers, channels, NET[net] if isinstance(net, str) else int(net))


def nqs_param_count(problem):
    return load().nqs_param_count(ctypes.byref(problem))


TC_PLAN_KIND = {'logpsi': 0, 'local_energy': 1, 'sample': 2}
TC_PLAN_FIELDS = ('G', 'slots', 'blocks_per_sm', 'epilogue_warps', 'tiles', 'smem_bytes', 'tmem_cols', 'grid',
                  'row_form')


def tc_plan(problem, kind, n, max_smem_per_block=232448, num_sms=152):
    """nqs_tc_plan: the tensor-core plan the launchers choose (host only).
    kind: 'logpsi', 'local_energy' (n = samples) or 'sample' (n = chains).
    Returns a dict of TC_PLAN_FIELDS, or None if the tensor-core path cannot
    run the problem."""
    out = (ctypes.c_int32 * 9)()
    rc = load().nqs_tc_plan(ctypes.byref(problem), TC_PLAN_KIND[kind], int(n), int(max_smem_per_block), int(num_sms),
                            out)
    if rc == NQS_ERR_UNSUPPORTED:
        return None
    if rc != 0:
        raise NQSError(rc, 'nqs_tc_plan: invalid argument')
    return dict(zip(TC_PLAN_FIELDS, list(out)))


def local_energy_multi(contexts, configs, precision='bf16', outs=None, logpsi=None, max_blocks=0):
    """nqs_local_energy_multi: E_loc of several contexts' configurations in
    one pass, enqueued on the first context's stream. Returns the list of
    [n_i, 2] float64 outputs."""
    lib = load()
    k = len(contexts)
    if outs is None:
        outs = [torch.empty((c.shape[0], 2), dtype=torch.float64, device=c.device) for c in configs]
    Arr = ctypes.c_void_p * k
    ctx_arr = Arr(*[c.ctx.value for c in contexts])
    cfg_arr = Arr(*[ctx._configs(c).value for ctx, c in zip(contexts, configs)])
    out_arr = Arr(*[_ptr(o, torch.float64, 'out').value for o in outs])
    lp_arr = Arr(*[_ptr(l, torch.float64, 'logpsi').value for l in logpsi]) if logpsi is not None else None
    n_arr = (ctypes.c_int64 * k)(*[c.shape[0] for c in configs])
    rc = lib.nqs_local_energy_multi(ctx_arr, k, cfg_arr, lp_arr, n_arr, out_arr, _prec(precision), int(max_blocks))
    if rc != NQS_OK:
        raise NQSError(rc, lib.nqs_last_error(contexts[0].ctx).decode())
    return outs


def nqs_logpsi_grad_noalloc(problem, params, configs, O_out, precision='fp64', stream=None):
    """Local derivatives through the allocation-free entry point (no context,
    no device allocation; see include/nqs.h). O_out: float64 [2n, P]."""
    lib = load()
    n = configs.shape[0]
    if stream is None:
        stream = torch.cuda.current_stream(configs.device)
    rc = lib.nqs_logpsi_grad_noalloc(ctypes.byref(problem), _ptr(params, torch.float64, 'params'),
                                     _ptr(configs, torch.int8, 'configs'), n, _ptr(O_out, torch.float64, 'O_out'),
                                     _prec(precision), ctypes.c_void_p(stream.cuda_stream))
    if rc != NQS_OK:
        raise NQSError(rc, lib.nqs_noalloc_last_error().decode())
    return O_out


class Context:
    """Owns one nqs_ctx. params: float64 CUDA tensor [P], borrowed (kept
    alive by this object) and updated in place by sr_solve(apply_update=True)."""

    def __init__(self, problem, params, seed=0, stream=None):
        lib = load()
        self.lib = lib
        self.problem = problem
        self.params = params
        self.N = problem.L * problem.L
        self.P = lib.nqs_param_count(ctypes.byref(problem))
        if self.P < 0:
            raise NQSError(-1, 'invalid problem')
        if params.numel() != self.P:
            raise ValueError('params has %d entries, problem needs %d' % (params.numel(), self.P))
        pptr = _ptr(params, torch.float64, 'params')   # a float64 CUDA tensor, checked before any CUDA call
        self.device = params.device
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        self.ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.nqs_init(ctypes.byref(self.ctx), ctypes.byref(problem), pptr, ctypes.c_uint64(seed),
                              ctypes.c_void_p(stream.cuda_stream))
        if rc != NQS_OK:
            raise NQSError(rc, lib.nqs_last_error(None).decode())

    def _check(self, rc, allow=()):
        if rc != NQS_OK and rc not in allow:
            raise NQSError(rc, self.lib.nqs_last_error(self.ctx).decode())
        return rc

    def close(self):
        if self.ctx:
            rc = self.lib.nqs_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()
            self._check(rc)

    def __del__(self):
        try:
            if self.ctx:
                self.lib.nqs_destroy(self.ctx)
                self.ctx = ctypes.c_void_p()
        except Exception:
            pass

    def sync(self):
        return self._check(self.lib.nqs_sync(self.ctx))

    def kernel_launches(self):
        return int(self.lib.nqs_kernel_launches(self.ctx))

    def _configs(self, configs):
        if configs.dim() != 2 or configs.shape[1] != self.N:
            raise ValueError('configs must be [n, %d] int8' % self.N)
        return _ptr(configs, torch.int8, 'configs')

    def logpsi(self, configs, precision='fp64', out=None):
        n = configs.shape[0]
        if out is None:
            out = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        self._check(self.lib.nqs_logpsi(self.ctx, self._configs(configs), n, _ptr(out, torch.float64, 'out'),
                                        _prec(precision)))
        return out

    def connected(self, configs, max_conn=None):
        n = configs.shape[0]
        nb = (4 if self.problem.model == 0 else 2) * self.N
        max_conn = max_conn or nb
        dev = self.device
        n_conn = torch.zeros(n, dtype=torch.int32, device=dev)
        pairs = torch.zeros((n, max_conn, 2), dtype=torch.int32, device=dev)
        h = torch.zeros((n, max_conn), dtype=torch.float64, device=dev)
        hdiag = torch.zeros(n, dtype=torch.float64, device=dev)
        self._check(self.lib.nqs_connected(self.ctx, self._configs(configs), n, max_conn,
                                           _ptr(n_conn, torch.int32, 'n_conn'), _ptr(pairs, torch.int32, 'pairs'),
                                           _ptr(h, torch.float64, 'h'), _ptr(hdiag, torch.float64, 'hdiag')))
        return n_conn, pairs, h, hdiag

    def local_energy(self, configs, logpsi=None, precision='fp64', out=None):
        n = configs.shape[0]
        if out is None:
            out = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        if logpsi is not None and tuple(logpsi.shape) != (n, 2):
            raise ValueError('logpsi must be [n, 2]')
        self._check(self.lib.nqs_local_energy(self.ctx, self._configs(configs), _ptr(logpsi, torch.float64, 'logpsi'),
                                              n, _ptr(out, torch.float64, 'out'), _prec(precision)))
        return out

    def sample(self, n_chains, samples_per_chain, sweeps_between=1, burn_in=10, precision='fp64', out=None,
               logpsi_out=None):
        """nqs_sample; out / logpsi_out: optional contiguous [n, N] int8 and [n, 2] float64 device tensors
        (for instance row slices of a larger buffer) that receive the samples."""
        n = n_chains * samples_per_chain
        cfg = out if out is not None else torch.empty((n, self.N), dtype=torch.int8, device=self.device)
        lp = logpsi_out if logpsi_out is not None else torch.empty((n, 2), dtype=torch.float64, device=self.device)
        if tuple(cfg.shape) != (n, self.N) or tuple(lp.shape) != (n, 2):
            raise ValueError('out must be [%d, %d] and logpsi_out [%d, 2]' % (n, self.N, n))
        self._check(self.lib.nqs_sample(self.ctx, n_chains, samples_per_chain, sweeps_between, burn_in,
                                        _ptr(cfg, torch.int8, 'configs_out'), _ptr(lp, torch.float64, 'logpsi_out'),
                                        _prec(precision)))
        return cfg, lp

    def sampler_counts(self, reset=False):
        """nqs_sampler_counts: (moves, accepted) since creation or the last reset."""
        mv, ac = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.nqs_sampler_counts(self.ctx, ctypes.byref(mv), ctypes.byref(ac), int(bool(reset))))
        return mv.value, ac.value

    def set_sm_limit(self, sms):
        """nqs_set_sm_limit: size later launches for `sms` SMs (0 = all)."""
        self._check(self.lib.nqs_set_sm_limit(self.ctx, int(sms)))

    def probe_wait_timeout(self, iterations=1000):
        """nqs_probe_wait_timeout: a bounded device wait that runs out; the
        next sync() raises NQSError with NQS_ERR_TIMEOUT."""
        self._check(self.lib.nqs_probe_wait_timeout(self.ctx, int(iterations)))

    def probe_bounds(self):
        """nqs_probe_bounds: report one failed device-side index check; the
        next sync() raises NQSError with NQS_ERR_BOUNDS."""
        self._check(self.lib.nqs_probe_bounds(self.ctx))

    def get_chains(self, n_chains):
        out = torch.empty((n_chains, self.N), dtype=torch.int8, device=self.device)
        step = ctypes.c_uint64()
        self._check(self.lib.nqs_get_chains(self.ctx, n_chains, _ptr(out, torch.int8, 'chains'), ctypes.byref(step)))
        return out, step.value

    def set_chains(self, chains, step):
        self._check(self.lib.nqs_set_chains(self.ctx, chains.shape[0], _ptr(chains, torch.int8, 'chains'),
                                            ctypes.c_uint64(step)))

    def logpsi_grad(self, configs, precision='fp64', out=None):
        n = configs.shape[0]
        if out is None:
            out = torch.empty((2 * n, self.P), dtype=torch.float64, device=self.device)
        self._check(self.lib.nqs_logpsi_grad(self.ctx, self._configs(configs), n, _ptr(out, torch.float64, 'O_out'),
                                             _prec(precision)))
        return out

    def logpsi_vjp(self, configs, grad_logpsi, precision='fp64', out=None):
        """nqs_logpsi_vjp: sum over samples of g_a d a / d theta + g_phi d phi / d theta ([P] float64)."""
        n = configs.shape[0]
        if tuple(grad_logpsi.shape) != (n, 2):
            raise ValueError('grad_logpsi must be [n, 2]')
        if out is None:
            out = torch.empty(self.P, dtype=torch.float64, device=self.device)
        self._check(self.lib.nqs_logpsi_vjp(self.ctx, self._configs(configs), n,
                                            _ptr(grad_logpsi, torch.float64, 'grad_logpsi'),
                                            _ptr(out, torch.float64, 'grad_params'), _prec(precision)))
        return out

    def sr_solve_woodbury(self, O, eloc, eps=1e-4, lr=0.02, apply_update=False, delta=None, refine_steps=0):
        """nqs_sr_solve_woodbury: delta from the 2n x 2n sample-space system."""
        n = eloc.shape[0]
        if tuple(O.shape) != (2 * n, self.P):
            raise ValueError('O must be [2n, P]')
        if delta is None:
            delta = torch.empty(self.P, dtype=torch.float64, device=self.device)
        resid = ctypes.c_double()
        energy = (ctypes.c_double * 2)()
        self._check(self.lib.nqs_sr_solve_woodbury(self.ctx, _ptr(O, torch.float64, 'O'),
                                                   _ptr(eloc, torch.float64, 'eloc'), n, eps, lr,
                                                   int(refine_steps), _ptr(delta, torch.float64, 'delta'),
                                                   ctypes.byref(resid),
                                                   ctypes.cast(energy, ctypes.POINTER(ctypes.c_double)),
                                                   int(bool(apply_update))))
        return delta, {'resid': resid.value, 'energy': complex(energy[0], energy[1])}

    def set_sx_arithmetic(self, mode):
        """nqs_set_sx_arithmetic: 'double_float' (default) or 'fp64' S.x passes in later sr_solve calls."""
        self._check(self.lib.nqs_set_sx_arithmetic(self.ctx, SX_ARITHMETIC[mode]))

    def sr_solve(self, O, eloc, eps=1e-4, rtol=1e-8, max_iter=10000, lr=0.02, apply_update=False, delta=None):
        n = eloc.shape[0]
        if tuple(O.shape) != (2 * n, self.P):
            raise ValueError('O must be [2n, P]')
        if delta is None:
            delta = torch.empty(self.P, dtype=torch.float64, device=self.device)
        iters = ctypes.c_int32()
        resid = ctypes.c_double()
        energy = (ctypes.c_double * 2)()
        rc = self.lib.nqs_sr_solve(self.ctx, _ptr(O, torch.float64, 'O'), _ptr(eloc, torch.float64, 'eloc'), n,
                                   eps, rtol, max_iter, lr, _ptr(delta, torch.float64, 'delta'), ctypes.byref(iters),
                                   ctypes.byref(resid), ctypes.cast(energy, ctypes.POINTER(ctypes.c_double)),
                                   int(bool(apply_update)))
        self._check(rc, allow=(NQS_ERR_NOT_CONVERGED,))
        return delta, {'iters': iters.value, 'resid': resid.value, 'energy': complex(energy[0], energy[1]),
                       'converged': rc == NQS_OK}
