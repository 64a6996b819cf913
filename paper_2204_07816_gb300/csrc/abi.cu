// C ABI of the library (declared in include/nqs.h): context lifetime,
// argument validation, workspace and chain-state ownership, dispatch to the
// CUDA-core and tensor-core kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "paper_net.cuh"

using namespace nqs;

namespace {
// NVTX range around each compute entry point (header-only NVTX: a no-op unless a profiler is attached), so
// timelines and ncu's --nvtx filters see the library's calls by name.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace

struct nqs_ctx {
    Problem p;
    nqs_problem spec;
    double *params = nullptr;      // borrowed
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    int sm_limit = 0;              // 0: whole device; else grids are sized for this many SMs
    size_t max_smem = 0;
    int *err_dev = nullptr;        // device error bits (int), then at +16 B the sampler counters (2 x u64)
    float *params32 = nullptr;     // float copy for the FP32 path
    void *packed = nullptr;        // tensor-core operand images
    int8_t *chains = nullptr;
    int n_chains = 0;
    uint64_t step = 0;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    int64_t launches = 0;
    int cg_hint = 0;               // iterations of the last CG solve (sizes the next solve's first launch batch)
    int sx_arith = NQS_SX_DOUBLE_FLOAT;   // arithmetic of the CG's S.x passes
    void *multi_table = nullptr;   // request table of grouped launches led by this context
    size_t multi_table_bytes = 0;
    std::string msg;
};

namespace {

const char *kNoCtx = "no context";
// sample-space SR: the 2n x 2n float64 matrix of n = 32,768 samples takes 34 GB
constexpr int64_t kWoodburyMaxSamples = 32768;
thread_local std::string g_init_error;

int fail(nqs_ctx *c, int code, const std::string &m) {
    if (c) c->msg = m;
    return code;
}

int cuda_fail(nqs_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? NQS_ERR_OOM : NQS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

bool valid_problem(const nqs_problem *q, std::string *why) {
    if (!q) { *why = "problem is NULL"; return false; }
    if (q->model != NQS_MODEL_J1J2 && q->model != NQS_MODEL_TJ) { *why = "model must be 0 (J1-J2) or 1 (t-J)"; return false; }
    if (q->L < 4 || q->L > 36) { *why = "L must be in [4, 36]"; return false; }
    if (q->n_layers < 1 || q->n_layers > 16) { *why = "n_layers must be in [1, 16]"; return false; }
    if (q->channels != 4 && q->channels != 8 && q->channels != 16 && q->channels != 32) {
        *why = "channels must be 4, 8, 16 or 32";
        return false;
    }
    const int N = q->L * q->L;
    if (q->n_up < 0 || q->n_down < 0 || q->n_up + q->n_down > N) { *why = "bad n_up / n_down"; return false; }
    if (q->model == NQS_MODEL_J1J2 && q->n_up + q->n_down != N) { *why = "J1-J2 needs n_up + n_down = L*L"; return false; }
    if (q->sign_rule != 0 && q->sign_rule != 1) { *why = "sign_rule must be 0 or 1"; return false; }
    if (q->sign_rule && q->model != NQS_MODEL_J1J2) { *why = "sign_rule applies to J1-J2 only"; return false; }
    if (q->net != NQS_NET_SILU && q->net != NQS_NET_CNN1 && q->net != NQS_NET_CNN2) {
        *why = "net must be 0 (SiLU stack), 1 (CNN1) or 2 (CNN2)";
        return false;
    }
    if (q->net == NQS_NET_CNN1 && N % 2) { *why = "CNN1 pools pairs of sites: L * L must be even"; return false; }
    return true;
}

Problem make_problem(const nqs_problem *q) {
    Problem p;
    p.model = q->model;
    p.L = q->L;
    p.N = q->L * q->L;
    p.c_in = q->model == NQS_MODEL_J1J2 ? 1 : 3;
    p.C = q->channels;
    p.n_layers = q->n_layers;
    p.J1 = q->J1; p.J2 = q->J2; p.t = q->t; p.J = q->J;
    p.sign_rule = q->sign_rule;
    p.net = q->net;
    p.P = p.net == NQS_NET_SILU ? (9 * p.c_in * p.C + p.C) + (p.n_layers - 1) * (9 * p.C * p.C + p.C) + 2 * p.C
                                : paper_param_count(p);
    p.n_bonds = (q->model == NQS_MODEL_J1J2 ? 4 : 2) * p.N;
    p.n_up = q->n_up;
    p.n_down = q->n_down;
    return p;
}

int sms_of(const nqs_ctx *c) { return (c->sm_limit > 0 && c->sm_limit < c->num_sms) ? c->sm_limit : c->num_sms; }

LaunchEnv env_of(nqs_ctx *c) {
    LaunchEnv e;
    e.stream = c->stream;
    e.num_sms = sms_of(c);
    e.sm_limited = e.num_sms < c->num_sms;
    e.max_smem = c->max_smem;
    e.err = c->err_dev;
    e.moves = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(c->err_dev) + 16);
    e.launches = &c->launches;
    e.msg = &c->msg;
    return e;
}

bool valid_precision(int prec) { return prec == NQS_FP64 || prec == NQS_FP32 || prec == NQS_BF16; }

// Prepare the parameter image a precision needs (read from the caller's
// float64 vector on every call, so caller-side changes are always seen).
int prepare_params(nqs_ctx *c, int prec, DeviceParams *dp) {
    dp->p64 = c->params;
    dp->p32 = c->params32;
    if (prec == NQS_FP32) {
        launch_convert_params(c->params, c->params32, c->p.P, c->stream);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "convert params");
        ++c->launches;
    } else if (prec == NQS_BF16 || prec == NQS_FP8) {
        LaunchEnv env = env_of(c);
        int rc = launch_tc_pack(c->p, c->params, c->packed, env);
        if (rc) return rc;
    }
    return NQS_OK;
}

int ensure_scratch(nqs_ctx *c, size_t bytes) {
    if (bytes <= c->scratch_bytes) return NQS_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    e = cudaMalloc(&c->scratch, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "workspace allocation");
    c->scratch_bytes = bytes;
    return NQS_OK;
}

int check_ctx(nqs_ctx *c) {
    if (!c) return NQS_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return NQS_OK;
}

}  // namespace

extern "C" {

int64_t nqs_param_count(const nqs_problem *q) {
    std::string why;
    if (!valid_problem(q, &why)) return -1;
    return make_problem(q).P;
}

int nqs_tc_plan(const nqs_problem *q, int32_t kind, int64_t n, int32_t max_smem_per_block, int32_t num_sms,
                int32_t *out) {
    std::string why;
    if (!out || kind < 0 || kind > 2 || n < 1 || max_smem_per_block <= 0 || num_sms <= 0) return NQS_ERR_INVALID_ARG;
    if (!valid_problem(q, &why)) return NQS_ERR_INVALID_ARG;
    if (kind == 2 && n > INT32_MAX) return NQS_ERR_INVALID_ARG;
    return tc_describe_plan(make_problem(q), kind, n, (size_t)max_smem_per_block, num_sms, out, &why);
}

int nqs_init(nqs_ctx **out, const nqs_problem *q, double *params, uint64_t seed, void *stream) {
    if (!out) return NQS_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    if (!valid_problem(q, &why)) { g_init_error = why; return NQS_ERR_INVALID_ARG; }
    if (!params) { g_init_error = "params is NULL"; return NQS_ERR_INVALID_ARG; }
    nqs_ctx *c = new nqs_ctx();
    c->spec = *q;
    c->p = make_problem(q);
    c->params = params;
    c->seed = seed;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { g_init_error = cudaGetErrorString(e); delete c; return NQS_ERR_CUDA; }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, c->device);
    if (e != cudaSuccess) { g_init_error = cudaGetErrorString(e); delete c; return NQS_ERR_CUDA; }
    if (prop.major != 10) {
        g_init_error = "needs a Blackwell (sm_10x) GPU";
        delete c;
        return NQS_ERR_CUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->max_smem = prop.sharedMemPerBlockOptin;
    e = cudaMalloc(&c->err_dev, 32);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err_dev, 0, 32, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&c->params32, sizeof(float) * c->p.P);
    if (e == cudaSuccess) {
        const size_t pk = tc_packed_bytes(c->p);
        e = cudaMalloc(&c->packed, pk ? pk : 16);
    }
    if (e != cudaSuccess) {
        g_init_error = std::string("allocation: ") + cudaGetErrorString(e);
        nqs_destroy(c);
        return e == cudaErrorMemoryAllocation ? NQS_ERR_OOM : NQS_ERR_CUDA;
    }
    *out = c;
    return NQS_OK;
}

int nqs_sync(nqs_ctx *c) {
    if (int rc = check_ctx(c)) return rc;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    int bits = 0;
    e = cudaMemcpy(&bits, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error flag");
    if (bits) {
        cudaMemset(c->err_dev, 0, sizeof(int));
        if (bits & ERRBIT_NONFINITE) return fail(c, NQS_ERR_NONFINITE, "a kernel produced a non-finite value");
        if (bits & ERRBIT_TIMEOUT) return fail(c, NQS_ERR_TIMEOUT, "a device-side wait ran out of iterations");
        return fail(c, NQS_ERR_BOUNDS, "a device-side index check failed");
    }
    return NQS_OK;
}

int nqs_sampler_counts(nqs_ctx *c, int64_t *moves, int64_t *accepted, int32_t reset) {
    if (int rc = check_ctx(c)) return rc;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream");
    unsigned long long h[2] = {0, 0};
    e = cudaMemcpy(h, reinterpret_cast<char *>(c->err_dev) + 16, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "sampler counters");
    if (moves) *moves = (int64_t)h[0];
    if (accepted) *accepted = (int64_t)h[1];
    if (reset) {
        e = cudaMemset(reinterpret_cast<char *>(c->err_dev) + 16, 0, sizeof(h));
        if (e != cudaSuccess) return cuda_fail(c, e, "sampler counters");
    }
    return NQS_OK;
}

int nqs_set_sm_limit(nqs_ctx *c, int32_t sms) {
    if (!c) return NQS_ERR_INVALID_ARG;
    if (sms < 0 || sms > c->num_sms) return fail(c, NQS_ERR_INVALID_ARG, "nqs_set_sm_limit: bad SM count");
    c->sm_limit = sms;
    return NQS_OK;
}

int nqs_probe_wait_timeout(nqs_ctx *c, int64_t iterations) {
    if (int rc = check_ctx(c)) return rc;
    if (iterations < 1 || iterations > 1000000) return fail(c, NQS_ERR_INVALID_ARG, "nqs_probe_wait_timeout: bad count");
    LaunchEnv env = env_of(c);
    return launch_wait_probe(iterations, env);
}

int nqs_probe_bounds(nqs_ctx *c) {
    if (int rc = check_ctx(c)) return rc;
    LaunchEnv env = env_of(c);
    return launch_bounds_probe(env);
}

int nqs_destroy(nqs_ctx *c) {
    if (!c) return NQS_ERR_INVALID_ARG;
    int rc = nqs_sync(c);
    cudaFree(c->err_dev);
    cudaFree(c->params32);
    cudaFree(c->packed);
    cudaFree(c->chains);
    cudaFree(c->scratch);
    cudaFree(c->multi_table);
    delete c;
    return rc;
}

int nqs_local_energy_multi(nqs_ctx *const *ctxs, int32_t count, const int8_t *const *configs,
                           const double *const *logpsi, const int64_t *n, double *const *eloc_out, int32_t prec,
                           int32_t max_blocks) {
    NvtxRange nvtx_range("nqs_local_energy_multi");
    if (count < 1 || !ctxs || !ctxs[0] || !configs || !n || !eloc_out) return NQS_ERR_INVALID_ARG;
    nqs_ctx *lead = ctxs[0];
    if (int rc = check_ctx(lead)) return rc;
    if (!valid_precision(prec)) return fail(lead, NQS_ERR_INVALID_ARG, "nqs_local_energy_multi: bad precision");
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || ctxs[i]->device != lead->device || n[i] < 0 || (n[i] > 0 && (!configs[i] || !eloc_out[i])))
            return fail(lead, NQS_ERR_INVALID_ARG, "nqs_local_energy_multi: bad context or arrays");
    }
    LaunchEnv env = env_of(lead);
    if (prec != NQS_BF16) {
        // CUDA-core precisions: one launch per problem, all on the lead stream
        for (int i = 0; i < count; ++i) {
            nqs_ctx *c = ctxs[i];
            DeviceParams dp;
            dp.p64 = c->params;
            dp.p32 = c->params32;
            if (prec == NQS_FP32) {
                launch_convert_params(c->params, c->params32, c->p.P, lead->stream);
                ++lead->launches;
            }
            const double *lp = logpsi ? logpsi[i] : nullptr;
            if (int rc = launch_eloc_plain(c->p, prec, dp, configs[i], lp, n[i], eloc_out[i], env)) return rc;
        }
        return NQS_OK;
    }
    // tensor cores: one grouped launch per channel count
    for (int i = 0; i < count; ++i)
        if (ctxs[i]->p.C != 16 && ctxs[i]->p.C != 32)
            return fail(lead, NQS_ERR_UNSUPPORTED, "the tensor-core path needs 16 or 32 channels");
    std::vector<TcMultiItem> items;
    for (int pass = 0; pass < 2; ++pass) {
        const int C = pass == 0 ? 16 : 32;
        items.clear();
        for (int i = 0; i < count; ++i) {
            nqs_ctx *c = ctxs[i];
            if (c->p.C != C) continue;
            if (int rc = launch_tc_pack(c->p, c->params, c->packed, env)) return rc;
            TcMultiItem it;
            it.p = c->p;
            it.packed = c->packed;
            it.configs = configs[i];
            it.logpsi = logpsi ? logpsi[i] : nullptr;
            it.n = n[i];
            it.out = eloc_out[i];
            items.push_back(it);
        }
        if (items.empty()) continue;
        const size_t need = tc_multi_table_bytes((int)items.size());
        if (need > lead->multi_table_bytes) {
            cudaError_t e = cudaStreamSynchronize(lead->stream);
            if (e != cudaSuccess) return cuda_fail(lead, e, "stream sync");
            cudaFree(lead->multi_table);
            lead->multi_table = nullptr;
            lead->multi_table_bytes = 0;
            e = cudaMalloc(&lead->multi_table, need);
            if (e != cudaSuccess) return cuda_fail(lead, e, "grouped table allocation");
            lead->multi_table_bytes = need;
        }
        if (int rc = launch_eloc_tc_multi(items.data(), (int)items.size(), lead->multi_table, max_blocks, env))
            return rc;
        // the next pass reuses the table: order it after this launch (same stream)
    }
    return NQS_OK;
}

int64_t nqs_kernel_launches(const nqs_ctx *c) { return c ? c->launches : -1; }

const char *nqs_last_error(const nqs_ctx *c) {
    if (!c) return g_init_error.empty() ? kNoCtx : g_init_error.c_str();
    return c->msg.c_str();
}

int nqs_logpsi(nqs_ctx *c, const int8_t *configs, int64_t n, double *out, int32_t prec) {
    NvtxRange nvtx_range("nqs_logpsi");
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || (n > 0 && (!configs || !out))) return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi: bad arrays");
    if (!valid_precision(prec)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi: bad precision");
    if (n == 0) return NQS_OK;
    DeviceParams dp;
    if (int rc = prepare_params(c, prec, &dp)) return rc;
    LaunchEnv env = env_of(c);
    if (prec == NQS_BF16) return launch_logpsi_tc(c->p, c->params, c->packed, configs, n, out, env);
    return launch_logpsi_plain(c->p, prec, dp, configs, n, out, env);
}

int nqs_connected(nqs_ctx *c, const int8_t *configs, int64_t n, int32_t max_conn, int32_t *n_conn,
                  int32_t *pairs, double *h, double *hdiag) {
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || (n > 0 && (!configs || !n_conn || !pairs || !h || !hdiag)))
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_connected: bad arrays");
    if (max_conn < c->p.n_bonds) return fail(c, NQS_ERR_INVALID_ARG, "nqs_connected: max_conn below the bond count");
    LaunchEnv env = env_of(c);
    return launch_connected(c->p, configs, n, max_conn, n_conn, pairs, h, hdiag, env);
}

int nqs_local_energy(nqs_ctx *c, const int8_t *configs, const double *logpsi, int64_t n, double *out, int32_t prec) {
    NvtxRange nvtx_range("nqs_local_energy");
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || (n > 0 && (!configs || !out))) return fail(c, NQS_ERR_INVALID_ARG, "nqs_local_energy: bad arrays");
    if (!valid_precision(prec) && prec != NQS_FP8)
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_local_energy: bad precision");
    if (n == 0) return NQS_OK;
    DeviceParams dp;
    if (int rc = prepare_params(c, prec, &dp)) return rc;
    LaunchEnv env = env_of(c);
    if (prec == NQS_FP8)
        return launch_eloc_tc(c->p, c->params, c->packed, configs, nullptr, n, out, nullptr, 0, env, true);
    if (prec == NQS_BF16) {
        const size_t cb = tc_eloc_cache_bytes(c->p, c->max_smem, sms_of(c), n);
        if (cb > 0)
            if (int rc = ensure_scratch(c, cb)) return rc;
        return launch_eloc_tc(c->p, c->params, c->packed, configs, logpsi, n, out, c->scratch, c->scratch_bytes, env);
    }
    return launch_eloc_plain(c->p, prec, dp, configs, logpsi, n, out, env);
}

int nqs_sample(nqs_ctx *c, int32_t n_chains, int32_t spc, int32_t sweeps_between, int32_t burn_in, int8_t *configs_out,
               double *logpsi_out, int32_t prec) {
    NvtxRange nvtx_range("nqs_sample");
    if (int rc = check_ctx(c)) return rc;
    if (n_chains <= 0 || spc < 0 || sweeps_between < 1 || burn_in < 0)
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_sample: bad counts");
    if (spc > 0 && (!configs_out || !logpsi_out)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sample: bad arrays");
    if (!valid_precision(prec)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sample: bad precision");
    LaunchEnv env = env_of(c);
    if (n_chains != c->n_chains || !c->chains) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
        cudaFree(c->chains);
        c->chains = nullptr;
        c->n_chains = 0;
        e = cudaMalloc(&c->chains, (size_t)n_chains * c->p.N);
        if (e != cudaSuccess) return cuda_fail(c, e, "chain allocation");
        if (int rc = launch_init_chains(c->p, c->seed, n_chains, c->chains, env)) return rc;
        c->n_chains = n_chains;
        c->step = 0;
    }
    DeviceParams dp;
    if (int rc = prepare_params(c, prec, &dp)) return rc;
    int rc;
    if (prec == NQS_BF16)
        rc = launch_sample_tc(c->p, c->params, c->packed, c->chains, n_chains, c->step, c->seed, spc, sweeps_between,
                              burn_in, configs_out, logpsi_out, env);
    else
        rc = launch_sample_plain(c->p, prec, dp, c->chains, n_chains, c->step, c->seed, spc, sweeps_between, burn_in,
                                 configs_out, logpsi_out, env);
    if (rc) return rc;
    c->step += (uint64_t)(burn_in + (int64_t)spc * sweeps_between) * c->p.N;
    return NQS_OK;
}

int nqs_get_chains(nqs_ctx *c, int32_t n_chains, int8_t *chains, uint64_t *step) {
    if (int rc = check_ctx(c)) return rc;
    if (n_chains != c->n_chains || !c->chains || !chains || !step)
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_get_chains: no chains of that size");
    cudaError_t e = cudaMemcpyAsync(chains, c->chains, (size_t)n_chains * c->p.N, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "chain copy");
    *step = c->step;
    return NQS_OK;
}

int nqs_set_chains(nqs_ctx *c, int32_t n_chains, const int8_t *chains, uint64_t step) {
    if (int rc = check_ctx(c)) return rc;
    if (n_chains <= 0 || !chains) return fail(c, NQS_ERR_INVALID_ARG, "nqs_set_chains: bad arguments");
    if (n_chains != c->n_chains) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
        cudaFree(c->chains);
        c->chains = nullptr;
        c->n_chains = 0;
        e = cudaMalloc(&c->chains, (size_t)n_chains * c->p.N);
        if (e != cudaSuccess) return cuda_fail(c, e, "chain allocation");
        c->n_chains = n_chains;
    }
    cudaError_t e = cudaMemcpyAsync(c->chains, chains, (size_t)n_chains * c->p.N, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "chain copy");
    c->step = step;
    return NQS_OK;
}

int nqs_logpsi_grad(nqs_ctx *c, const int8_t *configs, int64_t n, double *O, int32_t prec) {
    NvtxRange nvtx_range("nqs_logpsi_grad");
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || (n > 0 && (!configs || !O))) return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi_grad: bad arrays");
    if (!valid_precision(prec)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi_grad: bad precision");
    if (n == 0) return NQS_OK;
    // the tensor-core precision differentiates with float32 internals
    const int gp = prec == NQS_FP64 ? NQS_FP64 : NQS_FP32;
    DeviceParams dp;
    if (int rc = prepare_params(c, gp, &dp)) return rc;
    if (gp == NQS_FP32 && grad_fast_supported(c->p, c->max_smem)) {
        const int fb = (int)std::min<int64_t>(n, (int64_t)sms_of(c) * grad_fast_blocks_per_sm(c->p));
        if (int rc = ensure_scratch(c, grad_fast_scratch_bytes(c->p, fb))) return rc;
        LaunchEnv env = env_of(c);
        return launch_grad_fast(c->p, c->params32, c->params, configs, n, O, c->scratch, c->scratch_bytes, env);
    }
    const int blocks = (int)std::min<int64_t>(n, (int64_t)sms_of(c) * 2);
    if (int rc = ensure_scratch(c, grad_scratch_bytes(c->p, gp, blocks))) return rc;
    LaunchEnv env = env_of(c);
    return launch_grad_plain(c->p, gp, dp, configs, n, O, c->scratch, c->scratch_bytes, env);
}

int nqs_logpsi_vjp(nqs_ctx *c, const int8_t *configs, int64_t n, const double *grad_logpsi, double *grad_params,
                   int32_t prec) {
    NvtxRange nvtx_range("nqs_logpsi_vjp");
    if (int rc = check_ctx(c)) return rc;
    if (n < 0 || !grad_params || (n > 0 && (!configs || !grad_logpsi)))
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi_vjp: bad arrays");
    if (!valid_precision(prec)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_logpsi_vjp: bad precision");
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(grad_params, 0, sizeof(double) * (size_t)c->p.P, c->stream);
        return e == cudaSuccess ? NQS_OK : cuda_fail(c, e, "nqs_logpsi_vjp: clear");
    }
    // float32 internals for the tensor-core precision, as nqs_logpsi_grad
    const int gp = prec == NQS_FP64 ? NQS_FP64 : NQS_FP32;
    DeviceParams dp;
    if (int rc = prepare_params(c, gp, &dp)) return rc;
    const int64_t K = vjp_chunk_samples(n), nq = (n + K - 1) / K;
    const size_t part_bytes = ((size_t)nq * c->p.P * sizeof(double) + 255) & ~(size_t)255;
    const bool fast = gp == NQS_FP32 && grad_fast_supported(c->p, c->max_smem);
    const int blocks = (int)std::min<int64_t>(nq, (int64_t)sms_of(c) * (fast ? grad_fast_blocks_per_sm(c->p) : 2));
    const size_t work = fast ? grad_fast_scratch_bytes(c->p, blocks) : grad_scratch_bytes(c->p, gp, blocks);
    if (int rc = ensure_scratch(c, part_bytes + work)) return rc;
    LaunchEnv env = env_of(c);
    double *part = (double *)c->scratch;
    void *ws = (unsigned char *)c->scratch + part_bytes;
    const size_t ws_bytes = c->scratch_bytes - part_bytes;
    int rc = fast ? launch_vjp_fast(c->p, c->params32, c->params, configs, n, grad_logpsi, part, ws, ws_bytes, env)
                  : launch_vjp_plain(c->p, gp, dp, configs, n, grad_logpsi, part, ws, ws_bytes, env);
    if (rc) return rc;
    return launch_vjp_reduce(c->p, part, n, grad_params, env);
}

int nqs_sr_solve(nqs_ctx *c, const double *O, const double *eloc, int64_t n, double eps, double rtol,
                 int32_t max_iter, double lr, double *delta, int32_t *iters_out, double *resid_out,
                 double *energy_out, int32_t apply_update) {
    NvtxRange nvtx_range("nqs_sr_solve");
    if (int rc = check_ctx(c)) return rc;
    if (n <= 0 || !O || !eloc || !delta) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve: bad arrays");
    if (!(eps >= 0.0) || !(rtol >= 0.0) || max_iter < 0) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve: bad eps/rtol/max_iter");
    const int sx_fp64 = c->sx_arith == NQS_SX_FP64;
    if (int rc = ensure_scratch(c, sr_workspace_doubles(n, c->p.P, sx_fp64) * sizeof(double))) return rc;
    LaunchEnv env = env_of(c);
    // the CG's partial sums are split by the device's SM count, not by an SM
    // limit, so the solve's rounding does not depend on the share a context
    // holds (its kernels are short; they do not pin SMs)
    env.num_sms = c->num_sms;
    int iters = c->cg_hint;
    double resid = 0.0, energy[2] = {0.0, 0.0};
    const int rc = run_sr_solve(c->p, O, eloc, n, eps, rtol, max_iter, lr, delta, c->params, apply_update,
                                (double *)c->scratch, &iters, &resid, energy, sx_fp64, env);
    if (rc == NQS_OK || rc == NQS_ERR_NOT_CONVERGED) c->cg_hint = iters;
    if (iters_out) *iters_out = iters;
    if (resid_out) *resid_out = resid;
    if (energy_out) { energy_out[0] = energy[0]; energy_out[1] = energy[1]; }
    return rc;
}

int nqs_set_sx_arithmetic(nqs_ctx *c, int32_t mode) {
    if (int rc = check_ctx(c)) return rc;
    if (mode != NQS_SX_DOUBLE_FLOAT && mode != NQS_SX_FP64)
        return fail(c, NQS_ERR_INVALID_ARG, "nqs_set_sx_arithmetic: unknown mode");
    c->sx_arith = mode;
    return NQS_OK;
}

int nqs_sr_solve_woodbury(nqs_ctx *c, const double *O, const double *eloc, int64_t n, double eps, double lr,
                          int32_t refine_steps, double *delta, double *resid_out, double *energy_out,
                          int32_t apply_update) {
    NvtxRange nvtx_range("nqs_sr_solve_woodbury");
    if (int rc = check_ctx(c)) return rc;
    if (n <= 0 || !O || !eloc || !delta) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve_woodbury: bad arrays");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve_woodbury: eps must be > 0");
    if (n > kWoodburyMaxSamples) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve_woodbury: n_s above the limit");
    if (refine_steps < 0 || refine_steps > 8) return fail(c, NQS_ERR_INVALID_ARG, "nqs_sr_solve_woodbury: refine_steps not in 0..8");
    if (int rc = ensure_scratch(c, sr_woodbury_workspace_doubles(n, c->p.P) * sizeof(double))) return rc;
    LaunchEnv env = env_of(c);
    env.num_sms = c->num_sms;
    double resid = 0.0, energy[2] = {0.0, 0.0};
    const int rc = run_sr_woodbury(c->p, O, eloc, n, eps, lr, refine_steps, delta, c->params, apply_update,
                                   (double *)c->scratch, &resid, energy, env);
    if (resid_out) *resid_out = resid;
    if (energy_out) { energy_out[0] = energy[0]; energy_out[1] = energy[1]; }
    return rc;
}

}  // extern "C"
