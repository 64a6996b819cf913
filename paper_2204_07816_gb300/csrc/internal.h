// Host-side interface between the C ABI (abi.cu) and the kernel files.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "common.cuh"

namespace nqs {

struct LaunchEnv {
    cudaStream_t stream;
    int num_sms;
    bool sm_limited = false;   // num_sms is the context's SM share (nqs_set_sm_limit): grids stay within it
    size_t max_smem;     // opt-in shared memory per block
    int *err;            // device error bits
    unsigned long long *moves = nullptr;   // sampler counters [2]: moves that change the state, accepted moves
    int64_t *launches;   // kernels launched so far by this context
    std::string *msg;    // host error text
};

// Let a kernel use all the dynamic shared memory the device allows it (the opt-in maximum less the kernel's
// static shared memory). The limit is a per-function attribute shared by every host thread, so it is set to this
// fixed value and never to one launch's size: a context on another thread launching the same kernel with a
// smaller size cannot lower it below this launch's need. need: this launch's dynamic bytes.
template <typename K>
inline int allow_dynamic_smem(K kernel, size_t need, const LaunchEnv &env) {
    cudaFuncAttributes a{};
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e == cudaSuccess) {
        const size_t cap = env.max_smem > a.sharedSizeBytes ? env.max_smem - a.sharedSizeBytes : 0;
        if (need > cap) {
            *env.msg = "launch needs " + std::to_string(need) + " bytes of dynamic shared memory (max " +
                       std::to_string(cap) + ")";
            return NQS_ERR_UNSUPPORTED;
        }
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    }
    if (e != cudaSuccess) {
        *env.msg = std::string("kernel shared-memory attribute: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

// Parameters converted for a precision: T = float copies of the layer
// weights (FP32 path) or the packed bf16 operand images (tensor-core path).
struct DeviceParams {
    const double *p64;    // caller's float64 vector
    const float *p32;     // float copy (same layout)
};

// ---- plain CUDA-core path (plain.cu); prec = NQS_FP64 or NQS_FP32
int plain_max_group(const Problem &p, int prec, size_t extra_smem, size_t max_smem);
int launch_logpsi_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                        double *out, const LaunchEnv &env);
int launch_eloc_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs,
                      const double *logpsi, int64_t n, double *out, const LaunchEnv &env);
int launch_connected(const Problem &p, const int8_t *configs, int64_t n, int max_conn, int32_t *n_conn,
                     int32_t *pairs, double *h, double *hdiag, const LaunchEnv &env);
int launch_init_chains(const Problem &p, uint64_t seed, int n_chains, int8_t *chains, const LaunchEnv &env);
int launch_sample_plain(const Problem &p, int prec, const DeviceParams &dp, int8_t *chains, int n_chains,
                        uint64_t step0, uint64_t seed, int spc, int sweeps_between, int burn_in, int8_t *out_cfg,
                        double *out_logpsi, const LaunchEnv &env);
int launch_grad_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                      double *O, void *scratch, size_t scratch_bytes, const LaunchEnv &env);
size_t grad_scratch_bytes(const Problem &p, int prec, int num_blocks);
// float32-internal backward with shared-memory working sets (grad.cu)
bool grad_fast_supported(const Problem &p, size_t max_smem);
int grad_fast_blocks_per_sm(const Problem &p);
size_t grad_fast_scratch_bytes(const Problem &p, int num_blocks);
int launch_grad_fast(const Problem &p, const float *p32, const double *p64, const int8_t *configs, int64_t n,
                     double *O, void *scratch, size_t scratch_bytes, const LaunchEnv &env);
void launch_convert_params(const double *p64, float *p32, int P, cudaStream_t s);
// vector-Jacobian products sum_s (g_a d a_s / d theta + g_phi d phi_s / d theta): per-chunk partials
// part[ceil(n / K)][P] (K = vjp_chunk_samples(n), one block per chunk, samples in order), then
// launch_vjp_reduce sums the chunks in order
int64_t vjp_chunk_samples(int64_t n);
int launch_vjp_fast(const Problem &p, const float *p32, const double *p64, const int8_t *configs, int64_t n,
                    const double *grad, double *part, void *scratch, size_t scratch_bytes, const LaunchEnv &env);
int launch_vjp_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                     const double *grad, double *part, void *scratch, size_t scratch_bytes, const LaunchEnv &env);
int launch_vjp_reduce(const Problem &p, const double *part, int64_t n, double *out, const LaunchEnv &env);

// ---- tensor-core path (tc.cu)
bool tc_supported(const Problem &p, std::string *why);
size_t tc_packed_bytes(const Problem &p);
int launch_tc_pack(const Problem &p, const double *p64, void *packed, const LaunchEnv &env);
int launch_logpsi_tc(const Problem &p, const double *p64, const void *packed, const int8_t *configs, int64_t n,
                     double *out, const LaunchEnv &env);
size_t tc_eloc_cache_bytes(const Problem &p, size_t max_smem, int num_sms, int64_t n);
int launch_eloc_tc(const Problem &p, const double *p64, const void *packed, const int8_t *configs,
                   const double *logpsi, int64_t n, double *out, void *cache, size_t cache_bytes,
                   const LaunchEnv &env, bool f8 = false);
// grouped local energies of several problems with one channel count (tc.cu)
struct TcMultiItem {
    Problem p;
    const void *packed;
    const int8_t *configs;
    const double *logpsi;   // nullable
    int64_t n;
    double *out;
};
size_t tc_multi_table_bytes(int count);
int launch_eloc_tc_multi(const TcMultiItem *items, int count, void *dev_table, int max_blocks, const LaunchEnv &env);
int launch_wait_probe(int64_t iterations, const LaunchEnv &env);
int launch_bounds_probe(const LaunchEnv &env);
// Tensor-core plan the launchers choose (host only): kind 0 log psi, 1 local
// energy, 2 sampler (n = chains). out[9]: G, slots, blocks per SM, epilogue
// warps, tiles per group, shared bytes per block, TMEM columns, grid, form
// (0 tap form, 1 row form).
int tc_describe_plan(const Problem &p, int kind, int64_t n, size_t max_smem, int num_sms, int32_t *out,
                     std::string *why);
int launch_sample_tc(const Problem &p, const double *p64, const void *packed, int8_t *chains, int n_chains,
                     uint64_t step0, uint64_t seed, int spc, int sweeps_between, int burn_in, int8_t *out_cfg,
                     double *out_logpsi, const LaunchEnv &env);

// ---- SR (sr.cu)
struct SrWorkspace {
    double *buf;
    size_t doubles;
};
size_t sr_workspace_doubles(int64_t n, int P, int sx_fp64);
int run_sr_solve(const Problem &p, const double *O, const double *eloc, int64_t n, double eps, double rtol,
                 int max_iter, double lr, double *delta, double *params, int apply, double *workspace,
                 int *iters_out, double *resid_out, double *energy_out, int sx_fp64, const LaunchEnv &env);
// sample-space (Woodbury) form: 2n x 2n Cholesky in place of CG
size_t sr_woodbury_workspace_doubles(int64_t n, int P);
int run_sr_woodbury(const Problem &p, const double *O, const double *eloc, int64_t n, double eps, double lr,
                    int refine_steps, double *delta, double *params, int apply, double *workspace,
                    double *resid_out, double *energy_out, const LaunchEnv &env);

}  // namespace nqs
