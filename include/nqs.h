/*
 * nqs.h - C ABI of the GB300 (sm_103a) library for the hot path of
 * CNN-wavefunction variational Monte Carlo (arXiv 2204.07816).
 *
 * The library evaluates, for a convolutional wave function
 * W(S) = exp(a(S) + i phi(S)) (Eq. 1 of the paper), the quantities of one
 * stochastic-reconfiguration step of the self-learning procedure (Sec. 3.2):
 * MCMC samples drawn from |W(S)|^2, local energies E_loc (Sec. 5.4.1,
 * "Hotspot energy calculation"), local derivatives O_loc = d log W / d theta,
 * and the SR solve and parameter update (Sec. 5.4.1, "Distributed SR
 * computation"). Hamiltonians: J1-J2 (Eq. 2) and t-J (Eq. 3) on an L x L
 * periodic square lattice.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Sites: (x, y), 0 <= x, y < L, index y*L + x. N = L*L.
 * - Site values (int8): J1-J2 +1 = up, -1 = down; t-J 0 = hole, +1 = up,
 *   -1 = down.
 * - Network: n_layers x [3x3 periodic convolution + bias, SiLU], input one
 *   channel (the site value) for J1-J2 and three one-hot channels
 *   (hole, up, down) for t-J; head a = w_a . sum_sites h, phi = w_phi . sum_sites h.
 * - Parameters: one float64 vector, per layer W[C_out][C_in][3][3] then
 *   b[C_out], then w_a[C], w_phi[C]. Its length is nqs_param_count().
 * - log psi arrays are [n][2] float64 rows (a, phi); local energies are
 *   [n][2] float64 rows (Re E_loc, Im E_loc).
 * - Every array argument is a DEVICE pointer owned by the caller, unless a
 *   comment says otherwise. The library owns the context, the Markov chain
 *   state, the Philox counters and its workspace.
 * - Every call is enqueued on the stream given to nqs_init and returns once
 *   the work is enqueued; the outputs are valid after the stream has
 *   reached that point (nqs_sync waits for it). Argument errors are
 *   returned at once. Errors that the GPU finds (a non-finite value, a wait
 *   that ran out of iterations, a failed index check of the checked build)
 *   are latched in the context and returned by the next nqs_sync.
 * - Return values: NQS_OK or a negative nqs_status. On error the outputs
 *   are unspecified and the chain state is unchanged. nqs_last_error gives
 *   a one-line description.
 * - Precisions: NQS_FP64 and NQS_FP32 run the convolutions on CUDA cores in
 *   that type; NQS_BF16 runs them on the tcgen05 tensor cores with bf16
 *   operands and fp32 accumulation in tensor memory. NQS_FP8 (accepted by
 *   nqs_local_energy only; the other entry points return
 *   NQS_ERR_INVALID_ARG for it) keeps layer 0 in bf16 and runs layers >= 1
 *   with e4m3 operands (the FP8 form of Sec. 5.4.1's convolutions: the
 *   activations saturated to +-448, the weights scaled per output channel
 *   by their largest magnitude / 448, the scale applied to the fp32
 *   accumulator), 16-channel networks on lattices whose row-form plan fits
 *   (nqs_tc_plan reports row_form = 1), else NQS_ERR_UNSUPPORTED. In every
 *   precision the log-amplitude ratios, E_loc, energies and the SR solve
 *   are float64.
 */
#ifndef NQS_H
#define NQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nqs_ctx nqs_ctx;

typedef enum {
    NQS_OK = 0,
    NQS_ERR_INVALID_ARG = -1,
    NQS_ERR_OOM = -2,
    NQS_ERR_CUDA = -3,
    NQS_ERR_NONFINITE = -4,
    NQS_ERR_NOT_CONVERGED = -5,
    NQS_ERR_TIMEOUT = -6,
    NQS_ERR_UNSUPPORTED = -7,
    NQS_ERR_BOUNDS = -8
} nqs_status;

typedef enum { NQS_FP64 = 0, NQS_FP32 = 1, NQS_BF16 = 2, NQS_FP8 = 3 } nqs_precision;

typedef enum { NQS_MODEL_J1J2 = 0, NQS_MODEL_TJ = 1 } nqs_model;

/* Network family. NQS_NET_SILU: the SiLU convolution stack described at the
 * top of this file (every precision). NQS_NET_CNN1 / NQS_NET_CNN2: the
 * paper's two families (Sec. 5.2, "Neural network innovations"), in the
 * reading below; NQS_FP64 and NQS_FP32 only (NQS_BF16 returns
 * NQS_ERR_UNSUPPORTED).
 *   CNN1 (n_layers building blocks; N must be even): U = periodic 3x3
 *     convolution (cross-correlation) + beta; 1-D max-pooling of window 2,
 *     stride 2 over the row-major site order; transposed 1-D convolution of
 *     kernel 2, stride 2 + gamma. Input channels as the SiLU family. The last
 *     block's transposed convolution has one output channel.
 *   CNN2: an embedding E[state][C] of the site values (J1-J2: down 0, up 1;
 *     t-J: hole 0, up 1, down 2), then n_layers blocks of periodic 3x3
 *     convolution + beta, 1-D max-pooling of window 2, stride 1 (the first
 *     site copied to the end), transposed 1-D convolution of kernel 2,
 *     stride 1 (periodic) + gamma; a final periodic 3x3 convolution to one
 *     channel + beta_f.
 *   Both: W(S) = product of the N output neurons z_s, so a = sum log|z_s|
 *   and phi = pi (number of negative z_s mod 2); max-pooling ties go to the
 *   window's first element; local derivatives are real (d phi = 0).
 *   Parameter layout: CNN1 per block W[C][C_b][3][3], beta[C], T[C][C_o][2],
 *   gamma[C_o] (C_b = c_in for the first block, else C; C_o = 1 for the last,
 *   else C); CNN2 E[n_states][C], per block W[C][C][3][3], beta[C],
 *   T[C][C][2], gamma[C], then W_f[1][C][3][3], beta_f[1]. */
typedef enum { NQS_NET_SILU = 0, NQS_NET_CNN1 = 1, NQS_NET_CNN2 = 2 } nqs_net;

/* The physical problem and the network shape. Eq. 2 uses J1, J2 and
 * sign_rule; Eq. 3 uses t and J. n_up / n_down fix the sector the sampler
 * draws from (J1-J2: n_up + n_down = N; t-J: holes = N - n_up - n_down).
 * sign_rule (J1-J2 only, 0 or 1) multiplies the basis by
 * (-1)^(up spins on the (x+y)-even sublattice), which flips the sign of the
 * nearest-neighbour exchange elements. */
typedef struct {
    int32_t model;      /* nqs_model */
    int32_t L;          /* 4 <= L <= 36 */
    double J1, J2;      /* J1-J2 couplings */
    double t, J;        /* t-J couplings */
    int32_t n_up, n_down;
    int32_t sign_rule;
    int32_t n_layers;   /* >= 1 (CNN1 / CNN2: building blocks) */
    int32_t channels;   /* 4, 8, 16 or 32 */
    int32_t net;        /* nqs_net */
} nqs_problem;

/* Number of network parameters for problem p (layout above); -1 if p is
 * invalid. Host only, no GPU work. */
int64_t nqs_param_count(const nqs_problem *p);

/* The tensor-core (bf16) plan that the library's launchers choose for
 * problem p on a device with num_sms SMs and max_smem_per_block bytes of
 * opt-in shared memory per block (host only, no GPU work; the launchers use
 * the same code with the current device's values). kind: 0 = nqs_logpsi,
 * 1 = nqs_local_energy (n = samples), 2 = nqs_sample (n = chains).
 * out: host int32 [9] = configurations per group (G), groups in flight per
 * block, blocks per SM the plan is sized for, epilogue warps, 128-row tiles
 * per group, shared-memory bytes per block, tensor-memory columns per block,
 * grid size, form (0: one MMA per 3x3 tap and 128-row tile of padded
 * positions; 1: the local energy's row form, rows = (lattice row,
 * configuration) and x positions along tensor-memory columns). Returns NQS_ERR_INVALID_ARG for a bad problem or argument,
 * NQS_ERR_UNSUPPORTED if the tensor-core path cannot run p (channels other
 * than 16 or 32, or no plan fits). */
int nqs_tc_plan(const nqs_problem *p, int32_t kind, int64_t n, int32_t max_smem_per_block, int32_t num_sms,
                int32_t *out);

/* Create a context on the current CUDA device.
 * params: device float64 [nqs_param_count(p)], caller-owned and borrowed
 *   for the life of the context; the library reads it at every call (so
 *   the caller may change it between calls) and nqs_sr_solve with
 *   apply_update = 1 writes it in place.
 * seed: Philox key for the sampler (Sec. 3.2 MCMC): proposals use key
 *   (seed, 0), initial chain states key (seed, 1).
 * stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 * Returns NQS_ERR_INVALID_ARG for a bad problem, NQS_ERR_CUDA if no
 * sm_100-family device is current. */
int nqs_init(nqs_ctx **out, const nqs_problem *p, double *params, uint64_t seed, void *stream);

/* Waits for the context's stream and frees every resource. Returns the
 * latched device error, if any. */
int nqs_destroy(nqs_ctx *ctx);

/* One-line description of the last error of this context (static string if
 * ctx is NULL). Host memory owned by the library. */
const char *nqs_last_error(const nqs_ctx *ctx);

/* Wait for the context's stream; return and clear the latched device error. */
int nqs_sync(nqs_ctx *ctx);

/* Sampler statistics of this context since its creation or the last reset
 * (waits for the context's stream): moves = proposals whose two sites hold
 * different values (the others leave the configuration unchanged and count
 * as rejected steps, Sec. 3.2 reading of the exchange proposal), accepted =
 * moves accepted by the Metropolis test. The acceptance rate per proposal is
 * accepted / (chains x sweeps x N). Host int64 outputs (either may be NULL);
 * reset != 0 zeroes the counters after reading. */
int nqs_sampler_counts(nqs_ctx *ctx, int64_t *moves, int64_t *accepted, int32_t reset);

/* Size every later launch of this context for `sms` SMs instead of the
 * whole device (0 = whole device, the default; 1 .. SM count), so that
 * contexts running side by side on their own streams (a serving mix) keep
 * to disjoint shares of the GPU: grid sizes, chains per sampler block and
 * the E_loc cache follow the limit. Host only; NQS_ERR_INVALID_ARG if sms
 * is out of range. */
int nqs_set_sm_limit(nqs_ctx *ctx, int32_t sms);

/* Failure-path check of the device-side waits. Enqueues on the context's
 * stream a one-warp kernel that waits, through the same bounded wait loop
 * as the tensor-core kernels (limited here to `iterations` polls), on an
 * mbarrier phase that nothing completes. When the limit runs out the kernel
 * sets the timeout bit and exits; the next nqs_sync returns
 * NQS_ERR_TIMEOUT and clears it, and the context stays usable. No GPU fault
 * or hang is involved. iterations: 1 .. 1e6 (else NQS_ERR_INVALID_ARG). */
int nqs_probe_wait_timeout(nqs_ctx *ctx, int64_t iterations);

/* Device-side index checks. A library built with NQS_CHECK defined (see
 * paper_2204_07816_gb300/build.py, checked=True) tests every data-dependent
 * index of its kernels (sampled sites, connected pairs, table entries, row
 * destinations) before the access; an index out of range skips the access
 * and sets the bounds bit, which the next nqs_sync returns as
 * NQS_ERR_BOUNDS (then clears). In the default build the checks compile
 * away. nqs_probe_bounds enqueues a one-thread kernel that reports a failed
 * check without any access, so the reporting path is tested in either build;
 * the context stays usable. */
int nqs_probe_bounds(nqs_ctx *ctx);

/* Number of GPU kernels this context has launched so far (a monotone
 * counter for accounting; -1 if ctx is NULL). Host only. */
int64_t nqs_kernel_launches(const nqs_ctx *ctx);

/* log psi of n configurations (Eq. 1: the network's log-amplitude and
 * phase). configs: device int8 [n][N]; logpsi_out: device float64 [n][2]. */
int nqs_logpsi(nqs_ctx *ctx, const int8_t *configs, int64_t n, double *logpsi_out, int32_t precision);

/* Connected configurations (Sec. 5.4.1 "sprime_batch"; matrix elements of
 * Eq. 2 or Eq. 3). For sample s, the bonds that change configs[s] are
 * listed in bond order: site-major, then direction (x+1), (y+1), and for
 * J1-J2 also (x+1, y+1), (x+1, y-1). Entry k of sample s:
 *   pairs_out[s][k] = (i, j) (int32 x2), the swapped sites,
 *   h_out[s][k]     = <S|H|S'> (float64),
 * n_conn_out[s] = number of entries, hdiag_out[s] = <S|H|S> (float64).
 * Every output array is a device array sized for max_conn entries per
 * sample (max_conn >= 4N for J1-J2, >= 2N for t-J). Integer outputs and the
 * off-diagonal values are exact. */
int nqs_connected(nqs_ctx *ctx, const int8_t *configs, int64_t n, int32_t max_conn,
                  int32_t *n_conn_out, int32_t *pairs_out, double *h_out, double *hdiag_out);

/* Local energies (Sec. 5.4.1: E_loc(S) = sum_S' W(S')/W(S) <S'|H|S>):
 * eloc_out[s] = H_SS + sum_k H_k exp((a'_k - a) + i (phi'_k - phi)).
 * configs: device int8 [n][N]. logpsi: device float64 [n][2] giving
 * (a, phi) of each configuration, or NULL to have the library recompute it
 * with the same precision as the connected configurations (recommended for
 * NQS_BF16, so that the rounding of numerator and denominator matches;
 * with NQS_FP8 it is always recomputed and logpsi is not read).
 * eloc_out: device float64 [n][2]. */
int nqs_local_energy(nqs_ctx *ctx, const int8_t *configs, const double *logpsi, int64_t n,
                     double *eloc_out, int32_t precision);

/* Local energies of several independent problems in one pass (the
 * batched, fixed-length forward of Sec. 5.4.1 "Thread-level parallel
 * MCMC", extended across problems of different lattice sizes and
 * Hamiltonians). Entry i evaluates what nqs_local_energy(ctxs[i],
 * configs[i], logpsi ? logpsi[i] : NULL, n[i], eloc_out[i], precision)
 * evaluates, with bitwise the same results. With NQS_BF16 the problems that
 * share a channel count run in one tensor-core launch whose blocks move from
 * problem to problem; the CUDA-core precisions run one launch per problem.
 * All work is enqueued on the stream of ctxs[0], which must be on the same
 * device as the others; the caller orders it after the work that produces
 * the inputs (e.g. with events). Host arrays of `count` entries; device
 * arrays as in nqs_local_energy. max_blocks > 0 caps the grid of the
 * grouped launch (so that several grouped launches on different streams can
 * share the SMs); 0 uses every SM. */
int nqs_local_energy_multi(nqs_ctx *const *ctxs, int32_t count, const int8_t *const *configs,
                           const double *const *logpsi, const int64_t *n, double *const *eloc_out,
                           int32_t precision, int32_t max_blocks);

/* Metropolis exchange sampling from |W(S)|^2 (Sec. 3.2; Sec. 5.4.1
 * "Process-level / thread-level parallel MCMC": many independent chains).
 * The context keeps n_chains chains on the device across calls; the first
 * call (or a call with a different n_chains) starts them from Fisher-Yates
 * shuffles of the sector's site values. Proposal number s of chain c uses
 * Philox4x64-10 block (c, s, 0, 0) under key (seed, 0): site
 * i = floor(B0 N / 2^64), neighbour direction B1 >> 62 (x+1, x-1, y+1, y-1),
 * u = (B2 >> 11) 2^-53; it swaps i and j when their values differ and is
 * accepted iff 2(a' - a) >= 0 or u < exp(2(a' - a)). burn_in sweeps of N
 * proposals are discarded, then a sample is kept after every
 * sweeps_between-th sweep. configs_out: device int8
 * [n_chains * samples_per_chain][N], chain-major; logpsi_out: device
 * float64 [same][2]. */
int nqs_sample(nqs_ctx *ctx, int32_t n_chains, int32_t samples_per_chain, int32_t sweeps_between,
               int32_t burn_in, int8_t *configs_out, double *logpsi_out, int32_t precision);

/* Chain checkpoint / resume. chains: device int8 [n_chains][N]; step: host
 * uint64, the number of proposals every chain has made. get copies the
 * current state out (n_chains must match the context's); set replaces it
 * (the log-amplitudes are recomputed at the next nqs_sample). */
int nqs_get_chains(nqs_ctx *ctx, int32_t n_chains, int8_t *chains, uint64_t *step);
int nqs_set_chains(nqs_ctx *ctx, int32_t n_chains, const int8_t *chains, uint64_t step);

/* Local derivatives O_loc (Sec. 3.2: the backward of the network gives
 * O_loc), real-stacked: O_out is device float64 [2n][P] with row s equal to
 * d a(S_s)/d theta and row n + s equal to d phi(S_s)/d theta, so that
 * O_k = row s + i * row (n + s). */
int nqs_logpsi_grad(nqs_ctx *ctx, const int8_t *configs, int64_t n, double *O_out, int32_t precision);

/* Vector-Jacobian product of log psi (the backward of Sec. 3.2 seeded by
 * the caller): grad_params[k] = sum_s (grad_logpsi[s][0] d a(S_s)/d theta_k
 * + grad_logpsi[s][1] d phi(S_s)/d theta_k), for n configurations (device
 * int8 [n][N]) and output gradients grad_logpsi (device float64 [n][2]);
 * grad_params: device float64 [P]. One backward pass per sample, seeded with
 * g_a w_a + g_phi w_phi, is summed into per-chunk partials (chunks of
 * consecutive samples whose size depends on n only, samples in order) that
 * are added in chunk order, so the result does not depend on the device or
 * the grid; no [2n][P] matrix is formed. Precisions as nqs_logpsi_grad
 * (NQS_BF16 differentiates with float32 internals). n = 0 writes zeros. */
int nqs_logpsi_vjp(nqs_ctx *ctx, const int8_t *configs, int64_t n, const double *grad_logpsi, double *grad_params,
                   int32_t precision);

/* Local derivatives without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (code that runs where allocating is not allowed, such as an
 * application that owns all device memory through its own allocator, or a
 * framework that forbids allocations from libraries while it records work),
 * and that therefore cannot create an nqs_ctx either.
 * It runs the kernels nqs_logpsi_grad runs for the same precision
 * (NQS_FP64: the float64 backward; NQS_FP32 and NQS_BF16: the float32
 * shared-memory backward for 16 or 32 channels, else the plain float32
 * one), so O_out (device float64 [2n][P], real-stacked as there) is
 * bitwise the same, for the problem p, the device float64 parameters
 * `params` and the device int8 configurations [n][N], enqueued on `stream`
 * (cudaStream_t, NULL = legacy default stream) of the current device. Its
 * grid holds only as many blocks as have working arrays in the fixed array,
 * so large problems run on fewer SMs, and slower, than nqs_logpsi_grad.
 * Working memory: one fixed device array of 8 MiB that the library defines
 * at file scope (every GPU that loads the library holds it until the
 * process exits). The call rejects, with NQS_ERR_UNSUPPORTED, problems
 * whose per-block working arrays (plus a float32 copy of the parameters
 * for NQS_FP32 / NQS_BF16) do not fit in it, and devices with an ordinal of
 * 64 or more. All calls share the array and
 * it keeps the last call's contents; calls that overlap on the same GPU
 * (issued on two streams, or from two host threads) race on it, so the
 * caller must serialise them. Each GPU has its own copy of the array.
 * The first call on a device looks up the array's device address once
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Returns NQS_OK or a negative nqs_status; nqs_noalloc_last_error gives a
 * one-line description of the last failure of the calling host thread. */
int nqs_logpsi_grad_noalloc(const nqs_problem *p, const double *params, const int8_t *configs, int64_t n,
                            double *O_out, int32_t precision, void *stream);
const char *nqs_noalloc_last_error(void);

/* Arithmetic of the S.x products inside nqs_sr_solve's conjugate gradient.
 * NQS_SX_DOUBLE_FLOAT (the default): the pass that computes the force also
 * splits every float64 element of O into a float high part and a float low
 * part (|error| < 2^-46 of the element; exact when the element is a float,
 * as the NQS_FP32 and NQS_BF16 derivatives are), and each iteration's two
 * passes over O multiply-add in double-float arithmetic (pairs of floats,
 * renormalised sums, about 1e-15 of the sum of the terms' magnitudes) on the
 * float32 pipes, reading only the high plane when every low part is zero.
 * The force, every vector and scalar of the iteration and every row or
 * column total stay float64. Needs 8 bytes per element of O more working
 * memory (the two planes). Its values must stay in the float range: an
 * element of O of magnitude 2^128 or more, or a product or partial sum
 * beyond about 3.4e38, ends the solve with NQS_ERR_NONFINITE (parameters
 * unchanged), and elements below 2^-80 count as zero. NQS_SX_FP64: both
 * passes in float64 FMAs on the float64 O itself (float64 range; GB300's
 * float64 FMA rate bounds them). */
typedef enum { NQS_SX_DOUBLE_FLOAT = 0, NQS_SX_FP64 = 1 } nqs_sx_arithmetic;

/* Select the S.x arithmetic of ctx's later nqs_sr_solve calls. Returns
 * NQS_OK, or NQS_ERR_INVALID_ARG for another mode. */
int nqs_set_sx_arithmetic(nqs_ctx *ctx, int32_t mode);

/* Stochastic reconfiguration (Sec. 3.2; Sec. 5.4.1 "Distributed SR
 * computation", solved here matrix-free by conjugate gradient):
 *   <E> = mean E_loc, Oc = O - mean O,
 *   S = Re(Oc^H Oc)/n, F = Re(Oc^H (E_loc - <E>))/n,
 *   (S + eps I) delta = F by CG from delta = 0 until ||r|| <= rtol ||F||
 *   or max_iter iterations, then theta <- theta - lr delta if apply_update.
 * O: device float64 [2n][P] as written by nqs_logpsi_grad; eloc: device
 * float64 [n][2]; delta_out: device float64 [P]. iters_out, resid_out
 * (relative residual) and energy_out ([2]: Re, Im of <E>) are HOST
 * pointers, written before the call returns (the call waits for the
 * stream). Returns NQS_ERR_NOT_CONVERGED (delta and the update still
 * applied) when max_iter is reached first, and NQS_ERR_NONFINITE when the
 * force, the residual or the energy is not finite (a NaN or Inf in O or
 * eloc); the parameters are then left unchanged even if apply_update is
 * set. */
int nqs_sr_solve(nqs_ctx *ctx, const double *O, const double *eloc, int64_t n, double eps, double rtol,
                 int32_t max_iter, double lr, double *delta_out, int32_t *iters_out, double *resid_out,
                 double *energy_out, int32_t apply_update);

/* The same delta from the sample-space system (the paper forms a
 * covariance matrix and factorises it, Sec. 5.4.1; here the 2n x 2n one):
 *   Ohat = [Re Oc; Im Oc] ([2n][P]), Ehat = [Re(E - <E>); Im(E - <E>)],
 *   (Ohat Ohat^T / n + eps I) y = Ehat / n   (Cholesky, FP64),
 *   delta = Ohat^T y,
 * equal to the solution of (S + eps I) delta = F because
 * (Ohat^T Ohat / n + eps I)^-1 Ohat^T = Ohat^T (Ohat Ohat^T / n + eps I)^-1.
 * Work: 2 n^2 P (Gram matrix, lower half) + (2n)^3 / 6 (Cholesky)
 * multiply-adds, against 4 n P per CG iteration, so it pays when CG needs
 * more than about n / 2 iterations.
 * Arguments as nqs_sr_solve; eps must be > 0 and n <= 32,768 (workspace
 * (2n)^2 float64, owned by the context). refine_steps (0..8): steps of
 * iterative refinement, each recomputing the sample-space residual
 * Ehat / n - (Ohat Ohat^T / n + eps I) y from O (two passes over O) and
 * solving for the correction with the same factor. resid_out (HOST)
 * receives ||(S + eps I) delta - F|| / ||F||, evaluated matrix-free after
 * the solve. Returns NQS_ERR_NONFINITE if a pivot was not positive or a
 * value is not finite; the update is then not applied. */
int nqs_sr_solve_woodbury(nqs_ctx *ctx, const double *O, const double *eloc, int64_t n, double eps, double lr,
                          int32_t refine_steps, double *delta_out, double *resid_out, double *energy_out,
                          int32_t apply_update);

#ifdef __cplusplus
}
#endif

#endif /* NQS_H */
