// Per-sample local derivatives O_k = d log W / d theta_k (Sec. 3.2: the
// backward of the network gives O_loc) with float32 internals, for the
// FP32 and tensor-core precisions. One block per sample at a time:
//   forward   z_l = conv(h_{l-1}) + b_l, h_l = silu(z_l); h_l and
//             s_l = sigmoid(z_l) go to this block's (L2-resident) scratch
//   head      d a / d w_a = d phi / d w_phi = sum over sites of h_n
//   backward  for l = n_l - 1 .. 0, both outputs (a and phi) at once:
//             gz = g * silu'(z) with silu'(z) = s + h (1 - s)
//             dW[o][c][k] = sum_site gz[o][site] h_{l-1}[c][site + d_k]
//             db[o] = sum_site gz[o][site]
//             g_{l-1}[c][site] = sum_{o,k} W[o][c][k] gz[o][site - d_k]
// Every working array of the current layer lives in shared memory with a
// site stride of N + 1 (odd) so that threads reading different channels hit
// different banks; neighbour indices come from a table built once.
//
// Vector-Jacobian form (VJP = true): given per-sample output gradients
// (g_a, g_phi), one backward stream seeded with g_a w_a + g_phi w_phi gives
// g_a d a / d theta + g_phi d phi / d theta for every parameter, and the
// samples' vectors are summed per chunk of consecutive samples (each chunk
// owned by one block, samples in order) into chunk partials; a second kernel
// sums the partials in chunk order. No per-sample row is stored.
#include <algorithm>

#include "internal.h"

namespace nqs {

namespace {

constexpr int kGradThreads = 256;
// Blocks per SM the kernel is compiled for: four at 16 channels (64 registers,
// no spills; twice the resident warps of the unbounded 108-register build),
// two at 32 channels (more would spill).
template <int C> constexpr int kGradMinBlocks = C == 16 ? 4 : 2;

struct GradLayout {
    int NP;                // padded site stride
    size_t w, nbr, hprev, gz, gnext, hbar, total;
};

__host__ __device__ inline size_t a16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline GradLayout grad_layout(const Problem &p) {
    GradLayout g;
    g.NP = p.N + 1;
    const int cmax = p.C > p.c_in ? p.C : p.c_in;
    size_t o = 0;
    g.w = o; o = a16(o + 4 * (size_t)(9 * p.C * cmax + p.C));
    g.nbr = o; o = a16(o + 2 * (size_t)9 * p.N);
    g.hprev = o; o = a16(o + 4 * (size_t)cmax * g.NP);
    g.gz = o; o = a16(o + 4 * (size_t)2 * p.C * g.NP);
    g.gnext = o; o = a16(o + 4 * (size_t)2 * p.C * g.NP);
    g.hbar = o; o = a16(o + 4 * (size_t)p.C);
    g.total = o;
    return g;
}

// The shared-memory working set of one block.
struct GradSmem {
    float *w, *hprev, *gz, *gnext, *hbar;
    int16_t *nbr;
};

__device__ GradSmem grad_smem(const Problem &p, unsigned char *smem) {
    const GradLayout gl = grad_layout(p);
    GradSmem m;
    m.w = reinterpret_cast<float *>(smem + gl.w);
    m.nbr = reinterpret_cast<int16_t *>(smem + gl.nbr);      // [9][N]: site at (x + dx, y + dy)
    m.hprev = reinterpret_cast<float *>(smem + gl.hprev);    // [cin][NP]
    m.gz = reinterpret_cast<float *>(smem + gl.gz);          // [R][C][NP] (forward: output h)
    m.gnext = reinterpret_cast<float *>(smem + gl.gnext);    // [R][C][NP]
    m.hbar = reinterpret_cast<float *>(smem + gl.hbar);
    const int N = p.N, L = p.L;
    for (int e = threadIdx.x; e < 9 * N; e += blockDim.x) {
        const int k = e / N, s = e - k * N;
        const int x = s % L, y = s / L, dy = k / 3 - 1, dx = k % 3 - 1;
        m.nbr[e] = (int16_t)((((y + dy) % L + L) % L) * L + ((x + dx) % L + L) % L);
    }
    __syncthreads();
    return m;
}

// Backward of one sample. VJP = false: rows Oa = d a / d theta and
// Op = d phi / d theta are written (two streams). VJP = true: one stream
// seeded with ga w_a + gp w_phi, and the sample's vector is added to acc
// (every parameter by the same thread for every sample of the block).
template <int C, bool VJP>
__device__ void grad_sample(const Problem &p, const GradSmem &m, const float *__restrict__ prm,
                            const double *__restrict__ p64, const int8_t *__restrict__ cfg, double *Oa, double *Op,
                            double ga, double gp, double *acc, float *Hs) {
    constexpr int R = VJP ? 1 : 2;
    const int N = p.N, NP = p.N + 1, L = p.L, nl = p.n_layers;
    float *w = m.w, *hprev = m.hprev, *gz = m.gz, *gnext = m.gnext, *hbar = m.hbar;
    const int16_t *nbr = m.nbr;
    float *Ss = Hs + (size_t)nl * C * N;                             // [nl][C][N] sigmoid(z)
    {
        // ---------------- forward
        for (int s = threadIdx.x; s < N; s += blockDim.x) {
            const int v = cfg[s];
            if (p.c_in == 1) hprev[s] = (float)v;
            else { hprev[s] = (float)(v == 0); hprev[NP + s] = (float)(v == 1); hprev[2 * NP + s] = (float)(v == -1); }
        }
        for (int l = 0; l < nl; ++l) {
            const int cin = layer_cin(p, l), off = layer_offset(p, l);
            __syncthreads();
            // stage W as w[(k * cin + c) * C + o], bias after
            for (int e = threadIdx.x; e < 9 * cin * C; e += blockDim.x) {
                const int o = e / (9 * cin), rem = e - o * 9 * cin, c = rem / 9, k = rem - c * 9;
                w[(k * cin + c) * C + o] = prm[off + e];
            }
            for (int e = threadIdx.x; e < C; e += blockDim.x) w[9 * cin * C + e] = prm[off + 9 * cin * C + e];
            __syncthreads();
            float *hout = gz;   // [C][NP]
            // one work item per (site, half of the output channels): twice the threads of one item per
            // site on lattices with 2 N <= 256 sites, the same sums in the same order
            constexpr int CH = C / 2;
            for (int it = threadIdx.x; it < 2 * N; it += blockDim.x) {
                const int half = it >= N, s = it - half * N;
                float acc[CH];
#pragma unroll
                for (int o = 0; o < CH; ++o) acc[o] = w[9 * cin * C + half * CH + o];
                for (int k = 0; k < 9; ++k) {
                    const int sn = nbr[k * N + s];
                    for (int c = 0; c < cin; ++c) {
                        const float hv = hprev[c * NP + sn];
                        const float4 *wr = reinterpret_cast<const float4 *>(w + (k * cin + c) * C + half * CH);
#pragma unroll
                        for (int q = 0; q < CH / 4; ++q) {
                            const float4 wv = wr[q];
                            acc[4 * q] = fmaf(wv.x, hv, acc[4 * q]);
                            acc[4 * q + 1] = fmaf(wv.y, hv, acc[4 * q + 1]);
                            acc[4 * q + 2] = fmaf(wv.z, hv, acc[4 * q + 2]);
                            acc[4 * q + 3] = fmaf(wv.w, hv, acc[4 * q + 3]);
                        }
                    }
                }
                float *Hl = Hs + (size_t)l * C * N, *Sl = Ss + (size_t)l * C * N;
#pragma unroll
                for (int oo = 0; oo < CH; ++oo) {
                    const int o = half * CH + oo;
                    const float sg = 1.0f / (1.0f + expf(-acc[oo]));
                    const float h = acc[oo] * sg;
                    hout[o * NP + s] = h;
                    Hl[o * N + s] = h;
                    Sl[o * N + s] = sg;
                }
            }
            __syncthreads();
            for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
                const int c = e / N, s = e - c * N;
                hprev[c * NP + s] = hout[c * NP + s];
            }
        }
        __syncthreads();
        // ---------------- head
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int c = warp; c < C; c += nw) {
                float v = 0.f;
                for (int s = lane; s < N; s += 32) v += hprev[c * NP + s];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) hbar[c] = v;
            }
        }
        __syncthreads();
        const int ho = head_offset(p);
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            if (VJP) {
                acc[ho + c] += ga * (double)hbar[c];
                acc[ho + C + c] += gp * (double)hbar[c];
            } else {
                Oa[ho + c] = (double)hbar[c];
                Oa[ho + C + c] = 0.0;
                Op[ho + c] = 0.0;
                Op[ho + C + c] = (double)hbar[c];
            }
        }
        for (int e = threadIdx.x; e < R * C * N; e += blockDim.x) {
            const int r = e / (C * N), rem = e - r * C * N, c = rem / N, s = rem - c * N;
            gnext[(r * C + c) * NP + s] =
                VJP ? (float)(ga * p64[ho + c] + gp * p64[ho + C + c]) : (float)p64[ho + r * C + c];
        }
        // ---------------- backward
        for (int l = nl - 1; l >= 0; --l) {
            const int cin = layer_cin(p, l), off = layer_offset(p, l);
            const float *Hl = Hs + (size_t)l * C * N, *Sl = Ss + (size_t)l * C * N;
            __syncthreads();
            for (int e = threadIdx.x; e < R * C * N; e += blockDim.x) {
                const int r = e / (C * N), rem = e - r * C * N, c = rem / N, s = rem - c * N;
                const float h = Hl[c * N + s], sg = Sl[c * N + s];
                gz[(r * C + c) * NP + s] = gnext[(r * C + c) * NP + s] * (sg + h * (1.0f - sg));
            }
            // layer input h_{l-1} and the weights in [o][k][c] order (c contiguous)
            if (l == 0) {
                for (int s = threadIdx.x; s < N; s += blockDim.x) {
                    const int v = cfg[s];
                    if (p.c_in == 1) hprev[s] = (float)v;
                    else { hprev[s] = (float)(v == 0); hprev[NP + s] = (float)(v == 1); hprev[2 * NP + s] = (float)(v == -1); }
                }
            } else {
                const float *Hp = Hs + (size_t)(l - 1) * C * N;
                for (int e = threadIdx.x; e < C * N; e += blockDim.x) {
                    const int c = e / N, s = e - c * N;
                    hprev[c * NP + s] = Hp[e];
                }
            }
            for (int e = threadIdx.x; e < 9 * cin * C; e += blockDim.x) {
                const int o = e / (9 * cin), rem = e - o * 9 * cin, c = rem / 9, k = rem - c * 9;
                w[(o * 9 + k) * cin + c] = prm[off + e];
            }
            __syncthreads();
            // weight and bias gradients, both outputs
            for (int pc = threadIdx.x; pc < C * cin; pc += blockDim.x) {
                const int o = pc / cin, c = pc - o * cin;
                float a0[9], a1[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) { a0[k] = 0.f; a1[k] = 0.f; }
                const float *g0 = gz + o * NP, *g1 = gz + ((R - 1) * C + o) * NP;
                const float *hc = hprev + c * NP;
                // sites in row-major order with the 3 x 3 input window held in registers: moving one site
                // along x reuses six of its values and loads the three of the new column
                for (int y = 0; y < L; ++y) {
                    const int rb[3] = {((y + L - 1) % L) * L, y * L, ((y + 1) % L) * L};
                    float win[3][3];
#pragma unroll
                    for (int dy = 0; dy < 3; ++dy) {
                        win[dy][0] = hc[rb[dy] + L - 1];
                        win[dy][1] = hc[rb[dy]];
                        win[dy][2] = hc[rb[dy] + (L > 1 ? 1 : 0)];
                    }
                    for (int x = 0; x < L; ++x) {
                        const int s = y * L + x;
                        const float x0 = g0[s], x1 = g1[s];
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx) {
                                a0[3 * dy + dx] = fmaf(x0, win[dy][dx], a0[3 * dy + dx]);
                                if (!VJP) a1[3 * dy + dx] = fmaf(x1, win[dy][dx], a1[3 * dy + dx]);
                            }
                        const int xn = x + 2 < L ? x + 2 : x + 2 - L;
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy) {
                            win[dy][0] = win[dy][1];
                            win[dy][1] = win[dy][2];
                            win[dy][2] = hc[rb[dy] + xn];
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    if (VJP) {
                        acc[off + (o * cin + c) * 9 + k] += (double)a0[k];
                    } else {
                        Oa[off + (o * cin + c) * 9 + k] = (double)a0[k];
                        Op[off + (o * cin + c) * 9 + k] = (double)a1[k];
                    }
                }
            }
            {
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
                for (int ro = warp; ro < R * C; ro += nw) {
                    float v = 0.f;
                    for (int s = lane; s < N; s += 32) v += gz[ro * NP + s];
#pragma unroll
                    for (int q = 16; q > 0; q >>= 1) v += __shfl_xor_sync(0xffffffffu, v, q);
                    if (lane == 0) {
                        if (VJP) acc[off + 9 * cin * C + ro] += (double)v;
                        else (ro < C ? Oa : Op)[off + 9 * cin * C + (ro % C)] = (double)v;
                    }
                }
            }
            if (l > 0) {
                // input gradient g_{l-1}[r][c][s] = sum_{o,k} W[o][c][k] gz[r][o][s - d_k]
                for (int rs = threadIdx.x; rs < R * N; rs += blockDim.x) {
                    const int r = rs / N, s = rs - r * N;
                    float ac[C];
#pragma unroll
                    for (int c = 0; c < C; ++c) ac[c] = 0.f;
                    const float *gr = gz + r * C * NP;
                    for (int k = 0; k < 9; ++k) {
                        const int sm = nbr[(8 - k) * N + s];   // site - d_k
                        for (int o = 0; o < C; ++o) {
                            const float gv = gr[o * NP + sm];
                            const float4 *wr = reinterpret_cast<const float4 *>(w + (o * 9 + k) * C);
#pragma unroll
                            for (int q = 0; q < C / 4; ++q) {
                                const float4 wv = wr[q];
                                ac[4 * q] = fmaf(wv.x, gv, ac[4 * q]);
                                ac[4 * q + 1] = fmaf(wv.y, gv, ac[4 * q + 1]);
                                ac[4 * q + 2] = fmaf(wv.z, gv, ac[4 * q + 2]);
                                ac[4 * q + 3] = fmaf(wv.w, gv, ac[4 * q + 3]);
                            }
                        }
                    }
#pragma unroll
                    for (int c = 0; c < C; ++c) gnext[(r * C + c) * NP + s] = ac[c];
                }
            }
        }
        __syncthreads();
    }
}

template <int C>
__global__ void __launch_bounds__(kGradThreads, kGradMinBlocks<C>) grad_fast_kernel(Problem p, const float *__restrict__ prm,
                                                                const double *__restrict__ p64,
                                                                const int8_t *__restrict__ configs, int64_t n,
                                                                double *__restrict__ O, float *__restrict__ scratch,
                                                                size_t per_block) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GradSmem m = grad_smem(p, smem);
    float *Hs = scratch + per_block * blockIdx.x;                    // [nl][C][N] h, then sigmoid(z)
    for (int64_t smp = blockIdx.x; smp < n; smp += gridDim.x)
        grad_sample<C, false>(p, m, prm, p64, configs + smp * p.N, O + (size_t)smp * p.P, O + (size_t)(n + smp) * p.P,
                              0.0, 0.0, nullptr, Hs);
}

// Vector-Jacobian products summed per chunk: chunk q holds samples
// [q K, min(n, (q + 1) K)) and its partial row part[q][P] is owned by one
// block; grad[n][2] = (g_a, g_phi) per sample.
template <int C>
__global__ void __launch_bounds__(kGradThreads, kGradMinBlocks<C>) vjp_fast_kernel(Problem p, const float *__restrict__ prm,
                                                               const double *__restrict__ p64,
                                                               const int8_t *__restrict__ configs, int64_t n,
                                                               const double *__restrict__ grad, int64_t K,
                                                               double *__restrict__ part, float *__restrict__ scratch,
                                                               size_t per_block) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GradSmem m = grad_smem(p, smem);
    float *Hs = scratch + per_block * blockIdx.x;
    const int64_t nq = (n + K - 1) / K;
    for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
        double *acc = part + (size_t)q * p.P;
        for (int k = threadIdx.x; k < p.P; k += blockDim.x) acc[k] = 0.0;
        __syncthreads();
        const int64_t s1 = min(n, (q + 1) * K);
        for (int64_t smp = q * K; smp < s1; ++smp)
            grad_sample<C, true>(p, m, prm, p64, configs + smp * p.N, nullptr, nullptr, grad[2 * smp],
                                 grad[2 * smp + 1], acc, Hs);
    }
}

// out[k] = sum over chunks q = 0 .. nq - 1 (in order) of part[q][k].
__global__ void vjp_reduce_kernel(const double *__restrict__ part, int64_t nq, int P, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    double v = 0.0;
    for (int64_t q = 0; q < nq; ++q) v += part[(size_t)q * P + k];
    out[k] = v;
}

}  // namespace

int64_t vjp_chunk_samples(int64_t n) { return std::max<int64_t>(1, (n + 1023) / 1024); }

int launch_vjp_reduce(const Problem &p, const double *part, int64_t n, double *out, const LaunchEnv &env) {
    const int64_t nq = (n + vjp_chunk_samples(n) - 1) / vjp_chunk_samples(n);
    vjp_reduce_kernel<<<(p.P + 255) / 256, 256, 0, env.stream>>>(part, nq, p.P, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *env.msg = std::string("vjp_reduce_kernel: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    ++*env.launches;
    return NQS_OK;
}

int launch_vjp_fast(const Problem &p, const float *p32, const double *p64, const int8_t *configs, int64_t n,
                    const double *grad, double *part, void *scratch, size_t scratch_bytes, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    const GradLayout gl = grad_layout(p);
    const size_t per_block = (size_t)2 * p.n_layers * p.C * p.N;   // floats
    const int64_t K = vjp_chunk_samples(n), nq = (n + K - 1) / K;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(nq, (int64_t)env.num_sms * grad_fast_blocks_per_sm(p)),
                             (int64_t)(scratch_bytes / (per_block * sizeof(float)))));
    if (int rc = allow_dynamic_smem(p.C == 16 ? vjp_fast_kernel<16> : vjp_fast_kernel<32>, gl.total, env)) return rc;
    if (p.C == 16)
        vjp_fast_kernel<16><<<blocks, kGradThreads, gl.total, env.stream>>>(p, p32, p64, configs, n, grad, K, part,
                                                                            (float *)scratch, per_block);
    else
        vjp_fast_kernel<32><<<blocks, kGradThreads, gl.total, env.stream>>>(p, p32, p64, configs, n, grad, K, part,
                                                                            (float *)scratch, per_block);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *env.msg = std::string("vjp_fast_kernel: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    ++*env.launches;
    return NQS_OK;
}

int grad_fast_blocks_per_sm(const Problem &p) {
    const size_t smem = grad_layout(p).total + 1024;
    return (int)std::max<size_t>(1, std::min<size_t>(4, 233472 / smem));
}

bool grad_fast_supported(const Problem &p, size_t max_smem) {
    return p.net == NQS_NET_SILU && (p.C == 16 || p.C == 32) && grad_layout(p).total <= max_smem;
}

size_t grad_fast_scratch_bytes(const Problem &p, int num_blocks) {
    return (size_t)2 * p.n_layers * p.C * p.N * sizeof(float) * num_blocks;
}

int launch_grad_fast(const Problem &p, const float *p32, const double *p64, const int8_t *configs, int64_t n,
                     double *O, void *scratch, size_t scratch_bytes, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    const GradLayout gl = grad_layout(p);
    const size_t per_block = (size_t)2 * p.n_layers * p.C * p.N;   // floats
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(n, (int64_t)env.num_sms * grad_fast_blocks_per_sm(p)),
                             (int64_t)(scratch_bytes / (per_block * sizeof(float)))));
    if (int rc = allow_dynamic_smem(p.C == 16 ? grad_fast_kernel<16> : grad_fast_kernel<32>, gl.total, env))
        return rc;
    if (p.C == 16)
        grad_fast_kernel<16><<<blocks, kGradThreads, gl.total, env.stream>>>(p, p32, p64, configs, n, O,
                                                                             (float *)scratch, per_block);
    else
        grad_fast_kernel<32><<<blocks, kGradThreads, gl.total, env.stream>>>(p, p32, p64, configs, n, O,
                                                                             (float *)scratch, per_block);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *env.msg = std::string("grad_fast_kernel: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    ++*env.launches;
    return NQS_OK;
}

}  // namespace nqs
