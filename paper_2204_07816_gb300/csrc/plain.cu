// CUDA-core kernels (float64 and float32): log psi, local energies,
// connected-configuration lists, the Metropolis exchange sampler and the
// per-sample backward that produces the local derivatives O_loc.
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "plain_net.cuh"

namespace nqs {

namespace {

constexpr int kThreads = 256;

__global__ void convert_params_kernel(const double *__restrict__ p64, float *__restrict__ p32, int P) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) p32[i] = (float)p64[i];
}

// ------------------------------------------------------------------ log psi
template <typename T, int CB, bool PN>
__global__ void __launch_bounds__(kThreads) logpsi_plain_kernel(Problem p, const T *params, const double *p64,
                                                                const int8_t *configs, int64_t n, double *out,
                                                                PlainLayout lay) {
    extern __shared__ __align__(16) unsigned char smem[];
    PlainNet<T> net;
    net.bind(smem, lay);
    int8_t *spins = reinterpret_cast<int8_t *>(smem + lay.total);
    const int G = lay.G, N = p.N;
    for (int64_t b0 = (int64_t)blockIdx.x * G; b0 < n; b0 += (int64_t)gridDim.x * G) {
        const int gc = (int)std::min<int64_t>(G, n - b0);
        for (int r = threadIdx.x; r < gc * N; r += blockDim.x) spins[r] = configs[b0 * N + r];
        __syncthreads();
        plain_forward<T, CB, PN>(p, params, p64, spins, gc, net);
        for (int g = threadIdx.x; g < gc; g += blockDim.x) {
            out[2 * (b0 + g)] = net.a[g];
            out[2 * (b0 + g) + 1] = net.phi[g];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ E_loc
struct ElocSmem {
    size_t spins, sigma, ci, cj, ch, tre, tim, cum, total;
};

__host__ __device__ inline ElocSmem eloc_smem(const Problem &p, size_t base, int G) {
    ElocSmem e;
    size_t o = base;
    e.spins = o; o = align16(o + (size_t)G * p.N);
    e.sigma = o; o = align16(o + p.N);
    e.ci = o; o = align16(o + 2 * (size_t)p.n_bonds);
    e.cj = o; o = align16(o + 2 * (size_t)p.n_bonds);
    e.ch = o; o = align16(o + 8 * (size_t)p.n_bonds);
    e.tre = o; o = align16(o + 16 * (size_t)(G > 0 ? G : 1));   // this batch's terms (re, im)
    e.tim = e.tre;
    e.cum = o; o = align16(o + 4 * (size_t)(p.N + 1));
    e.total = o + sizeof(EnumScratch) + 4 * sizeof(double);
    return e;
}

template <typename T, int CB, bool PN>
__global__ void __launch_bounds__(kThreads) eloc_plain_kernel(Problem p, const T *params, const double *p64,
                                                              const int8_t *configs, const double *logpsi,
                                                              int64_t n, double *out, PlainLayout lay, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    PlainNet<T> net;
    net.bind(smem, lay);
    const ElocSmem es = eloc_smem(p, lay.total, lay.G);
    int8_t *spins = reinterpret_cast<int8_t *>(smem + es.spins);
    int8_t *sigma = reinterpret_cast<int8_t *>(smem + es.sigma);
    int16_t *ci = reinterpret_cast<int16_t *>(smem + es.ci);
    int16_t *cj = reinterpret_cast<int16_t *>(smem + es.cj);
    double *ch = reinterpret_cast<double *>(smem + es.ch);
    double *terms = reinterpret_cast<double *>(smem + es.tre);
    int *cum = reinterpret_cast<int *>(smem + es.cum);
    EnumScratch &scr = *reinterpret_cast<EnumScratch *>(smem + es.total - sizeof(EnumScratch) - 4 * sizeof(double));
    // ref: a0, phi0, running sums of Re and Im of the off-diagonal terms
    double *ref = reinterpret_cast<double *>(smem + es.total - 4 * sizeof(double));
    const int G = lay.G, N = p.N;
    const int recompute = logpsi == nullptr;

    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        for (int r = threadIdx.x; r < N; r += blockDim.x) sigma[r] = configs[s * N + r];
        __syncthreads();
        double hd;
        const int nconn = enumerate_connected(p, sigma, ci, cj, ch, &hd, cum, scr);
        if (threadIdx.x == 0) {
            ref[2] = 0.0;
            ref[3] = 0.0;
            if (!recompute) { ref[0] = logpsi[2 * s]; ref[1] = logpsi[2 * s + 1]; }
        }
        __syncthreads();
        const int n_entries = nconn + recompute;
        for (int e0 = 0; e0 < n_entries; e0 += G) {
            const int gc = std::min(G, n_entries - e0);
            for (int r = threadIdx.x; r < gc * N; r += blockDim.x) {
                const int g = r / N, site = r - g * N;
                const int k = e0 + g - recompute;
                int v = sigma[site];
                if (k >= 0) {
                    const int i = ci[k], j = cj[k];
                    if (!NQS_INDEX_OK(k < nconn && i >= 0 && i < N && j >= 0 && j < N, err)) v = 0;
                    else if (site == i) v = sigma[j];
                    else if (site == j) v = sigma[i];
                }
                spins[r] = (int8_t)v;
            }
            __syncthreads();
            plain_forward<T, CB, PN>(p, params, p64, spins, gc, net);
            if (e0 == 0 && recompute && threadIdx.x == 0) { ref[0] = net.a[0]; ref[1] = net.phi[0]; }
            __syncthreads();
            for (int g = threadIdx.x; g < gc; g += blockDim.x) {
                const int k = e0 + g - recompute;
                double tr = 0.0, ti = 0.0;
                if (k >= 0) {
                    const double m = ch[k] * exp(net.a[g] - ref[0]);
                    double sn, cs;
                    sincos(net.phi[g] - ref[1], &sn, &cs);
                    tr = m * cs;
                    ti = m * sn;
                }
                terms[2 * g] = tr;
                terms[2 * g + 1] = ti;
            }
            __syncthreads();
            if (threadIdx.x == 0) {   // terms added in list order
                double sr = ref[2], si = ref[3];
                for (int g = 0; g < gc; ++g) { sr += terms[2 * g]; si += terms[2 * g + 1]; }
                ref[2] = sr;
                ref[3] = si;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double er = hd + ref[2], ei = ref[3];
            out[2 * s] = er;
            out[2 * s + 1] = ei;
            if (!isfinite(er) || !isfinite(ei)) atomicOr(err, ERRBIT_NONFINITE);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ connected list
__global__ void __launch_bounds__(kThreads) connected_kernel(Problem p, const int8_t *configs, int64_t n,
                                                             int max_conn, int32_t *n_conn, int32_t *pairs,
                                                             double *h, double *hdiag) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ElocSmem es = eloc_smem(p, 0, 0);
    int8_t *sigma = reinterpret_cast<int8_t *>(smem + es.sigma);
    int16_t *ci = reinterpret_cast<int16_t *>(smem + es.ci);
    int16_t *cj = reinterpret_cast<int16_t *>(smem + es.cj);
    double *ch = reinterpret_cast<double *>(smem + es.ch);
    int *cum = reinterpret_cast<int *>(smem + es.cum);
    EnumScratch &scr = *reinterpret_cast<EnumScratch *>(smem + es.total - sizeof(EnumScratch) - 4 * sizeof(double));
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        for (int r = threadIdx.x; r < p.N; r += blockDim.x) sigma[r] = configs[s * p.N + r];
        __syncthreads();
        double hd;
        const int nc = enumerate_connected(p, sigma, ci, cj, ch, &hd, cum, scr);
        for (int k = threadIdx.x; k < nc; k += blockDim.x) {
            pairs[(s * max_conn + k) * 2] = ci[k];
            pairs[(s * max_conn + k) * 2 + 1] = cj[k];
            h[s * max_conn + k] = ch[k];
        }
        if (threadIdx.x == 0) { n_conn[s] = nc; hdiag[s] = hd; }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ chains
// Initial states: canonical multiset (up, down, holes) shuffled by
// Fisher-Yates; swap partner of position k drawn from Philox block
// (chain, k, 0, 0) under key (seed, 1).
__global__ void init_chains_kernel(Problem p, uint64_t seed, int n_chains, int8_t *chains) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    int8_t *row = chains + (size_t)c * p.N;
    for (int k = 0; k < p.N; ++k) row[k] = (int8_t)(k < p.n_up ? 1 : (k < p.n_up + p.n_down ? -1 : 0));
    for (int k = p.N - 1; k >= 1; --k) {
        const Philox4 b = philox((uint64_t)c, (uint64_t)k, 0, 0, seed, 1);
        const int j = (int)mulhi64(b.v[0], (uint64_t)(k + 1));
        const int8_t t = row[k];
        row[k] = row[j];
        row[j] = t;
    }
}

struct SampleSmem {
    size_t cur, spins, pi, pj, pu, ca, cphi, list, cnt, total;
};

__host__ __device__ inline SampleSmem sample_smem(const Problem &p, size_t base, int G) {
    SampleSmem e;
    size_t o = base;
    e.cur = o; o = align16(o + (size_t)G * p.N);
    e.spins = o; o = align16(o + (size_t)G * p.N);
    e.pi = o; o = align16(o + 4 * (size_t)G);
    e.pj = o; o = align16(o + 4 * (size_t)G);
    e.pu = o; o = align16(o + 8 * (size_t)G);
    e.ca = o; o = align16(o + 8 * (size_t)G);
    e.cphi = o; o = align16(o + 8 * (size_t)G);
    e.list = o; o = align16(o + 4 * (size_t)(G + 1));
    e.cnt = o; o = align16(o + 16);   // moves, accepted moves of the block (kept out of registers)
    e.total = o;
    return e;
}

__device__ __forceinline__ int neighbour_dir(int i, int d, int L) {
    const int x = i % L, y = i / L;
    const int dx = d == 0 ? 1 : (d == 1 ? -1 : 0);
    const int dy = d == 2 ? 1 : (d == 3 ? -1 : 0);
    return site_at(x + dx, y + dy, L);
}

template <typename T, int CB, bool PN>
__global__ void __launch_bounds__(kThreads) sample_plain_kernel(Problem p, const T *params, const double *p64,
                                                                int8_t *chains, int n_chains, uint64_t step0,
                                                                uint64_t seed, int spc, int sweeps_between,
                                                                int burn_in, int8_t *out_cfg, double *out_logpsi,
                                                                PlainLayout lay, int *err,
                                                                unsigned long long *moves) {
    extern __shared__ __align__(16) unsigned char smem[];
    PlainNet<T> net;
    net.bind(smem, lay);
    const int G = lay.G, N = p.N;
    const SampleSmem ss = sample_smem(p, lay.total, G);
    int8_t *cur = reinterpret_cast<int8_t *>(smem + ss.cur);
    int8_t *spins = reinterpret_cast<int8_t *>(smem + ss.spins);
    int *pi = reinterpret_cast<int *>(smem + ss.pi);
    int *pj = reinterpret_cast<int *>(smem + ss.pj);
    double *pu = reinterpret_cast<double *>(smem + ss.pu);
    double *ca = reinterpret_cast<double *>(smem + ss.ca);
    double *cphi = reinterpret_cast<double *>(smem + ss.cphi);
    int *list = reinterpret_cast<int *>(smem + ss.list);
    unsigned long long *scnt = reinterpret_cast<unsigned long long *>(smem + ss.cnt);

    const int c0 = blockIdx.x * G;
    if (c0 >= n_chains) return;
    const int gc = min(G, n_chains - c0);
    for (int r = threadIdx.x; r < gc * N; r += blockDim.x) cur[r] = chains[(size_t)c0 * N + r];
    __syncthreads();
    plain_forward<T, CB, PN>(p, params, p64, cur, gc, net);
    for (int g = threadIdx.x; g < gc; g += blockDim.x) { ca[g] = net.a[g]; cphi[g] = net.phi[g]; }
    if (threadIdx.x == 0) { scnt[0] = 0; scnt[1] = 0; }
    __syncthreads();

    const int n_sweeps = burn_in + spc * sweeps_between;
    for (int sweep = 0; sweep < n_sweeps; ++sweep) {
        for (int q = 0; q < N; ++q) {
            const uint64_t step = step0 + (uint64_t)sweep * N + q;
            for (int g = threadIdx.x; g < gc; g += blockDim.x) {
                const Philox4 b = philox((uint64_t)(c0 + g), step, 0, 0, seed, 0);
                const int i = (int)mulhi64(b.v[0], (uint64_t)N);
                const int d = (int)(b.v[1] >> 62);
                const int j = neighbour_dir(i, d, p.L);
                pi[g] = i;
                pj[g] = j;
                pu[g] = (double)(b.v[2] >> 11) * 0x1.0p-53;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int cnt = 0;
                for (int g = 0; g < gc; ++g)
                    if (NQS_INDEX_OK(pi[g] >= 0 && pi[g] < N && pj[g] >= 0 && pj[g] < N, err) &&
                        cur[g * N + pi[g]] != cur[g * N + pj[g]])
                        list[cnt++] = g;
                list[G] = cnt;
                scnt[0] += (unsigned long long)cnt;
            }
            __syncthreads();
            const int cnt = list[G];
            if (cnt > 0) {
                for (int r = threadIdx.x; r < cnt * N; r += blockDim.x) {
                    const int m = r / N, site = r - m * N;
                    const int g = list[m];
                    const int i = pi[g], j = pj[g];
                    const int src = site == i ? j : (site == j ? i : site);
                    spins[r] = cur[g * N + src];
                }
                __syncthreads();
                plain_forward<T, CB, PN>(p, params, p64, spins, cnt, net);
                for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
                    const int g = list[m];
                    const double delta = 2.0 * (net.a[m] - ca[g]);
                    if (delta >= 0.0 || pu[g] < exp(delta)) {
                        atomicAdd(&scnt[1], 1ull);
                        const int i = pi[g], j = pj[g];
                        const int8_t t = cur[g * N + i];
                        cur[g * N + i] = cur[g * N + j];
                        cur[g * N + j] = t;
                        ca[g] = net.a[m];
                        cphi[g] = net.phi[m];
                    }
                }
                __syncthreads();
            }
        }
        if (sweep >= burn_in && (sweep - burn_in + 1) % sweeps_between == 0) {
            const int k = (sweep - burn_in + 1) / sweeps_between - 1;
            for (int r = threadIdx.x; r < gc * N; r += blockDim.x) {
                const int g = r / N, site = r - g * N;
                out_cfg[((size_t)(c0 + g) * spc + k) * N + site] = cur[r];
            }
            for (int g = threadIdx.x; g < gc; g += blockDim.x) {
                out_logpsi[2 * ((size_t)(c0 + g) * spc + k)] = ca[g];
                out_logpsi[2 * ((size_t)(c0 + g) * spc + k) + 1] = cphi[g];
                if (!isfinite(ca[g])) atomicOr(err, ERRBIT_NONFINITE);
            }
            __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < gc * N; r += blockDim.x) chains[(size_t)c0 * N + r] = cur[r];
    __syncthreads();
    if (threadIdx.x == 0 && moves && scnt[0]) {
        atomicAdd(&moves[0], scnt[0]);
        atomicAdd(&moves[1], scnt[1]);
    }
}

// ------------------------------------------------------------------ backward
// Per sample: forward with every layer's pre-activation z_l and output
// h_l kept in this block's global scratch, then reverse-mode through the
// head, the SiLU (silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)) and the
// periodic convolutions, for both outputs (a and phi) at once.
template <typename T>
__device__ __forceinline__ T sigmoid_t(T z) { return T(1) / (T(1) + exp(-z)); }

template <typename T>
__device__ __forceinline__ void acc_out(double *acc, int k, T v) { acc[k] += (double)v; }

// One sample. VJP = false: rows Oa, Op of O (two output-gradient streams).
// VJP = true: one stream seeded with ga w_a + gp w_phi, the sample's vector
// added to acc (each parameter by the same thread for every sample).
template <typename T, bool VJP, bool PN>
__device__ void grad_plain_sample(const Problem &p, const T *params, const double *p64, const int8_t *cfg, double *Oa,
                                  double *Op, double ga, double gp, double *acc, T *base, T *hbar) {
    if constexpr (PN) {   // the paper's CNN1 / CNN2 (d phi = 0)
        paper_grad_sample<T, VJP>(p, params, cfg, Oa, Op, ga, acc, base);
        return;
    }
    constexpr int R = VJP ? 1 : 2;
    const int N = p.N, C = p.C, L = p.L, nl = p.n_layers;
    T *h0 = base;                                  // [c_in][N]
    T *z = h0 + (size_t)p.c_in * N;                // [nl][C][N]
    T *h = z + (size_t)nl * C * N;                 // [nl][C][N]
    T *g = h + (size_t)nl * C * N;                 // [R][C][N]
    T *gz = g + (size_t)2 * C * N;                 // [R][C][N]
    {
        for (int r = threadIdx.x; r < N; r += blockDim.x) {
            const int v = cfg[r];
            if (p.c_in == 1) h0[r] = (T)v;
            else { h0[r] = (T)(v == 0); h0[N + r] = (T)(v == 1); h0[2 * N + r] = (T)(v == -1); }
        }
        __syncthreads();
        for (int l = 0; l < nl; ++l) {
            const int cin = layer_cin(p, l), off = layer_offset(p, l);
            const T *hin = l == 0 ? h0 : h + (size_t)(l - 1) * C * N;
            for (int r = threadIdx.x; r < C * N; r += blockDim.x) {
                const int co = r / N, site = r - co * N, x = site % L, y = site / L;
                T acc = params[off + 9 * cin * C + co];
                for (int c = 0; c < cin; ++c)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx)
                            acc = fma(params[off + (co * cin + c) * 9 + ky * 3 + kx],
                                      hin[c * N + site_at(x + kx - 1, y + ky - 1, L)], acc);
                z[(size_t)l * C * N + r] = acc;
                h[(size_t)l * C * N + r] = acc * sigmoid_t<T>(acc);
            }
            __syncthreads();
        }
        const T *hn = h + (size_t)(nl - 1) * C * N;
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            T v = 0;
            for (int site = 0; site < N; ++site) v += hn[c * N + site];
            hbar[c] = v;
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
        for (int r = threadIdx.x; r < C * N; r += blockDim.x) {
            const int c = r / N;
            if (VJP) {
                g[r] = (T)(ga * p64[ho + c] + gp * p64[ho + C + c]);
            } else {
                g[r] = (T)p64[ho + c];
                g[C * N + r] = (T)p64[ho + C + c];
            }
        }
        __syncthreads();
        for (int l = nl - 1; l >= 0; --l) {
            const int cin = layer_cin(p, l), off = layer_offset(p, l);
            const T *zl = z + (size_t)l * C * N;
            const T *hin = l == 0 ? h0 : h + (size_t)(l - 1) * C * N;
            for (int r = threadIdx.x; r < R * C * N; r += blockDim.x) {
                const T zz = zl[r % (C * N)];
                const T sg = sigmoid_t<T>(zz);
                gz[r] = g[r] * (sg * (T(1) + zz * (T(1) - sg)));
            }
            __syncthreads();
            // weight and bias gradients for both outputs
            const int nw = 9 * cin * C;
            for (int e = threadIdx.x; e < R * (nw + C); e += blockDim.x) {
                const int rr = e / (nw + C), idx = e - rr * (nw + C);
                const T *gzr = gz + (size_t)rr * C * N;
                T a = 0;
                if (idx < nw) {
                    const int co = idx / (9 * cin), rem = idx - co * 9 * cin, c = rem / 9, o = rem - c * 9;
                    const int dy = o / 3 - 1, dx = o % 3 - 1;
                    for (int site = 0; site < N; ++site) {
                        const int x = site % L, y = site / L;
                        a = fma(gzr[co * N + site], hin[c * N + site_at(x + dx, y + dy, L)], a);
                    }
                } else {
                    const int co = idx - nw;
                    for (int site = 0; site < N; ++site) a += gzr[co * N + site];
                }
                if (VJP) acc_out(acc, off + idx, a);
                else (rr == 0 ? Oa : Op)[off + idx] = (double)a;
            }
            if (l > 0) {
                // gradient wrt the layer input: g[c][y][x] = sum_{o, d} W[o][c][d] gz[o][y - dy][x - dx]
                for (int r = threadIdx.x; r < R * C * N; r += blockDim.x) {
                    const int rr = r / (C * N), rem = r - rr * C * N, c = rem / N, site = rem - c * N;
                    const int x = site % L, y = site / L;
                    const T *gzr = gz + (size_t)rr * C * N;
                    T a = 0;
                    for (int co = 0; co < C; ++co)
                        for (int ky = 0; ky < 3; ++ky)
                            for (int kx = 0; kx < 3; ++kx)
                                a = fma(params[off + (co * cin + c) * 9 + ky * 3 + kx],
                                        gzr[co * N + site_at(x - (kx - 1), y - (ky - 1), L)], a);
                    g[r] = a;
                }
            }
            __syncthreads();
        }
    }
}

template <typename T, bool PN>
__global__ void __launch_bounds__(kThreads) grad_plain_kernel(Problem p, const T *params, const double *p64,
                                                              const int8_t *configs, int64_t n, double *O,
                                                              T *scratch, size_t per_block) {
    __shared__ T hbar[64];
    T *base = scratch + per_block * blockIdx.x;
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x)
        grad_plain_sample<T, false, PN>(p, params, p64, configs + s * p.N, O + (size_t)s * p.P, O + (size_t)(n + s) * p.P,
                                    0.0, 0.0, nullptr, base, hbar);
}

// Vector-Jacobian products summed per chunk of K consecutive samples (one
// block per chunk, samples in order) into part[chunk][P].
template <typename T, bool PN>
__global__ void __launch_bounds__(kThreads) vjp_plain_kernel(Problem p, const T *params, const double *p64,
                                                             const int8_t *configs, int64_t n, const double *grad,
                                                             int64_t K, double *part, T *scratch, size_t per_block) {
    __shared__ T hbar[64];
    T *base = scratch + per_block * blockIdx.x;
    const int64_t nq = (n + K - 1) / K;
    for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
        double *acc = part + (size_t)q * p.P;
        for (int k = threadIdx.x; k < p.P; k += blockDim.x) acc[k] = 0.0;
        __syncthreads();
        const int64_t s1 = min(n, (q + 1) * K);
        for (int64_t s = q * K; s < s1; ++s)
            grad_plain_sample<T, true, PN>(p, params, p64, configs + s * p.N, nullptr, nullptr, grad[2 * s],
                                       grad[2 * s + 1], acc, base, hbar);
        __syncthreads();
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
void launch_convert_params(const double *p64, float *p32, int P, cudaStream_t s) {
    convert_params_kernel<<<(P + 255) / 256, 256, 0, s>>>(p64, p32, P);
}

int plain_max_group(const Problem &p, int prec, size_t extra_smem, size_t max_smem) {
    int G = 32;
    while (G > 1) {
        const size_t need = (prec == NQS_FP64 ? plain_layout<double>(p, G).total : plain_layout<float>(p, G).total) +
                            extra_smem + 64 * (size_t)G + 2 * (size_t)G * p.N + 1024;
        if (need <= max_smem && (size_t)G * p.N <= 8192) break;
        --G;
    }
    return G;
}

// PN: the network family's instantiation; CB: channel block of the SiLU
// convolutions (one instantiation serves the paper's families)
#define NQS_DISPATCH_NET(P, ...)                                           \
    if ((P).net != NQS_NET_SILU) { constexpr bool PN = true; __VA_ARGS__; } \
    else { constexpr bool PN = false; __VA_ARGS__; }
#define NQS_DISPATCH_CB(P, ...)                                            \
    if ((P).C != 4 && (P).C != 8 && (P).C != 16 && (P).C != 32) return NQS_ERR_UNSUPPORTED; \
    if ((P).net != NQS_NET_SILU) { constexpr bool PN = true; constexpr int CB = 4; __VA_ARGS__; } \
    else {                                                                 \
        constexpr bool PN = false;                                         \
        switch ((P).C) {                                                   \
            case 4: { constexpr int CB = 4; __VA_ARGS__; } break;         \
            case 8: { constexpr int CB = 8; __VA_ARGS__; } break;         \
            default: { constexpr int CB = 16; __VA_ARGS__; } break;       \
        }                                                                  \
    }

static int check_launch(const LaunchEnv &env, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *env.msg = std::string(what) + ": " + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    ++*env.launches;
    return NQS_OK;
}

template <typename T, typename K>
static int set_smem(K kernel, size_t bytes, const LaunchEnv &env) {
    if (bytes > env.max_smem) {
        *env.msg = "problem needs " + std::to_string(bytes) + " bytes of shared memory per block (max " +
                   std::to_string(env.max_smem) + ")";
        return NQS_ERR_UNSUPPORTED;
    }
    return allow_dynamic_smem(kernel, bytes, env);
}

template <typename T>
static int logpsi_plain_t(const Problem &p, const T *params, const double *p64, const int8_t *configs, int64_t n,
                          double *out, const LaunchEnv &env) {
    const int G = plain_max_group(p, sizeof(T) == 8 ? NQS_FP64 : NQS_FP32, 0, env.max_smem);
    const PlainLayout lay = plain_layout<T>(p, G);
    const size_t bytes = lay.total + align16((size_t)G * p.N);
    const int64_t groups = (n + G - 1) / G;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)env.num_sms * 4));
    NQS_DISPATCH_CB(p, {
        auto k = logpsi_plain_kernel<T, CB, PN>;
        int rc = set_smem<T>(k, bytes, env);
        if (rc) return rc;
        k<<<grid, kThreads, bytes, env.stream>>>(p, params, p64, configs, n, out, lay);
    });
    return check_launch(env, "logpsi_plain_kernel");
}

int launch_logpsi_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                        double *out, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    if (prec == NQS_FP64) return logpsi_plain_t<double>(p, dp.p64, dp.p64, configs, n, out, env);
    return logpsi_plain_t<float>(p, dp.p32, dp.p64, configs, n, out, env);
}

template <typename T>
static int eloc_plain_t(const Problem &p, const T *params, const double *p64, const int8_t *configs,
                        const double *logpsi, int64_t n, double *out, const LaunchEnv &env) {
    const size_t extra = eloc_smem(p, 0, 0).total + 64;
    const int G = plain_max_group(p, sizeof(T) == 8 ? NQS_FP64 : NQS_FP32, extra, env.max_smem);
    const PlainLayout lay = plain_layout<T>(p, G);
    const size_t bytes = eloc_smem(p, lay.total, G).total;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)env.num_sms * 8));
    NQS_DISPATCH_CB(p, {
        auto k = eloc_plain_kernel<T, CB, PN>;
        int rc = set_smem<T>(k, bytes, env);
        if (rc) return rc;
        k<<<grid, kThreads, bytes, env.stream>>>(p, params, p64, configs, logpsi, n, out, lay, env.err);
    });
    return check_launch(env, "eloc_plain_kernel");
}

int launch_eloc_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs,
                      const double *logpsi, int64_t n, double *out, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    if (prec == NQS_FP64) return eloc_plain_t<double>(p, dp.p64, dp.p64, configs, logpsi, n, out, env);
    return eloc_plain_t<float>(p, dp.p32, dp.p64, configs, logpsi, n, out, env);
}

int launch_connected(const Problem &p, const int8_t *configs, int64_t n, int max_conn, int32_t *n_conn,
                     int32_t *pairs, double *h, double *hdiag, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    const size_t bytes = eloc_smem(p, 0, 0).total;
    int rc = set_smem<double>(connected_kernel, bytes, env);
    if (rc) return rc;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)env.num_sms * 8));
    connected_kernel<<<grid, kThreads, bytes, env.stream>>>(p, configs, n, max_conn, n_conn, pairs, h, hdiag);
    return check_launch(env, "connected_kernel");
}

int launch_init_chains(const Problem &p, uint64_t seed, int n_chains, int8_t *chains, const LaunchEnv &env) {
    if (n_chains == 0) return NQS_OK;
    init_chains_kernel<<<(n_chains + 127) / 128, 128, 0, env.stream>>>(p, seed, n_chains, chains);
    return check_launch(env, "init_chains_kernel");
}

template <typename T>
static int sample_plain_t(const Problem &p, const T *params, const double *p64, int8_t *chains, int n_chains,
                          uint64_t step0, uint64_t seed, int spc, int sb, int burn, int8_t *out_cfg,
                          double *out_logpsi, const LaunchEnv &env) {
    const size_t per_g = sample_smem(p, 0, 1).total;
    int G = plain_max_group(p, sizeof(T) == 8 ? NQS_FP64 : NQS_FP32, per_g * 32 + 64, env.max_smem);
    // enough blocks to cover the GPU: at most ceil(n_chains / num_sms) chains per block
    G = std::max(1, std::min(G, (n_chains + env.num_sms - 1) / env.num_sms));
    const PlainLayout lay = plain_layout<T>(p, G);
    const size_t bytes = sample_smem(p, lay.total, G).total;
    const int grid = (n_chains + G - 1) / G;
    NQS_DISPATCH_CB(p, {
        auto k = sample_plain_kernel<T, CB, PN>;
        int rc = set_smem<T>(k, bytes, env);
        if (rc) return rc;
        k<<<grid, kThreads, bytes, env.stream>>>(p, params, p64, chains, n_chains, step0, seed, spc, sb, burn,
                                                 out_cfg, out_logpsi, lay, env.err, env.moves);
    });
    return check_launch(env, "sample_plain_kernel");
}

int launch_sample_plain(const Problem &p, int prec, const DeviceParams &dp, int8_t *chains, int n_chains,
                        uint64_t step0, uint64_t seed, int spc, int sweeps_between, int burn_in, int8_t *out_cfg,
                        double *out_logpsi, const LaunchEnv &env) {
    if (prec == NQS_FP64)
        return sample_plain_t<double>(p, dp.p64, dp.p64, chains, n_chains, step0, seed, spc, sweeps_between,
                                      burn_in, out_cfg, out_logpsi, env);
    return sample_plain_t<float>(p, dp.p32, dp.p64, chains, n_chains, step0, seed, spc, sweeps_between, burn_in,
                                 out_cfg, out_logpsi, env);
}

static size_t grad_per_block(const Problem &p) {
    if (p.net != NQS_NET_SILU) return paper_grad_per_block(p);
    return (size_t)p.c_in * p.N + 2 * (size_t)p.n_layers * p.C * p.N + 4 * (size_t)p.C * p.N;
}

size_t grad_scratch_bytes(const Problem &p, int prec, int num_blocks) {
    return grad_per_block(p) * num_blocks * (prec == NQS_FP64 ? 8 : 4);
}

int launch_vjp_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                     const double *grad, double *part, void *scratch, size_t scratch_bytes, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    const size_t esz = prec == NQS_FP64 ? 8 : 4;
    const int64_t K = vjp_chunk_samples(n), nq = (n + K - 1) / K;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(nq, (int64_t)env.num_sms * 2),
                             (int64_t)(scratch_bytes / (grad_per_block(p) * esz))));
    NQS_DISPATCH_NET(p, {
        if (prec == NQS_FP64)
            vjp_plain_kernel<double, PN><<<blocks, kThreads, 0, env.stream>>>(p, dp.p64, dp.p64, configs, n, grad, K,
                                                                              part, (double *)scratch, grad_per_block(p));
        else
            vjp_plain_kernel<float, PN><<<blocks, kThreads, 0, env.stream>>>(p, dp.p32, dp.p64, configs, n, grad, K,
                                                                             part, (float *)scratch, grad_per_block(p));
    });
    return check_launch(env, "vjp_plain_kernel");
}

int launch_grad_plain(const Problem &p, int prec, const DeviceParams &dp, const int8_t *configs, int64_t n,
                      double *O, void *scratch, size_t scratch_bytes, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    const size_t esz = prec == NQS_FP64 ? 8 : 4;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(scratch_bytes / (grad_per_block(p) * esz))));
    NQS_DISPATCH_NET(p, {
        if (prec == NQS_FP64)
            grad_plain_kernel<double, PN><<<blocks, kThreads, 0, env.stream>>>(p, dp.p64, dp.p64, configs, n, O,
                                                                                (double *)scratch, grad_per_block(p));
        else
            grad_plain_kernel<float, PN><<<blocks, kThreads, 0, env.stream>>>(p, dp.p32, dp.p64, configs, n, O,
                                                                               (float *)scratch, grad_per_block(p));
    });
    return check_launch(env, "grad_plain_kernel");
}

// Reports one failed index check without touching memory (the host-side reporting path of the checked build).
__global__ void bounds_probe_kernel(int *err) {
    if (!NQS_INDEX_OK(false, err)) return;
    atomicOr(err, ERRBIT_BOUNDS);   // the default build's check is a constant true: report the failure directly
}

int launch_bounds_probe(const LaunchEnv &env) {
    bounds_probe_kernel<<<1, 1, 0, env.stream>>>(env.err);
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "bounds probe launch failed"; return NQS_ERR_CUDA; }
    ++*env.launches;
    return NQS_OK;
}

}  // namespace nqs

// ------------------------------------------------------------------ allocation-free local derivatives
// Some callers cannot allocate device memory: code running where cudaMalloc
// is not allowed (under an allocator that forbids foreign allocations, or in
// a process that manages all device memory itself). nqs_logpsi_grad_noalloc
// serves them: it runs the per-sample backward kernels of nqs_logpsi_grad,
// with their per-block working arrays in
// a fixed device array that the library defines at file scope, so the call
// itself allocates nothing. Every GPU that loads the library holds this
// array until the process exits. All calls share it and it keeps the last
// call's contents; calls whose work overlaps on the GPU (two streams, two
// host threads) race on it and must be serialised by the caller.
#include <mutex>

namespace nqs {
namespace {

constexpr size_t kNoAllocScratchBytes = 8u << 20;   // 8 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kNoAllocMaxDevices];     // device address of the array, per device
thread_local std::string g_noalloc_error;

}  // namespace

}  // namespace nqs

extern "C" int64_t nqs_param_count(const nqs_problem *p);

extern "C" const char *nqs_noalloc_last_error(void) { return nqs::g_noalloc_error.c_str(); }

extern "C" int nqs_logpsi_grad_noalloc(const nqs_problem *q, const double *params, const int8_t *configs, int64_t n,
                                       double *O_out, int32_t precision, void *stream) {
    using namespace nqs;
    const int64_t P = nqs_param_count(q);
    if (P < 0) { g_noalloc_error = "invalid problem"; return NQS_ERR_INVALID_ARG; }
    if (precision != NQS_FP64 && precision != NQS_FP32 && precision != NQS_BF16) {
        g_noalloc_error = "bad precision";
        return NQS_ERR_INVALID_ARG;
    }
    if (n < 0 || (n > 0 && (!params || !configs || !O_out))) { g_noalloc_error = "bad arrays"; return NQS_ERR_INVALID_ARG; }
    if (n == 0) return NQS_OK;
    Problem p;
    p.model = q->model;
    p.L = q->L;
    p.N = q->L * q->L;
    p.c_in = q->model == NQS_MODEL_J1J2 ? 1 : 3;
    p.C = q->channels;
    p.n_layers = q->n_layers;
    p.J1 = q->J1; p.J2 = q->J2; p.t = q->t; p.J = q->J;
    p.sign_rule = q->sign_rule;
    p.P = (int)P;
    p.n_bonds = (q->model == NQS_MODEL_J1J2 ? 4 : 2) * p.N;
    p.n_up = q->n_up;
    p.n_down = q->n_down;
    p.net = q->net;
    // the bf16 precision differentiates with float32 internals, as nqs_logpsi_grad does; like it, float32 runs
    // grad_fast_kernel (shared-memory working sets, per-block float32 scratch) where that kernel supports the
    // problem, else the plain float kernel
    const bool f64 = precision == NQS_FP64;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_noalloc_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        g_noalloc_error = "device " + std::to_string(dev) + " is beyond the " + std::to_string(kNoAllocMaxDevices) +
                          " devices the allocation-free entry point serves";
        return NQS_ERR_UNSUPPORTED;
    }
    int num_sms = 0, optin = 0;
    e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) { g_noalloc_error = cudaGetErrorString(e); return NQS_ERR_CUDA; }
    const bool fast = !f64 && grad_fast_supported(p, (size_t)optin);
    const size_t params_bytes = f64 ? 0 : align16((size_t)P * 4);
    // per-block float / double working arrays of the kernel that runs
    const size_t per_block = fast ? grad_fast_scratch_bytes(p, 1) : grad_per_block(p) * (f64 ? 8 : 4);
    if (params_bytes + per_block > kNoAllocScratchBytes) {
        g_noalloc_error = "problem needs " + std::to_string(params_bytes + per_block) +
                           " bytes of working memory; the fixed array holds " + std::to_string(kNoAllocScratchBytes);
        return NQS_ERR_UNSUPPORTED;
    }
    void *base = nullptr;
    {
        // first call on this device: resolve the array's device address (the
        // host-side symbol is only a stand-in); do this before any capture
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                g_noalloc_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return NQS_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        base = g_noalloc_ptr[dev];
    }
    const cudaStream_t s = (cudaStream_t)stream;
    unsigned char *scratch = static_cast<unsigned char *>(base) + params_bytes;
    const size_t scratch_bytes = kNoAllocScratchBytes - params_bytes;
    if (fast) {
        float *p32 = static_cast<float *>(base);
        convert_params_kernel<<<(p.P + 255) / 256, 256, 0, s>>>(params, p32, p.P);
        e = cudaGetLastError();
        if (e != cudaSuccess) { g_noalloc_error = std::string("launch: ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
        // the fast kernel's launcher sizes its grid by the blocks whose scratch fits in the array
        int64_t launches = 0;
        std::string msg;
        LaunchEnv env;
        env.stream = s;
        env.num_sms = num_sms;
        env.max_smem = (size_t)optin;
        env.err = nullptr;
        env.launches = &launches;
        env.msg = &msg;
        const int rc = launch_grad_fast(p, p32, params, configs, n, O_out, scratch, scratch_bytes, env);
        if (rc) g_noalloc_error = msg;
        return rc;
    }
    const int64_t fit = (int64_t)(scratch_bytes / per_block);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(n, fit), (int64_t)num_sms * 2));
    if (f64) {
        NQS_DISPATCH_NET(p, grad_plain_kernel<double, PN><<<blocks, kThreads, 0, s>>>(
                                p, params, params, configs, n, O_out, reinterpret_cast<double *>(scratch),
                                grad_per_block(p)));
    } else {
        float *p32 = static_cast<float *>(base);
        convert_params_kernel<<<(p.P + 255) / 256, 256, 0, s>>>(params, p32, p.P);
        NQS_DISPATCH_NET(p, grad_plain_kernel<float, PN><<<blocks, kThreads, 0, s>>>(
                                p, p32, params, configs, n, O_out, reinterpret_cast<float *>(scratch),
                                grad_per_block(p)));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) { g_noalloc_error = std::string("launch: ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
    return NQS_OK;
}
