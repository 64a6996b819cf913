// Tensor-core (tcgen05 / TMEM) path: the periodic 3x3 convolution stack in
// bf16 with fp32 accumulation, used for log psi, local energies and the
// Metropolis sampler.
//
// Layout. A group of G configurations is evaluated together. Activations
// live in shared memory on the periodically padded (L+2) x (L+2) lattice:
// padded position p = (y + 1)(L + 2) + (x + 1), matrix row = p * G + g
// (configuration g), and each row holds 8 channels in 16 bytes per
// "k-chunk" plane: byte address = plane(kc) + row * 16. Because padded
// positions are linear, the input of tap (dy, dx) for every output row is
// the same matrix shifted by ((dy (L + 2) + dx) * G) rows, so each tap is
// one tcgen05.mma whose A descriptor starts at a shifted address (an
// implicit GEMM with no im2col copy): M = 128 rows, N = C, K = 16.
// Halo rows are refreshed by the epilogue, which writes every interior
// output also to its periodic images (a per-row destination table built
// once per kernel). Weights of the next layer stream in by bulk copy (TMA)
// while the current layer computes. Each 128-row tile commits to its own
// mbarrier, so the epilogue of tile t overlaps the MMAs of later tiles.
// Layer 0 (one spin channel or three one-hot channels) runs on CUDA cores
// in fp32 from a padded copy of the spins.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace nqs {

namespace {

constexpr int kTcThreads = 256;   // 8 warps: warp w reads TMEM lanes 32 (w % 4) ...; tiles split by w / 4
constexpr int kMaxTiles = 16;
constexpr int kIssuers = 4;       // threads issuing tcgen05.mma (lane 0 of warps 0..3)
constexpr uint32_t kNone = 0xFFFFu;

struct TcPlan {
    int L, Lp, N, G, C, KC, c_in, n_layers, n_tc;
    int count_out, n_tiles, r0, rbuf;
    uint32_t plane, act_bytes, wbytes, tmem_cols;
    // packed parameter image (global): fp32 block then one bf16 block per tensor-core layer
    uint32_t f32_count;    // 9 c_in C + n_layers C + 2 C floats
    uint32_t f32_bytes;    // padded to 16
    // shared-memory offsets
    uint32_t o_act0, o_act1, o_w0, o_w1, o_f32, o_rowtab, o_sitetab, o_spad, o_spins, o_res, o_bar, o_extra, total;
};

__host__ __device__ inline uint32_t al16(uint32_t v) { return (v + 15u) & ~15u; }

struct TcShared {
    unsigned char *base;
    uint64_t *bar_w;             // [2] weight buffers
    uint64_t *bar_tile;          // [kMaxTiles] per-tile MMA completion
    uint32_t *tmem_addr;
    int *abort_flag;
    int8_t *spins;               // [G][N] the group's configurations
    int8_t *spad;                // [Lp * Lp * G] padded copy, row = pos * G + g
    const uint2 *rowtab;         // [n_tiles * 128] destination rows of each output row
    const uint2 *sitetab;        // [N] padded positions of each site (main + images)
    float *f32;                  // w0s [9][c_in][C], biases [n_layers][C], head [2][C]
    double *a, *phi;             // [G] results
};

struct TcState {        // per-CTA pipeline state (all threads keep identical copies)
    uint32_t layers;    // tensor-core layers executed so far (tile-barrier parity)
    uint32_t wseq;      // weight loads consumed so far
    uint32_t wissued;   // weight loads issued so far
};

__device__ __forceinline__ const unsigned char *tc_layer_weights(const TcPlan &pl, const unsigned char *packed, int l) {
    return packed + pl.f32_bytes + (size_t)(l - 1) * pl.wbytes;
}

// Issue the bulk copy of weight-load number q (tensor-core layer 1 + q mod n_tc).
__device__ __forceinline__ void issue_weight_load(const TcPlan &pl, const TcShared &sh, const unsigned char *packed,
                                                  uint32_t q) {
    const int l = 1 + (int)(q % (uint32_t)pl.n_tc);
    const int b = q & 1;
    unsigned char *dst = sh.base + (b ? pl.o_w1 : pl.o_w0);
    ptx::mbar_arrive_expect_tx(&sh.bar_w[b], pl.wbytes);
    ptx::bulk_g2s(dst, tc_layer_weights(pl, packed, l), pl.wbytes, &sh.bar_w[b]);
}

// Wait on an mbarrier phase; gives up when another thread raised the abort
// flag or after the iteration limit.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, const int *abort_flag) {
    for (long long it = 0; it < ptx::kWaitLimit; ++it) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && *(volatile const int *)abort_flag) return false;
    }
    return false;
}

// Padded positions holding interior site (x, y) and its periodic images.
__device__ __forceinline__ int images(int L, int Lp, int x, int y, int (&pos)[4]) {
    const int ys[2] = {y + 1, y == 0 ? L + 1 : (y == L - 1 ? 0 : -1)};
    const int xs[2] = {x + 1, x == 0 ? L + 1 : (x == L - 1 ? 0 : -1)};
    int n = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (ys[a] >= 0 && xs[b] >= 0) pos[n++] = ys[a] * Lp + xs[b];
    return n;
}

__device__ __forceinline__ uint2 pack4(const int (&v)[4], int n) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = i < n ? (uint32_t)v[i] : kNone;
    return make_uint2(w[0] | (w[1] << 16), w[2] | (w[3] << 16));
}

template <int C>
__device__ __forceinline__ void store_rows(const TcPlan &pl, uint32_t act, uint2 dst, const uint32_t (&w)[C / 2]) {
    const uint32_t d[4] = {dst.x & 0xFFFFu, dst.x >> 16, dst.y & 0xFFFFu, dst.y >> 16};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (d[i] == kNone) break;
#pragma unroll
        for (int kc = 0; kc < C / 8; ++kc)
            ptx::st_shared_v4(act + kc * pl.plane + d[i] * 16u, w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
    }
}

// Layer 0 on CUDA cores: input channels from the padded spins, fp32 weights.
// Each thread handles the same output rows as in the tensor-core epilogue.
template <int C>
__device__ void layer0(const TcPlan &pl, const TcShared &sh, uint32_t act_out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3;
    const float *w0 = sh.f32;                         // [9][c_in][C]
    const float *b0 = sh.f32 + 9 * pl.c_in * C;       // bias of layer 0
    int offg[9];
#pragma unroll
    for (int o = 0; o < 9; ++o) offg[o] = ((o / 3 - 1) * pl.Lp + (o % 3 - 1)) * pl.G;
    for (int t = warp >> 2; t < pl.n_tiles; t += kTcThreads / 128) {
        const uint2 dst = sh.rowtab[t * 128 + quarter * 32 + lane];
        const uint32_t main = dst.x & 0xFFFFu;
        if (main == kNone) continue;
        float z[C];
#pragma unroll
        for (int c = 0; c < C; ++c) z[c] = b0[c];
#pragma unroll
        for (int o = 0; o < 9; ++o) {
            const int s = sh.spad[(int)main + offg[o]];
            if (pl.c_in == 1) {
                const float fs = (float)s;
                const float *wr = w0 + o * C;
#pragma unroll
                for (int c = 0; c < C; ++c) z[c] = fmaf(wr[c], fs, z[c]);
            } else {
                const int ch = s == 0 ? 0 : (s == 1 ? 1 : 2);
                const float *wr = w0 + (o * 3 + ch) * C;
#pragma unroll
                for (int c = 0; c < C; ++c) z[c] += wr[c];
            }
        }
        uint32_t w[C / 2];
#pragma unroll
        for (int c = 0; c < C / 2; ++c) w[c] = ptx::pack_bf16(ptx::silu_fast(z[2 * c]), ptx::silu_fast(z[2 * c + 1]));
        store_rows<C>(pl, act_out, dst, w);
    }
}

// Evaluate the G configurations in sh.spins; results to sh.a / sh.phi
// (double). Returns false if a wait timed out (the block must stop).
template <int C>
__device__ bool tc_group_forward(const TcPlan &pl, const TcShared &sh, const unsigned char *packed, TcState &st,
                                 int *err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3;
    const uint32_t act[2] = {ptx::smem_u32(sh.base + pl.o_act0), ptx::smem_u32(sh.base + pl.o_act1)};
    const uint32_t tmem = *sh.tmem_addr;
    const uint32_t idesc = ptx::idesc_bf16(128, C);
    const int G = pl.G;

    // padded spins: every site to its main position and periodic images
    for (int r = threadIdx.x; r < G * pl.N; r += blockDim.x) {
        const int g = r / pl.N, site = r - g * pl.N;
        const uint2 pos = sh.sitetab[site];
        const int8_t v = sh.spins[r];
        const uint32_t d[4] = {pos.x & 0xFFFFu, pos.x >> 16, pos.y & 0xFFFFu, pos.y >> 16};
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (d[i] != kNone) sh.spad[d[i] * G + g] = v;
    }
    __syncthreads();
    layer0<C>(pl, sh, act[0]);
    ptx::fence_async_smem();
    __syncthreads();

    int cur = 0;
    for (int l = 1; l < pl.n_layers; ++l) {
        const bool last = (l == pl.n_layers - 1);
        const uint32_t parity = st.layers & 1u;
        // four issuing threads (lane 0 of warps 0-3, one per SM sub-partition),
        // issuer w owns tiles w, w + 4, ...; each tile commits to its own barrier
        if (lane == 0 && warp < kIssuers) {
            const uint32_t q = st.wseq;
            if (wait_or_abort(&sh.bar_w[q & 1], (q >> 1) & 1, sh.abort_flag)) {
                // prefetch the next load into the other buffer (its last reader, load q - 1, has completed)
                if (warp == 0) issue_weight_load(pl, sh, packed, q + 1);
                ptx::tc_fence_after();
                const uint64_t a_base = ptx::smem_desc(act[cur], pl.plane, 128);
                const uint64_t b_base =
                    ptx::smem_desc(ptx::smem_u32(sh.base + ((q & 1) ? pl.o_w1 : pl.o_w0)), C * 16, 128);
                uint32_t offs[9];
#pragma unroll
                for (int o = 0; o < 9; ++o)
                    offs[o] = (uint32_t)(pl.r0 + ((o / 3 - 1) * pl.Lp + (o % 3 - 1)) * G);   // row of tile 0
                for (int t = warp; t < pl.n_tiles; t += kIssuers) {
                    const uint32_t d = tmem + (uint32_t)(t * C);
#pragma unroll
                    for (int o = 0; o < 9; ++o) {
                        const uint32_t arow = offs[o] + (uint32_t)(t * 128);
#pragma unroll
                        for (int kk = 0; kk < C / 16; ++kk) {
                            const uint64_t ad = a_base + ((arow * 16u + (uint32_t)(2 * kk) * pl.plane) >> 4);
                            const uint64_t bd = b_base + (uint64_t)(((o * (C / 8) + 2 * kk) * C * 16) >> 4);
                            ptx::mma_bf16(d, ad, bd, idesc, (o | kk) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit(&sh.bar_tile[t]);
                }
            } else {
                atomicOr(sh.abort_flag, 1);
                atomicOr(err, ERRBIT_TIMEOUT);
            }
        }
        st.wseq += 1;
        st.wissued = st.wseq + 1;
        st.layers += 1;

        // epilogue per tile as soon as its MMAs complete: bias + SiLU; bf16
        // rows (and halo images) or head contributions
        const float *bias = sh.f32 + 9 * pl.c_in * C + l * C;
        const float *wa = sh.f32 + 9 * pl.c_in * C + pl.n_layers * C;
        const uint32_t out = act[cur ^ 1];
        float *contrib = reinterpret_cast<float *>(sh.base + (cur ? pl.o_act0 : pl.o_act1));
        bool ok = true;
        for (int t = warp >> 2; t < pl.n_tiles; t += kTcThreads / 128) {
            const bool got = wait_or_abort(&sh.bar_tile[t], parity, sh.abort_flag);
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }   // reconverges the warp
            ptx::tc_fence_after();
            float v[C];
#pragma unroll
            for (int h = 0; h < C / 16; ++h) {
                float tmp[16];
                ptx::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * C + 16 * h), tmp);
#pragma unroll
                for (int i = 0; i < 16; ++i) v[16 * h + i] = tmp[i];
            }
            const uint2 dst = sh.rowtab[t * 128 + quarter * 32 + lane];
            const uint32_t main = dst.x & 0xFFFFu;
            if (main == kNone) continue;
            if (!last) {
                uint32_t w[C / 2];
#pragma unroll
                for (int c = 0; c < C / 2; ++c)
                    w[c] = ptx::pack_bf16(ptx::silu_fast(v[2 * c] + bias[2 * c]),
                                          ptx::silu_fast(v[2 * c + 1] + bias[2 * c + 1]));
                store_rows<C>(pl, out, dst, w);
            } else {
                float ca = 0.f, cp = 0.f;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const float hv = ptx::silu_fast(v[c] + bias[c]);
                    ca = fmaf(wa[c], hv, ca);
                    cp = fmaf(wa[C + c], hv, cp);
                }
                contrib[2 * main] = ca;       // indexed by the row p * G + g
                contrib[2 * main + 1] = cp;
            }
        }
        if (!ok) {
            atomicOr(sh.abort_flag, 1);
            atomicOr(err, ERRBIT_TIMEOUT);
        }
        ptx::tc_fence_before();
        ptx::fence_async_smem();
        __syncthreads();
        if (*sh.abort_flag) return false;
        cur ^= 1;
    }
    // head: a[g] = sum over sites of the contributions (one warp per g,
    // fixed order); after the last swap the contributions sit in buffer `cur`
    const float *contrib = reinterpret_cast<const float *>(sh.base + (cur ? pl.o_act1 : pl.o_act0));
    for (int g = warp; g < G; g += kTcThreads / 32) {
        float sa = 0.f, sp = 0.f;
        for (int site = lane; site < pl.N; site += 32) {
            const int row = (int)(sh.sitetab[site].x & 0xFFFFu) * G + g;
            sa += contrib[2 * row];
            sp += contrib[2 * row + 1];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
        }
        if (lane == 0) {
            sh.a[g] = (double)sa;
            sh.phi[g] = (double)sp;
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- kernel prologue / epilogue
__device__ void tc_setup(const TcPlan &pl, TcShared &sh, unsigned char *smem, const unsigned char *packed,
                         TcState &st) {
    sh.base = smem;
    sh.bar_w = reinterpret_cast<uint64_t *>(smem + pl.o_bar);
    sh.bar_tile = sh.bar_w + 2;
    sh.tmem_addr = reinterpret_cast<uint32_t *>(smem + pl.o_bar + 8 * (2 + kMaxTiles));
    sh.abort_flag = reinterpret_cast<int *>(smem + pl.o_bar + 8 * (2 + kMaxTiles) + 4);
    sh.spins = reinterpret_cast<int8_t *>(smem + pl.o_spins);
    sh.spad = reinterpret_cast<int8_t *>(smem + pl.o_spad);
    sh.rowtab = reinterpret_cast<const uint2 *>(smem + pl.o_rowtab);
    sh.sitetab = reinterpret_cast<const uint2 *>(smem + pl.o_sitetab);
    sh.f32 = reinterpret_cast<float *>(smem + pl.o_f32);
    sh.a = reinterpret_cast<double *>(smem + pl.o_res);
    sh.phi = sh.a + pl.G;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&sh.bar_w[0], 1);
        ptx::mbar_init(&sh.bar_w[1], 1);
        for (int t = 0; t < kMaxTiles; ++t) ptx::mbar_init(&sh.bar_tile[t], 1);
        *sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    const float *src = reinterpret_cast<const float *>(packed);
    for (uint32_t i = threadIdx.x; i < pl.f32_count; i += blockDim.x) sh.f32[i] = src[i];
    // destination table of every output row: main row and periodic images
    uint2 *rowtab = reinterpret_cast<uint2 *>(smem + pl.o_rowtab);
    for (int lr = threadIdx.x; lr < pl.n_tiles * 128; lr += blockDim.x) {
        const int row = pl.r0 + lr;
        int pos[4];
        int n = 0;
        const int p = row / pl.G, g = row - p * pl.G;
        const int y = p / pl.Lp - 1, x = p % pl.Lp - 1;
        if (row < pl.r0 + pl.count_out * pl.G && x >= 0 && x < pl.L && y >= 0 && y < pl.L) {
            n = images(pl.L, pl.Lp, x, y, pos);
            for (int i = 0; i < n; ++i) pos[i] = pos[i] * pl.G + g;
        }
        rowtab[lr] = pack4(pos, n);
    }
    uint2 *sitetab = reinterpret_cast<uint2 *>(smem + pl.o_sitetab);
    for (int s = threadIdx.x; s < pl.N; s += blockDim.x) {
        int pos[4];
        const int n = images(pl.L, pl.Lp, s % pl.L, s / pl.L, pos);
        sitetab[s] = pack4(pos, n);
    }
    // zero both activation buffers and the padded spins once: rows outside
    // the lattice are read by discarded output rows only, but keep them finite
    for (uint32_t i = threadIdx.x; i < pl.act_bytes / 4; i += blockDim.x) {
        reinterpret_cast<uint32_t *>(smem + pl.o_act0)[i] = 0u;
        reinterpret_cast<uint32_t *>(smem + pl.o_act1)[i] = 0u;
    }
    for (uint32_t i = threadIdx.x; i < (uint32_t)(pl.Lp * pl.Lp * pl.G); i += blockDim.x) sh.spad[i] = 0;
    ptx::fence_async_smem();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        ptx::tmem_alloc(sh.tmem_addr, pl.tmem_cols);
        ptx::tmem_relinquish();
    }
    if (threadIdx.x == 0) issue_weight_load(pl, sh, packed, 0);
    st.layers = 0;
    st.wseq = 0;
    st.wissued = 1;
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
}

__device__ void tc_teardown(const TcPlan &pl, TcShared &sh, TcState &st) {
    __syncthreads();
    if (threadIdx.x == 0) {
        // the prefetched weight load that nobody consumed
        for (uint32_t q = st.wseq; q < st.wissued; ++q) ptx::mbar_wait(&sh.bar_w[q & 1], (q >> 1) & 1);
    }
    ptx::tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(*sh.tmem_addr, pl.tmem_cols);
    }
}

// ---------------------------------------------------------------- kernels
template <int C>
__global__ void __launch_bounds__(kTcThreads, 1) logpsi_tc_kernel(TcPlan pl, const unsigned char *packed,
                                                                   const int8_t *configs, int64_t n, double *out,
                                                                   int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    const int G = pl.G, N = pl.N;
    for (int64_t b0 = (int64_t)blockIdx.x * G; b0 < n; b0 += (int64_t)gridDim.x * G) {
        const int gc = (int)min((int64_t)G, n - b0);
        for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
            const int g = r / N;
            sh.spins[r] = configs[(b0 + (g < gc ? g : 0)) * N + (r - g * N)];
        }
        __syncthreads();
        if (!tc_group_forward<C>(pl, sh, packed, st, err)) break;
        for (int g = threadIdx.x; g < gc; g += blockDim.x) {
            out[2 * (b0 + g)] = sh.a[g];
            out[2 * (b0 + g) + 1] = sh.phi[g];
        }
        __syncthreads();
    }
    tc_teardown(pl, sh, st);
}

template <int C>
__global__ void __launch_bounds__(kTcThreads, 1) eloc_tc_kernel(TcPlan pl, Problem p, const unsigned char *packed,
                                                                 const int8_t *configs, const double *logpsi,
                                                                 int64_t n, double *out, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    const int G = pl.G, N = pl.N;
    unsigned char *ex = smem + pl.o_extra;
    int8_t *sigma = reinterpret_cast<int8_t *>(ex);
    int16_t *ci = reinterpret_cast<int16_t *>(ex + al16(N));
    int16_t *cj = ci + p.n_bonds;
    double *ch = reinterpret_cast<double *>(ex + al16(N) + al16(4 * p.n_bonds));
    int *cum = reinterpret_cast<int *>(ch + p.n_bonds);
    EnumScratch *scr = reinterpret_cast<EnumScratch *>(ex + al16(N) + al16(4 * p.n_bonds) + al16(8 * p.n_bonds) +
                                                       al16(4 * (N + 1)));
    double *ref = reinterpret_cast<double *>(scr + 1);   // a0, phi0
    double *lp = ref + 4;                                 // [n_bonds + 1][2]: (a, phi) of every list entry
    const int recompute = logpsi == nullptr;
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
        for (int r = threadIdx.x; r < N; r += blockDim.x) sigma[r] = configs[s * N + r];
        __syncthreads();
        double hd;
        const int nconn = enumerate_connected(p, sigma, ci, cj, ch, &hd, cum, *scr);
        if (threadIdx.x == 0 && !recompute) { ref[0] = logpsi[2 * s]; ref[1] = logpsi[2 * s + 1]; }
        __syncthreads();
        const int n_entries = nconn + recompute;
        bool ok = true;
        for (int e0 = 0; e0 < n_entries; e0 += G) {
            const int gc = min(G, n_entries - e0);
            for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
                const int g = r / N, site = r - g * N;
                const int k = e0 + g - recompute;
                int v = sigma[site];
                if (g < gc && k >= 0) {
                    const int i = ci[k], j = cj[k];
                    if (site == i) v = sigma[j];
                    else if (site == j) v = sigma[i];
                }
                sh.spins[r] = (int8_t)v;
            }
            __syncthreads();
            if (!tc_group_forward<C>(pl, sh, packed, st, err)) { ok = false; break; }
            if (threadIdx.x < gc) {
                lp[2 * (e0 + threadIdx.x)] = sh.a[threadIdx.x];
                lp[2 * (e0 + threadIdx.x) + 1] = sh.phi[threadIdx.x];
            }
        }
        if (!ok) break;
        __syncthreads();
        if (recompute && threadIdx.x == 0) { ref[0] = lp[0]; ref[1] = lp[1]; }
        __syncthreads();
        // E_loc = H_diag + sum_k H_k exp((a'_k - a) + i (phi'_k - phi)) in float64,
        // all terms of the sample at once, fixed-order block reduction
        double tr = 0.0, ti = 0.0;
        for (int k = threadIdx.x; k < nconn; k += blockDim.x) {
            const double m = ch[k] * exp(lp[2 * (k + recompute)] - ref[0]);
            double sn, cs;
            sincos(lp[2 * (k + recompute) + 1] - ref[1], &sn, &cs);
            tr = fma(m, cs, tr);
            ti = fma(m, sn, ti);
        }
        const double sr = block_sum(tr, scr->dscr);
        const double si = block_sum(ti, scr->dscr);
        if (threadIdx.x == 0) {
            const double er = hd + sr, ei = si;
            out[2 * s] = er;
            out[2 * s + 1] = ei;
            if (!isfinite(er) || !isfinite(ei)) atomicOr(err, ERRBIT_NONFINITE);
        }
        __syncthreads();
    }
    tc_teardown(pl, sh, st);
}

__device__ __forceinline__ int neighbour_dir_tc(int i, int d, int L) {
    const int x = i % L, y = i / L;
    const int dx = d == 0 ? 1 : (d == 1 ? -1 : 0);
    const int dy = d == 2 ? 1 : (d == 3 ? -1 : 0);
    return ((y + dy + L) % L) * L + (x + dx + L) % L;
}

// Metropolis exchange sampler; each block owns up to G chains.
template <int C>
__global__ void __launch_bounds__(kTcThreads, 1) sample_tc_kernel(TcPlan pl, const unsigned char *packed,
                                                                   int8_t *chains, int n_chains, int per_block,
                                                                   uint64_t step0, uint64_t seed, int spc,
                                                                   int sweeps_between, int burn_in, int8_t *out_cfg,
                                                                   double *out_logpsi, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    const int G = pl.G, N = pl.N;
    unsigned char *ex = smem + pl.o_extra;
    int8_t *cur = reinterpret_cast<int8_t *>(ex);                                // [per_block][N]
    int *pi = reinterpret_cast<int *>(ex + al16(G * N));
    int *pj = pi + G;
    int *list = pj + G;                                                          // [G + 1]
    double *pu = reinterpret_cast<double *>(ex + al16(G * N) + al16(4 * (3 * G + 1)));
    double *ca = pu + G;
    double *cphi = ca + G;
    const int c0 = blockIdx.x * per_block;
    const int gc = min(per_block, n_chains - c0);
    bool ok = gc > 0;
    if (ok) {
        for (int r = threadIdx.x; r < gc * N; r += blockDim.x) cur[r] = chains[(size_t)c0 * N + r];
        __syncthreads();
        for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
            const int g = r / N;
            sh.spins[r] = cur[(g < gc ? g : 0) * N + (r - g * N)];
        }
        __syncthreads();
        ok = tc_group_forward<C>(pl, sh, packed, st, err);
        for (int g = threadIdx.x; g < gc; g += blockDim.x) { ca[g] = sh.a[g]; cphi[g] = sh.phi[g]; }
        __syncthreads();
    }
    const int n_sweeps = burn_in + spc * sweeps_between;
    for (int sweep = 0; ok && sweep < n_sweeps; ++sweep) {
        for (int q = 0; q < N; ++q) {
            const uint64_t step = step0 + (uint64_t)sweep * N + q;
            for (int g = threadIdx.x; g < gc; g += blockDim.x) {
                const Philox4 b = philox((uint64_t)(c0 + g), step, 0, 0, seed, 0);
                const int i = (int)mulhi64(b.v[0], (uint64_t)N);
                pi[g] = i;
                pj[g] = neighbour_dir_tc(i, (int)(b.v[1] >> 62), pl.L);
                pu[g] = (double)(b.v[2] >> 11) * 0x1.0p-53;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                int cnt = 0;
                for (int g = 0; g < gc; ++g)
                    if (cur[g * N + pi[g]] != cur[g * N + pj[g]]) list[cnt++] = g;
                list[G] = cnt;
            }
            __syncthreads();
            const int cnt = list[G];
            if (cnt == 0) continue;
            for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
                const int m = r / N, site = r - m * N;
                const int g = list[m < cnt ? m : 0];
                const int i = pi[g], j = pj[g];
                const int src = site == i ? j : (site == j ? i : site);
                sh.spins[r] = cur[g * N + src];
            }
            __syncthreads();
            if (!tc_group_forward<C>(pl, sh, packed, st, err)) { ok = false; break; }
            for (int m = threadIdx.x; m < cnt; m += blockDim.x) {
                const int g = list[m];
                const double delta = 2.0 * (sh.a[m] - ca[g]);
                if (delta >= 0.0 || pu[g] < exp(delta)) {
                    const int i = pi[g], j = pj[g];
                    const int8_t t = cur[g * N + i];
                    cur[g * N + i] = cur[g * N + j];
                    cur[g * N + j] = t;
                    ca[g] = sh.a[m];
                    cphi[g] = sh.phi[m];
                }
            }
            __syncthreads();
        }
        if (ok && sweep >= burn_in && (sweep - burn_in + 1) % sweeps_between == 0) {
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
    if (gc > 0 && ok)
        for (int r = threadIdx.x; r < gc * N; r += blockDim.x) chains[(size_t)c0 * N + r] = cur[r];
    tc_teardown(pl, sh, st);
}

// ---------------------------------------------------------------- packing
// fp32 block: w0s[o][ci][c] = W0[c][ci][o], biases[l][c], head[2][c];
// bf16 block per layer l >= 1: B operand [o][kc][n][8]: element (o, k = c_in, n = c_out).
__global__ void tc_pack_kernel(Problem p, TcPlan pl, const double *params, unsigned char *packed) {
    const int C = p.C;
    float *f = reinterpret_cast<float *>(packed);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int e = tid; e < 9 * p.c_in * C; e += nth) {
        const int o = e / (p.c_in * C), rem = e - o * p.c_in * C, ci = rem / C, c = rem - ci * C;
        f[e] = (float)params[(c * p.c_in + ci) * 9 + o];
    }
    for (int e = tid; e < p.n_layers * C; e += nth) {
        const int l = e / C, c = e - l * C;
        f[9 * p.c_in * C + e] = (float)params[layer_offset(p, l) + 9 * layer_cin(p, l) * C + c];
    }
    for (int e = tid; e < 2 * C; e += nth) f[9 * p.c_in * C + p.n_layers * C + e] = (float)params[head_offset(p) + e];
    const int per = 9 * C * C;
    for (int e = tid; e < (p.n_layers - 1) * per; e += nth) {
        const int l = 1 + e / per, r = e - (l - 1) * per;
        const int o = r / (C * C), r2 = r - o * C * C, n = r2 / C, k = r2 - n * C;
        const double w = params[layer_offset(p, l) + (n * C + k) * 9 + o];
        __nv_bfloat16 *dst = reinterpret_cast<__nv_bfloat16 *>(packed + pl.f32_bytes + (size_t)(l - 1) * pl.wbytes);
        dst[((o * (C / 8) + k / 8) * C + n) * 8 + (k % 8)] = __float2bfloat16_rn((float)w);
    }
}

// ---------------------------------------------------------------- host planning
bool make_plan(const Problem &p, int G, size_t max_smem, int extra_bytes, TcPlan *out, std::string *why) {
    TcPlan pl{};
    pl.L = p.L;
    pl.Lp = p.L + 2;
    pl.N = p.N;
    pl.G = G;
    pl.C = p.C;
    pl.KC = p.C / 8;
    pl.c_in = p.c_in;
    pl.n_layers = p.n_layers;
    pl.n_tc = p.n_layers - 1;
    pl.count_out = (p.L - 1) * pl.Lp + p.L;
    pl.r0 = (pl.Lp + 1) * G;
    pl.n_tiles = (pl.count_out * G + 127) / 128;
    const int reach = (pl.Lp + 1) * G;
    pl.rbuf = std::max(pl.r0 + pl.n_tiles * 128 + reach, pl.Lp * pl.Lp * G);
    pl.rbuf = (pl.rbuf + 7) & ~7;
    pl.plane = (uint32_t)pl.rbuf * 16u;
    pl.act_bytes = pl.plane * pl.KC;
    pl.wbytes = 9u * p.C * p.C * 2u;
    uint32_t cols = 32;
    while (cols < (uint32_t)(pl.n_tiles * p.C)) cols <<= 1;
    pl.tmem_cols = cols;
    pl.f32_count = 9 * p.c_in * p.C + p.n_layers * p.C + 2 * p.C;
    pl.f32_bytes = al16(pl.f32_count * 4);
    uint32_t o = 0;
    pl.o_act0 = o; o = al16(o + pl.act_bytes);
    pl.o_act1 = o; o = al16(o + pl.act_bytes);
    pl.o_w0 = o; o = al16(o + pl.wbytes);
    pl.o_w1 = o; o = al16(o + pl.wbytes);
    pl.o_f32 = o; o = al16(o + pl.f32_count * 4);
    pl.o_rowtab = o; o = al16(o + 8 * pl.n_tiles * 128);
    pl.o_sitetab = o; o = al16(o + 8 * p.N);
    pl.o_spad = o; o = al16(o + pl.Lp * pl.Lp * G);
    pl.o_spins = o; o = al16(o + G * p.N);
    pl.o_res = o; o = al16(o + 16 * G);
    pl.o_bar = o; o = al16(o + 8 * (2 + kMaxTiles) + 8);
    pl.o_extra = o; o = al16(o + extra_bytes);
    // co-resident blocks must not ask for more than the SM's 512 TMEM
    // columns together: pad shared memory to cap residency
    const uint32_t sm_bytes = 233472u;   // 228 KB per SM, 1 KB reserved per block
    while (cols * (sm_bytes / (o + 1024u)) > 512u) o += 1024u;
    pl.total = o;
    if (cols > 512) { *why = "tensor-memory tile does not fit in 512 columns"; return false; }
    if (pl.n_tiles > kMaxTiles) { *why = "more than 16 row tiles per group"; return false; }
    if (pl.rbuf >= (int)kNone) { *why = "row index range exceeds 16 bits"; return false; }
    if (pl.total > max_smem) { *why = "shared memory plan exceeds the per-block limit"; return false; }
    if (pl.n_tc < 1) { *why = "the tensor-core path needs at least two conv layers"; return false; }
    *out = pl;
    return true;
}

int eloc_extra(const Problem &p, int G) {
    (void)G;
    return (int)(al16(p.N) + al16(4 * p.n_bonds) + al16(8 * p.n_bonds) + al16(4 * (p.N + 1)) + sizeof(EnumScratch) +
                 4 * sizeof(double) + 16 * (p.n_bonds + 1));
}

int sample_extra(const Problem &p, int G) { return (int)(al16(G * p.N) + al16(4 * (3 * G + 1)) + 24 * G); }

// Choose G maximising useful rows / computed rows within the limits.
bool best_plan(const Problem &p, size_t max_smem, bool eloc, int gmax, TcPlan *out, std::string *why) {
    double best = -1.0;
    bool found = false;
    for (int G = 1; G <= gmax; ++G) {
        TcPlan pl;
        std::string w;
        if (!make_plan(p, G, max_smem, eloc ? eloc_extra(p, G) : 0, &pl, &w)) { if (!found) *why = w; continue; }
        const double eff = (double)(p.N * G) / (double)(pl.n_tiles * 128);
        if (eff > best + 1e-9) { best = eff; *out = pl; found = true; }
    }
    return found;
}

int check(const LaunchEnv &env, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        *env.msg = std::string(what) + ": " + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    ++*env.launches;
    return NQS_OK;
}

template <typename K>
int prep(K kernel, const TcPlan &pl, const LaunchEnv &env) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.total);
    if (e != cudaSuccess) {
        *env.msg = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return NQS_ERR_CUDA;
    }
    return NQS_OK;
}

TcPlan plan_for_pack(const Problem &p) {
    TcPlan pl{};
    pl.f32_count = 9 * p.c_in * p.C + p.n_layers * p.C + 2 * p.C;
    pl.f32_bytes = al16(pl.f32_count * 4);
    pl.wbytes = 9u * p.C * p.C * 2u;
    return pl;
}

}  // namespace

bool tc_supported(const Problem &p, std::string *why) {
    if (p.C != 16 && p.C != 32) { *why = "the tensor-core path needs 16 or 32 channels"; return false; }
    if (p.n_layers < 2) { *why = "the tensor-core path needs at least two conv layers"; return false; }
    return true;
}

size_t tc_packed_bytes(const Problem &p) {
    const TcPlan pl = plan_for_pack(p);
    return pl.f32_bytes + (size_t)(p.n_layers > 1 ? p.n_layers - 1 : 0) * pl.wbytes;
}

int launch_tc_pack(const Problem &p, const double *p64, void *packed, const LaunchEnv &env) {
    std::string why;
    if (!tc_supported(p, &why)) { *env.msg = why; return NQS_ERR_UNSUPPORTED; }
    const TcPlan pl = plan_for_pack(p);
    tc_pack_kernel<<<64, 256, 0, env.stream>>>(p, pl, p64, (unsigned char *)packed);
    return check(env, "tc_pack_kernel");
}

#define NQS_TC_DISPATCH(C, ...)                                      \
    if ((C) == 16) { constexpr int CC = 16; __VA_ARGS__; }            \
    else { constexpr int CC = 32; __VA_ARGS__; }

int launch_logpsi_tc(const Problem &p, const double *, const void *packed, const int8_t *configs, int64_t n,
                     double *out, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    std::string why;
    TcPlan pl;
    if (!tc_supported(p, &why) || !best_plan(p, env.max_smem, false, 16, &pl, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    const int64_t groups = (n + pl.G - 1) / pl.G;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(groups, env.num_sms));
    NQS_TC_DISPATCH(p.C, {
        auto k = logpsi_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, kTcThreads, pl.total, env.stream>>>(pl, (const unsigned char *)packed, configs, n, out, env.err);
    });
    return check(env, "logpsi_tc_kernel");
}

int launch_eloc_tc(const Problem &p, const double *, const void *packed, const int8_t *configs,
                   const double *logpsi, int64_t n, double *out, const LaunchEnv &env) {
    if (n == 0) return NQS_OK;
    std::string why;
    TcPlan pl;
    if (!tc_supported(p, &why) || !best_plan(p, env.max_smem, true, 16, &pl, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, env.num_sms));
    NQS_TC_DISPATCH(p.C, {
        auto k = eloc_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, kTcThreads, pl.total, env.stream>>>(pl, p, (const unsigned char *)packed, configs, logpsi, n, out,
                                                      env.err);
    });
    return check(env, "eloc_tc_kernel");
}

int launch_sample_tc(const Problem &p, const double *, const void *packed, int8_t *chains, int n_chains,
                     uint64_t step0, uint64_t seed, int spc, int sweeps_between, int burn_in, int8_t *out_cfg,
                     double *out_logpsi, const LaunchEnv &env) {
    std::string why;
    if (!tc_supported(p, &why)) { *env.msg = why; return NQS_ERR_UNSUPPORTED; }
    // chains per block: enough blocks to cover the SMs, at most G
    const int want = std::max(1, (n_chains + env.num_sms - 1) / env.num_sms);
    TcPlan pl;
    bool ok = false;
    for (int G = std::min(want, 16); G >= 1 && !ok; --G)
        ok = make_plan(p, G, env.max_smem, sample_extra(p, G), &pl, &why);
    if (!ok) { *env.msg = why; return NQS_ERR_UNSUPPORTED; }
    const int per_block = pl.G;
    const int grid = (n_chains + per_block - 1) / per_block;
    NQS_TC_DISPATCH(p.C, {
        auto k = sample_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, kTcThreads, pl.total, env.stream>>>(pl, (const unsigned char *)packed, chains, n_chains, per_block,
                                                      step0, seed, spc, sweeps_between, burn_in, out_cfg, out_logpsi,
                                                      env.err);
    });
    return check(env, "sample_tc_kernel");
}

}  // namespace nqs
