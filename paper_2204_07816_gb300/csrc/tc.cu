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
// Layer 0 (one spin channel, or three one-hot channels) instead reads a
// small im2col matrix of the spins (K = 16 or 32).
//
// Pipeline. Halo rows are refreshed by the epilogue, which writes every
// interior output also to its periodic images (a per-row destination table
// built once per kernel). Each 128-row tile commits to its own mbarrier, so
// the epilogue of tile t overlaps the MMAs of later tiles; two dedicated
// warps issue the MMAs while four or eight warps run epilogues. A plan keeps
// one or two groups ("slots") in flight per block, and one or two blocks per
// SM: while the CUDA cores run the epilogue of one group's layer, the tensor
// core runs another group's MMAs. The next layer's weights stream in by
// bulk copy (cp.async.bulk) into a double buffer while the current layer
// runs. One-block plans evaluate each connected configuration of a local
// energy on its cone only (struct Band below).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include <vector>

#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace nqs {

namespace {

// Warp roles: pl.epi epilogue warps (a multiple of 4; warp w reads TMEM lanes
// 32 (w % 4) ... and takes tiles w / 4, w / 4 + epi / 4, ...), then kIssuers
// issuing warps (lane 0 issues tcgen05.mma). The single-problem kernels are
// compiled for two co-resident blocks per SM (at most 102 registers a
// thread), so that one block's MMAs run while the other block is between
// layers or between groups of configurations.
constexpr int kMaxEpiWarps = 8;
constexpr int kIssuers = 2;
constexpr int kTcThreads = 32 * (kMaxEpiWarps + kIssuers);
// Blocks per SM the log psi / local-energy kernels are compiled for: two for
// 16 channels (register cap 102), one for 32 channels (two-block plans are
// slower there, and the uncapped registers are measured 2-3 % faster). The
// sampler is compiled for two blocks at both widths.
template <int C> constexpr int kMinBlocks = C == 16 ? 2 : 1;
constexpr int kMaxTiles = 16;
constexpr int kPropWindow = 16;   // sampler: proposal steps drawn at once
constexpr int kPropWindowOne = 64;   // the same with one chain per block (one draw per thread either way)
__host__ __device__ inline int prop_window(int per_block) { return per_block == 1 ? kPropWindowOne : kPropWindow; }

// A configuration read with two sites exchanged (the sampler's proposal),
// in place of the group's copy in shared memory (one-configuration groups).
struct SwapSrc {
    const int8_t *cfg;
    int i, j;
};
constexpr int kMaxSlots = 2;
constexpr uint32_t kNone = 0xFFFFu;

struct TcPlan {
    int L, Lp, N, G, C, KC, c_in, K0, n_layers, slots;
    int epi, ctas;       // epilogue warps per block; blocks per SM the plan is sized for
    int count_out, n_tiles, r0, rbuf;
    uint32_t plane, act_bytes, w0bytes, wbytes, tmem_cols, slot_cols;
    // packed parameter image (global): fp32 biases + head, then bf16 operand
    // images of layer 0 (K0 x C) and of every later layer (9 x C x C)
    uint32_t f32_count, f32_bytes;
    // shared-memory offsets; act holds slots x 2 buffers of act_bytes (row form: one buffer)
    uint32_t o_act, o_w0, o_w1, o_f32, o_rowtab, o_sitetab, o_spins, o_res, o_bar, o_extra, total;
    // row form (rows = 1, local energies): activations [kc][(xp * Lp + yp) * G + g][16 B] updated in place,
    // rows_total rows per plane; a 4 KB zero block; the MMA lists; the layer images of layers >= 1 sit wimg
    // bytes after the tap-form images
    int rows, rows_total;
    uint32_t wimg, o_zero, o_mtab;
    // weight loads of layers >= 1: bytes per layer (their stride in the packed image); f8: the row form with
    // e4m3 operands in layers >= 1 (f8bytes per layer image)
    uint32_t wstride, f8bytes;
    int f8;
};

// Row form: per issuer, the MMAs of a layer >= 1 (kMtabLayer entries at
// most) and of layer 0 (kMtab0), precomputed at bind time:
// {A descriptor low word, B descriptor low word relative to the weight
// buffer, TMEM column, instruction descriptor}. Both descriptors' high words
// are the same for every entry (SBO = 128 bytes, tcgen05 version bit).
constexpr int kMtabLayer = 64, kMtab0 = 32;
constexpr uint32_t kMtabBytes = 16u * kIssuers * (kMtabLayer + kMtab0) + 16u * kIssuers;   // + counts

__host__ __device__ inline uint32_t al16(uint32_t v) { return (v + 15u) & ~15u; }

// Bonds enumerated per chunk by the local-energy kernels (all of them up to
// 16 x 16 J1-J2; larger lattices are processed chunk by chunk).
constexpr int kBondChunk = 1024;
__host__ __device__ inline int bond_chunk(const Problem &p) { return p.n_bonds < kBondChunk ? p.n_bonds : kBondChunk; }

struct TcShared {
    unsigned char *base;
    uint64_t *bar_w;             // [2] weight buffers
    uint64_t *bar_tile;          // [slots][kMaxTiles] per-tile MMA completion
    uint32_t *tmem_addr;
    int *abort_flag;
    int8_t *spins;               // [slots][G][N] the groups' configurations
    const uint2 *rowtab;         // [n_tiles * 128] destination rows of each output row
    const uint2 *sitetab;        // [N] padded positions of each site (main + images)
    float *f32;                  // biases [n_layers][C], head [2][C]
    double *res;                 // [slots][2][G]: a, then phi
};

struct TcState {        // per-CTA pipeline state (all threads keep identical copies)
    uint32_t tphase;    // parity of tile barrier t of slot s at bit s * kMaxTiles + t
    uint32_t wseq;      // weight load used by the next forward's layer 0
    uint32_t wissued;   // weight loads issued so far
    uint32_t wbase;     // first weight load of the bound problem (load q holds layer (q - wbase) mod n_layers)
};

// Rows a group computes, layer by layer: a connected configuration differs
// from its sample in two sites, so layer l's output (0-based) differs from
// the sample's own activations only within distance l + 1 of them (the cone
// of Sec. 5.4.1's local energy). The two sites lie in one row (class 0) or
// in adjacent rows (class 1); every configuration of a group shares the
// class and is rolled along y so that its pair sits at canonical row `top`
// (and top + 1). Layer l then computes canonical rows top - (l + 1) ...
// top + cls + l + 1 only; rows outside that band hold the sample's own
// activations, rolled by the same amount and copied in from a per-block
// cache. The convolution is translation invariant with periodic padding, so
// every value equals bitwise what the dense forward of the unrolled
// configuration computes. cls < 0: dense (every row of every layer).
struct Band {
    int cls, top;
    const int *roll;     // [G]: original row = (canonical row + roll[g]) mod L
};

__device__ __forceinline__ Band dense_band() { return Band{-1, 0, nullptr}; }

// Band rows [lo, hi] of layer l; false if the layer is computed densely
// (dense group, last layer, or the band spans the lattice).
__device__ __forceinline__ bool band_rows(const TcPlan &pl, const Band &b, int l, int &lo, int &hi) {
    if (b.cls < 0 || l >= pl.n_layers - 1) return false;
    lo = b.top - (l + 1);
    hi = b.top + b.cls + (l + 1);
    return lo >= 0 && hi <= pl.L - 1 && hi - lo + 1 < pl.L;
}

// Tiles [t0, t1) holding layer l's rows.
__device__ __forceinline__ void band_tiles(const TcPlan &pl, const Band &b, int l, int &t0, int &t1) {
    int lo, hi;
    t0 = 0;
    t1 = pl.n_tiles;
    if (!band_rows(pl, b, l, lo, hi)) return;
    const int first = ((lo + 1) * pl.Lp + 1) * pl.G, last = ((hi + 1) * pl.Lp + pl.L) * pl.G + pl.G - 1;
    t0 = (first - pl.r0) >> 7;
    t1 = min(pl.n_tiles, ((last - pl.r0) >> 7) + 1);
}

// Per-block cache of the sample's activations, layers 0 .. n_layers - 2, in
// padded positions: [layer][Lp * Lp][C / 8 planes][16 bytes].
__host__ __device__ inline size_t sigma_cache_bytes(const TcPlan &pl) {
    const size_t b = (size_t)(pl.n_layers - 1) * pl.Lp * pl.Lp * pl.C * 2;
    return (b + 255) & ~(size_t)255;
}

// Barriers, TMEM address and abort flag sit at a fixed offset (0) so that a
// block can re-bind to another problem without re-initialising them.
constexpr uint32_t kBarBytes = 8 * (2 + kMaxSlots * kMaxTiles) + 16;

__device__ __forceinline__ uint32_t act_addr(const TcPlan &pl, const TcShared &sh, int slot, int b) {
    return ptx::smem_u32(sh.base + pl.o_act + (uint32_t)(slot * 2 + b) * pl.act_bytes);
}

__device__ __forceinline__ const unsigned char *tc_layer_weights(const TcPlan &pl, const unsigned char *packed, int l) {
    return packed + pl.f32_bytes + (l == 0 ? 0 : pl.w0bytes + pl.wimg + (size_t)(l - 1) * pl.wstride);
}

// Issue the bulk copy of weight-load number q (layer (q - wbase) mod n_layers).
__device__ __forceinline__ void issue_weight_load(const TcPlan &pl, const TcShared &sh, const unsigned char *packed,
                                                  uint32_t q, uint32_t wbase) {
    const int l = (int)((q - wbase) % (uint32_t)pl.n_layers);
    const int b = q & 1;
    const uint32_t bytes = l == 0 ? pl.w0bytes : pl.wstride;
    unsigned char *dst = sh.base + (b ? pl.o_w1 : pl.o_w0);
    ptx::mbar_arrive_expect_tx(&sh.bar_w[b], bytes);
    ptx::bulk_g2s(dst, tc_layer_weights(pl, packed, l), bytes, &sh.bar_w[b]);
}

// Wait on an mbarrier phase; gives up when another thread raised the abort
// flag or after the iteration limit.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, const int *abort_flag,
                                              long long limit = ptx::kWaitLimit) {
    for (long long it = 0; it < limit; ++it) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && *(volatile const int *)abort_flag) return false;
    }
    return false;
}

// Wait on an mbarrier phase the tensor core completes after many cycles (a
// layer's or a tile's MMAs): sleeping try_waits instead of polling, so the
// waiting epilogue warps leave the issue slots to the warps that work.
// Gives up when another thread raised the abort flag or after the time limit.
__device__ __forceinline__ bool wait_sleep_or_abort(uint64_t *bar, uint32_t parity, const int *abort_flag) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    for (long long it = 0; it < ptx::kWaitLimit; ++it) {
        if (ptx::mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (*(volatile const int *)abort_flag) return false;
        if (ptx::globaltimer_ns() - t0 > ptx::kSleepWaitLimitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void raise_abort(const TcShared &sh, int *err) {
    atomicOr(sh.abort_flag, 1);
    atomicOr(err, ERRBIT_TIMEOUT);
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

// Layer-0 im2col matrix of a slot (row = output row, K0 columns: tap-major,
// one-hot channel minor; zero padded) into the slot's second activation
// buffer. Each interior output row reads its 3 x 3 neighbourhood straight
// from the configuration (periodic wrap by index arithmetic).
__device__ void build_slot(const TcPlan &pl, const TcShared &sh, int slot, const Band &band,
                           const SwapSrc *swap = nullptr) {
    const int G = pl.G, L = pl.L, Lp = pl.Lp;
    const int8_t *spins = swap ? swap->cfg : sh.spins + slot * G * pl.N;
    const int si = swap ? swap->i : -1, sj = swap ? swap->j : -1;
    const uint32_t a0 = act_addr(pl, sh, slot, 1);
    const uint32_t one = 0x3F80u, minus_one = 0xBF80u;   // bf16 +1, -1
    int t0, t1;
    band_tiles(pl, band, 0, t0, t1);
    for (int lr = t0 * 128 + (int)threadIdx.x; lr < t1 * 128; lr += blockDim.x) {
        const uint32_t main = sh.rowtab[lr].x & 0xFFFFu;
        const uint32_t row = (uint32_t)(pl.r0 + lr);
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) w[i] = 0u;
        if (main != kNone) {
            const int pos = (int)main / G, g = (int)main - pos * G;
            const int y = pos / Lp - 1, x = pos - (y + 1) * Lp - 1;
            const int8_t *sp = spins + g * pl.N;
            const int yr[3] = {(y == 0 ? L - 1 : y - 1) * L, y * L, (y == L - 1 ? 0 : y + 1) * L};
            const int xc[3] = {x == 0 ? L - 1 : x - 1, x, x == L - 1 ? 0 : x + 1};
            int sv[9];
#pragma unroll
            for (int o = 0; o < 9; ++o) {
                const int site = yr[o / 3] + xc[o % 3];
                sv[o] = sp[site == si ? sj : (site == sj ? si : site)];
            }
#pragma unroll
            for (int o = 0; o < 9; ++o) {
                const int sval = sv[o];
                if (pl.c_in == 1) {
                    const uint32_t bv = sval > 0 ? one : minus_one;
                    w[o >> 1] |= bv << (16 * (o & 1));
                } else {
                    // one-hot channel (hole, up, down) = column 3 o + channel; every index is a
                    // compile-time constant, so w stays in registers
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        const int k = 3 * o + ch;
                        const bool hit = ch == 0 ? sval == 0 : (ch == 1 ? sval == 1 : sval == -1);
                        if (hit) w[k >> 1] |= one << (16 * (k & 1));
                    }
                }
            }
        }
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
            if (kc < pl.K0 / 8)
                ptx::st_shared_v4(a0 + kc * pl.plane + row * 16u, w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
    }
    ptx::fence_async_smem();
    __syncthreads();
}

// Issue the MMAs of layer l for one slot (issuer warps: the whole warp runs
// the loop, one elected lane issues).
template <int C>
__device__ void issue_layer(const TcPlan &pl, const TcShared &sh, const unsigned char *packed, TcState &st, int slot,
                            int l, int *err, const Band &band) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = st.wseq + (uint32_t)l;
    const int iw = warp - pl.epi;   // issuer index
    if (iw >= 0 && iw < kIssuers) {
        if (__all_sync(0xffffffffu, wait_or_abort(&sh.bar_w[q & 1], (q >> 1) & 1, sh.abort_flag))) {
            // the last slot prefetches the next load into the other buffer (its previous user, load q - 1, has
            // completed for every slot); the last issuer does it, so issuer 0's MMAs start at once (a one-tile
            // plan leaves that warp free; the bulk copy takes about 370 cycles to issue)
            if (lane == 0 && iw == kIssuers - 1 && slot == pl.slots - 1)
                issue_weight_load(pl, sh, packed, q + 1, st.wbase);
            ptx::tc_fence_after();
            const uint32_t tmem = *sh.tmem_addr + (uint32_t)(slot * pl.slot_cols);
            const uint32_t wb = ptx::smem_u32(sh.base + ((q & 1) ? pl.o_w1 : pl.o_w0));
            const uint64_t b_base = ptx::smem_desc(wb, C * 16, 128);
            const uint32_t idesc = ptx::idesc_bf16(128, C);
            int t0, t1;
            band_tiles(pl, band, l, t0, t1);
            if (l == 0) {
                const uint64_t a_base = ptx::smem_desc(act_addr(pl, sh, slot, 1), pl.plane, 128);
                for (int t = t0 + iw; t < t1; t += kIssuers) {
                    const uint32_t arow = (uint32_t)(pl.r0 + t * 128);
                    for (int kk = 0; kk < pl.K0 / 16; ++kk)
                        ptx::mma_bf16_elect(tmem + (uint32_t)(t * C), a_base + ((arow * 16u + (uint32_t)(2 * kk) * pl.plane) >> 4),
                                      b_base + (uint64_t)((2 * kk * C * 16) >> 4), idesc, kk ? 1u : 0u);
                    ptx::mma_commit_elect(&sh.bar_tile[slot * kMaxTiles + t]);
                }
            } else {
                const uint64_t a_base = ptx::smem_desc(act_addr(pl, sh, slot, (l - 1) & 1), pl.plane, 128);
                uint32_t offs[9];
#pragma unroll
                for (int o = 0; o < 9; ++o) offs[o] = (uint32_t)(pl.r0 + ((o / 3 - 1) * pl.Lp + (o % 3 - 1)) * pl.G);
                for (int t = t0 + iw; t < t1; t += kIssuers) {
                    const uint32_t d = tmem + (uint32_t)(t * C);
#pragma unroll
                    for (int o = 0; o < 9; ++o) {
                        const uint32_t arow = offs[o] + (uint32_t)(t * 128);
#pragma unroll
                        for (int kk = 0; kk < C / 16; ++kk) {
                            const uint64_t ad = a_base + ((arow * 16u + (uint32_t)(2 * kk) * pl.plane) >> 4);
                            const uint64_t bd = b_base + (uint64_t)(((o * (C / 8) + 2 * kk) * C * 16) >> 4);
                            ptx::mma_bf16_elect(d, ad, bd, idesc, (o | kk) ? 1u : 0u);
                        }
                    }
                    ptx::mma_commit_elect(&sh.bar_tile[slot * kMaxTiles + t]);
                }
            }
        } else if (lane == 0) {
            raise_abort(sh, err);
        }
    }
    if (slot == pl.slots - 1) st.wissued = q + 2;
}

// Epilogue of layer l for one slot: per tile as soon as its MMAs complete,
// bias + SiLU, then bf16 rows (and halo images) or, after the last layer,
// head contributions. Ends with a block barrier. False on abort.
template <int C>
__device__ bool epilogue_layer(const TcPlan &pl, const TcShared &sh, TcState &st, int slot, int l, int *err,
                               const Band &band, const unsigned char *cache, unsigned char *cache_w) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3;
    const bool last = l == pl.n_layers - 1;
    const uint32_t tmem = *sh.tmem_addr + (uint32_t)(slot * pl.slot_cols);
    const float *bias = sh.f32 + l * C;
    const float *wa = sh.f32 + pl.n_layers * C;
    const uint32_t out = act_addr(pl, sh, slot, l & 1);
    float *contrib = reinterpret_cast<float *>(sh.base + pl.o_act + (uint32_t)(slot * 2 + (l & 1)) * pl.act_bytes);
    // halved biases in registers for 16 channels (for 32 the registers are
    // kept for two co-resident blocks; the loads stay in the loop)
    constexpr int HB = C == 16 ? C : 1;
    float hb[HB];
#pragma unroll
    for (int c = 0; c < HB; ++c) hb[c] = 0.5f * bias[c];
    int t0, t1, lo = 0, hi = 0;
    band_tiles(pl, band, l, t0, t1);
    const bool banded = band_rows(pl, band, l, lo, hi);
    const uint32_t mlo = banded ? (uint32_t)((lo + 1) * pl.Lp * pl.G) : 0u;
    const uint32_t mhi = banded ? (uint32_t)((hi + 2) * pl.Lp * pl.G) : kNone;
    const int Lp2 = pl.Lp * pl.Lp;
    constexpr int KC = C / 8;
    if (banded && warp < pl.epi) {
        // Rows the next layer reads that this layer does not compute: the
        // sample's layer-l activations, rolled into each configuration's
        // frame (with their periodic images), copied asynchronously from the
        // cache while the tiles below are processed (waited for before the
        // layer's closing barrier); disjoint from the band rows they write.
        int nlo, nhi;
        const bool next_banded = band_rows(pl, band, l + 1, nlo, nhi);
        const int width = hi - lo + 1;
        const int nf = next_banded ? 4 : pl.L - width;
        const int items = pl.G * nf * pl.L;
        for (int it = (int)threadIdx.x; it < items; it += 32 * pl.epi) {
            const int q = it / pl.L, x = it - q * pl.L;
            const int g = q / nf, f = q - g * nf;
            int yc;
            if (next_banded) yc = f < 2 ? lo - 2 + f : hi - 1 + f;   // lo - 2, lo - 1, hi + 1, hi + 2
            else yc = f < lo ? f : f + width;
            yc = (yc + pl.L) % pl.L;
            int ys = yc + band.roll[g];
            if (ys >= pl.L) ys -= pl.L;
            const uint32_t src_pos = sh.sitetab[ys * pl.L + x].x & 0xFFFFu;
            const unsigned char *src = cache + (size_t)(l * Lp2 + (int)src_pos) * KC * 16;
            const uint2 d = sh.sitetab[yc * pl.L + x];
            const uint32_t dp[4] = {d.x & 0xFFFFu, d.x >> 16, d.y & 0xFFFFu, d.y >> 16};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (dp[i] != kNone)
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc)
                        ptx::cp_async16(out + (uint32_t)kc * pl.plane + (dp[i] * (uint32_t)pl.G + (uint32_t)g) * 16u,
                                        src + kc * 16);
        }
    }
    bool ok = true;
    for (int t = t0 + (warp >> 2); warp < pl.epi && t < t1; t += pl.epi / 4) {
        const uint32_t parity = (st.tphase >> (slot * kMaxTiles + t)) & 1u;
        const uint2 dst = sh.rowtab[t * 128 + quarter * 32 + lane];
        const bool got = wait_sleep_or_abort(&sh.bar_tile[slot * kMaxTiles + t], parity, sh.abort_flag);
        if (!__all_sync(0xffffffffu, got)) { ok = false; break; }   // reconverges the warp
        ptx::tc_fence_after();
        uint32_t r[C / 16][16];
#pragma unroll
        for (int h = 0; h < C / 16; ++h)
            ptx::tmem_ld16_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * C + 16 * h), r[h]);
        ptx::tmem_wait_ld();
        float v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = __uint_as_float(r[c >> 4][c & 15]);
        const uint32_t main = dst.x & 0xFFFFu;
        if (main == kNone || main < mlo || main >= mhi) continue;   // halo, or outside the band
        if (!last) {
            uint32_t w[C / 2];
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
                const float h0 = C == 16 ? hb[(2 * c) % HB] : 0.5f * bias[2 * c];
                const float h1 = C == 16 ? hb[(2 * c + 1) % HB] : 0.5f * bias[2 * c + 1];
                if constexpr (C == 16) {   // packed pairs (32 channels: scalar, fewer live registers)
                    const float2 o = ptx::silu_bias2(make_float2(v[2 * c], v[2 * c + 1]), make_float2(h0, h1));
                    w[c] = ptx::pack_bf16(o.x, o.y);
                } else {
                    w[c] = ptx::pack_bf16(ptx::silu_bias(v[2 * c], h0), ptx::silu_bias(v[2 * c + 1], h1));
                }
            }
            if (!NQS_INDEX_OK(((dst.x & 0xFFFFu) == kNone || (dst.x & 0xFFFFu) < (uint32_t)pl.rbuf) &&
                                  ((dst.x >> 16) == kNone || (dst.x >> 16) < (uint32_t)pl.rbuf) &&
                                  ((dst.y & 0xFFFFu) == kNone || (dst.y & 0xFFFFu) < (uint32_t)pl.rbuf) &&
                                  ((dst.y >> 16) == kNone || (dst.y >> 16) < (uint32_t)pl.rbuf), err))
                continue;
            store_rows<C>(pl, out, dst, w);
            if (cache_w) {   // the sample itself (configuration 0) fills the cache
                const uint32_t pos = main / (uint32_t)pl.G;
                if (main == pos * (uint32_t)pl.G) {
                    uint4 *c4 = reinterpret_cast<uint4 *>(cache_w + (size_t)(l * Lp2 + (int)pos) * KC * 16);
#pragma unroll
                    for (int kc = 0; kc < KC; ++kc) c4[kc] = make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
                }
            }
        } else {
            // biases and head weights as 16-byte broadcast loads (the fp32 block is 16-byte aligned and every
            // offset a multiple of 16 floats); the sums run over c = 0 .. C - 1 in order as before
            float ca = 0.f, cp = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < C; c4 += 4) {
                const float4 xa = *reinterpret_cast<const float4 *>(wa + c4);
                const float4 xp = *reinterpret_cast<const float4 *>(wa + C + c4);
                const float aa[4] = {xa.x, xa.y, xa.z, xa.w}, pp[4] = {xp.x, xp.y, xp.z, xp.w};
                float hv[4];
                if constexpr (C == 16) {
                    // SiLU(v + b) from the halved biases held in registers: fma(0.5, v, b / 2) rounds to the
                    // value 0.5 (v + b) rounds to (scaling by 2 is exact), so the result is that of silu_fast
                    const float2 h01 = ptx::silu_bias2(make_float2(v[c4], v[c4 + 1]), make_float2(hb[c4], hb[c4 + 1]));
                    const float2 h23 = ptx::silu_bias2(make_float2(v[c4 + 2], v[c4 + 3]),
                                                       make_float2(hb[c4 + 2], hb[c4 + 3]));
                    hv[0] = h01.x, hv[1] = h01.y, hv[2] = h23.x, hv[3] = h23.y;
                } else {
                    const float4 b = *reinterpret_cast<const float4 *>(bias + c4);
                    const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) hv[k] = ptx::silu_fast(v[c4 + k] + bb[k]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    ca = fmaf(aa[k], hv[k], ca);
                    cp = fmaf(pp[k], hv[k], cp);
                }
            }
            // configuration-major in site order ([a | phi][g][y L + x]), so that the head reads one
            // configuration's sites as consecutive words
            const uint32_t pos = main / (uint32_t)pl.G, g = main - pos * (uint32_t)pl.G;
            const uint32_t yy = pos / (uint32_t)pl.Lp - 1u, xx = pos - (yy + 1u) * (uint32_t)pl.Lp - 1u;
            const uint32_t idx = g * (uint32_t)pl.N + yy * (uint32_t)pl.L + xx;
            contrib[idx] = ca;
            contrib[(uint32_t)(pl.G * pl.N) + idx] = cp;
        }
    }
    if (!ok) raise_abort(sh, err);
    st.tphase ^= (((1u << (t1 - t0)) - 1u) << t0) << (slot * kMaxTiles);
    if (banded) ptx::cp_async_wait_all();   // the fill's copies have landed
    ptx::tc_fence_before();
    ptx::fence_async_smem();
    __syncthreads();
    return *(volatile int *)sh.abort_flag == 0;
}

// a[g] = sum over sites of the head contributions (one warp per g, fixed
// order: lane k sums sites k, k + 32, ... in order, then an xor-shuffle tree).
// contrib: [a | phi][g][site y L + x], as the last layer's epilogue stores
// them; roll: rows by which each configuration was rolled (or null).
__device__ void head_slot(const TcPlan &pl, const TcShared &sh, int slot, const int *roll, const float *contrib) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, G = pl.G, N = pl.N;
    double *res = sh.res + slot * 2 * G;
    for (int g = warp; g < G; g += (int)(blockDim.x >> 5)) {
        float sa = 0.f, sp = 0.f;
        const int rg = roll ? roll[g] : 0;
        for (int site = lane; site < pl.N; site += 32) {
            // sum in the original site order, whatever frame the configuration was evaluated in
            int cs = site;
            if (rg) {
                const int y = site / pl.L, x = site - y * pl.L;
                cs = ((y - rg + pl.L) % pl.L) * pl.L + x;
            }
            const int idx = g * N + cs;
            sa += contrib[idx];
            sp += contrib[G * N + idx];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sp += __shfl_xor_sync(0xffffffffu, sp, o);
        }
        if (lane == 0) {
            res[g] = (double)sa;
            res[G + g] = (double)sp;
        }
    }
    __syncthreads();
}

// Evaluate every slot's G configurations (sh.spins); results in sh.res.
// Returns false if a wait timed out (the block must stop).
// band: rows per layer (one slot only; dense_band() otherwise); cache: the
// sample's activations (read by banded groups); cache_w: where a dense group
// holding the sample as configuration 0 of slot 0 stores them (or null).
template <int C>
__device__ bool tc_forward(const TcPlan &pl, const TcShared &sh, const unsigned char *packed, TcState &st, int *err,
                           const Band &band = dense_band(), const unsigned char *cache = nullptr,
                           unsigned char *cache_w = nullptr, const SwapSrc *swap = nullptr) {
    for (int s = 0; s < pl.slots; ++s) {
        build_slot(pl, sh, s, band, swap);
        issue_layer<C>(pl, sh, packed, st, s, 0, err, band);
    }
    for (int l = 0; l < pl.n_layers; ++l) {
        for (int s = 0; s < pl.slots; ++s) {
            if (!epilogue_layer<C>(pl, sh, st, s, l, err, band, cache, s == 0 ? cache_w : nullptr)) return false;
            if (l + 1 < pl.n_layers) issue_layer<C>(pl, sh, packed, st, s, l + 1, err, band);
            else head_slot(pl, sh, s, band.roll,
                           reinterpret_cast<const float *>(sh.base + pl.o_act +
                                                           (uint32_t)(s * 2 + ((pl.n_layers - 1) & 1)) * pl.act_bytes));
        }
    }
    st.wseq += (uint32_t)pl.n_layers;
    return true;
}

// ---------------------------------------------------------------- row form (local energies)
// The tap form above issues one N = C MMA per 3x3 tap and output tile, so
// every A byte (128 rows x 16 channels) feeds only C MACs and the shared-
// memory operand path bounds it. The row form lays a group's activations out
// as rows m = y * G + g (lattice row, configuration) and puts the x positions
// along tensor-memory columns: D[m][x * C + c]. For one padded input column
// xp and one kernel row dy, a single MMA with N = 3C (the three dx taps'
// weights side by side) writes its three column blocks onto the outputs
// x = xp - 2, xp - 1, xp (the TMEM column offset does the dx shift), so an
// A operand serves 3C outputs per row. Per layer: one zeroing MMA per issuer,
// then 3 (dy) x (L + 2) (xp) MMAs. Each output still accumulates its taps in
// the tap form's order (dy, then dx, then the K halves), onto a zeroed
// accumulator. Layer 0 keeps the tap form's 9-tap im2col (K = 16 or 32,
// N = C) per x. All MMAs of a layer complete before its epilogue writes, so
// one activation buffer is updated in place. The two issuing warps take the
// left and right halves of the output columns (disjoint accumulators); the
// epilogue warps take a TMEM lane quarter and every other column each.

__device__ __forceinline__ uint32_t row_act(const TcPlan &pl, const TcShared &sh) {
    return ptx::smem_u32(sh.base + pl.o_act);
}

// Low 32 bits of a no-swizzle smem descriptor (start address and LBO, both
// in 16-byte units); the high word is kDescHi for every operand here.
__device__ __forceinline__ uint32_t desc_lo(uint32_t saddr, uint32_t lbo) {
    return ((saddr & 0x3FFFFu) >> 4) | (((lbo & 0x3FFFFu) >> 4) << 16);
}
constexpr uint32_t kDescHi = (128u >> 4) | (1u << 14);   // SBO = 128 B; bit 46: descriptor version

// Issuer iw's MMA lists (called by the issuer lane at bind time). Layer >= 1:
// per kernel row dy and input column xp in [xa, xb + 1], the outputs
// lo .. hi = max(xp - 2, xa) .. min(xp, xb - 1) with weight blocks from
// j0 = 2 - xp + lo, K halves innermost: every output sees its taps in the
// tap form's order (dy, then dx, then K). The padded columns 0 and L + 1 are
// the periodic images of columns L and 1, so the A operands are read there
// and the images are never stored.
template <int C>
__device__ void row_build_mtab(const TcPlan &pl, const TcShared &sh, int iw) {
    uint4 *tab = reinterpret_cast<uint4 *>(sh.base + pl.o_mtab) + iw * (kMtabLayer + kMtab0);
    int *cnt = reinterpret_cast<int *>(sh.base + pl.o_mtab + 16u * kIssuers * (kMtabLayer + kMtab0)) + 2 * iw;
    const uint32_t act = row_act(pl, sh);
    const int xa = iw * pl.L / kIssuers, xb = (iw + 1) * pl.L / kIssuers;
    constexpr int KC = C / 8;
    int n = 0;
    if (pl.f8) {
        // e4m3 (16 channels): per kernel-row pair q and input column, one K = 32 MMA whose two K halves are
        // kernel rows 2 q and 2 q + 1, G rows apart in the activations (the A operand's K stride); the B image
        // holds zeros for kernel row 3
        for (int q = 0; q < 2; ++q)
            for (int xp = xa; xp <= xb + 1; ++xp) {
                const int lo = max(xp - 2, xa), hi = min(xp, xb - 1);
                const int j0 = 2 - xp + lo;
                const int xs = xp == 0 ? pl.L : (xp == pl.L + 1 ? 1 : xp);
                const uint32_t arow = (uint32_t)((xs * pl.Lp + 2 * q) * pl.G);
                const uint32_t boff = (uint32_t)((2 * q * 3 * C + j0 * C) * 16);
                tab[n++] = make_uint4(desc_lo(act + arow * 16u, (uint32_t)pl.G * 16u), desc_lo(boff, 3 * C * 16),
                                      (uint32_t)(lo * C), ptx::idesc_e4m3(128, (hi - lo + 1) * C));
            }
    }
    for (int dy = 0; dy < 3 && !pl.f8; ++dy)
        for (int xp = xa; xp <= xb + 1; ++xp) {
            const int lo = max(xp - 2, xa), hi = min(xp, xb - 1);
            const int j0 = 2 - xp + lo;
            const int xs = xp == 0 ? pl.L : (xp == pl.L + 1 ? 1 : xp);
            const uint32_t arow = (uint32_t)((xs * pl.Lp + dy) * pl.G);
            for (int kk = 0; kk < C / 16; ++kk) {
                const uint32_t boff = (uint32_t)(((dy * KC + 2 * kk) * 3 * C + j0 * C) * 16);
                tab[n++] = make_uint4(desc_lo(act + arow * 16u + (uint32_t)(2 * kk) * pl.plane, pl.plane),
                                      desc_lo(boff, 3 * C * 16), (uint32_t)(lo * C),
                                      ptx::idesc_bf16(128, (hi - lo + 1) * C));
            }
        }
    cnt[0] = n;
    int n0 = 0;
    for (int x = xa; x < xb; ++x)
        for (int kk = 0; kk < pl.K0 / 16; ++kk)
            tab[kMtabLayer + n0++] = make_uint4(desc_lo(act + (uint32_t)x * 128u * 16u + (uint32_t)(2 * kk) * pl.plane,
                                                        pl.plane),
                                                desc_lo((uint32_t)(2 * kk * C * 16), C * 16),
                                                (uint32_t)(x * C) | (kk ? 0x80000000u : 0u), ptx::idesc_bf16(128, C));
    cnt[1] = n0;
}

// Spins of the group to the layer-0 im2col: row x * 128 + m (m = y * G + g),
// K0 columns tap-major (one-hot channel minor), as build_slot writes them.
// Threads 0 .. 255 each keep one accumulator row m and walk every other
// column x; the 3 x 3 neighbourhood comes from the row's three lattice rows.
__device__ void build_rows(const TcPlan &pl, const TcShared &sh) {
    const int G = pl.G, N = pl.N, L = pl.L;
    const uint32_t a0 = row_act(pl, sh);
    const uint32_t one = 0x3F80u, minus_one = 0xBF80u;   // bf16 +1, -1
    if (threadIdx.x < 256) {
        const int m = threadIdx.x & 127;
        const bool valid = m < G * L;
        const int y = valid ? m / G : 0, g = valid ? m - y * G : 0;
        const int8_t *sp = sh.spins + g * N;
        const int yr[3] = {(y == 0 ? L - 1 : y - 1) * L, y * L, (y == L - 1 ? 0 : y + 1) * L};
        for (int x = (int)(threadIdx.x >> 7); x < L; x += 2) {
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) w[i] = 0u;
            if (valid) {
                const int xc[3] = {x == 0 ? L - 1 : x - 1, x, x == L - 1 ? 0 : x + 1};
                int sv[9];
#pragma unroll
                for (int o = 0; o < 9; ++o) sv[o] = sp[yr[o / 3] + xc[o % 3]];
#pragma unroll
                for (int o = 0; o < 9; ++o) {
                    const int sval = sv[o];
                    if (pl.c_in == 1) {
                        const uint32_t b = sval > 0 ? one : minus_one;
                        w[o >> 1] |= b << (16 * (o & 1));
                    } else {
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            const int k = 3 * o + ch;
                            const bool hit = ch == 0 ? sval == 0 : (ch == 1 ? sval == 1 : sval == -1);
                            if (hit) w[k >> 1] |= one << (16 * (k & 1));
                        }
                    }
                }
            }
            const uint32_t row = (uint32_t)(x * 128 + m);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc)
                if (kc < pl.K0 / 8)
                    ptx::st_shared_v4(a0 + kc * pl.plane + row * 16u, w[4 * kc], w[4 * kc + 1], w[4 * kc + 2],
                                      w[4 * kc + 3]);
        }
    }
    ptx::fence_async_smem();
    __syncthreads();
}

// Issue layer l's MMAs (issuer warps: the whole warp runs the loop, one
// elected lane issues): issuer iw owns output columns
// x in [iw L / kIssuers, (iw + 1) L / kIssuers) and commits to bar_tile[iw].
template <int C, bool F8 = false>
__device__ void row_issue(const TcPlan &pl, const TcShared &sh, const unsigned char *packed, TcState &st, int l,
                          int *err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = st.wseq + (uint32_t)l;
    const int iw = warp - pl.epi;
    if (iw >= 0 && iw < kIssuers) {
        if (__all_sync(0xffffffffu, wait_or_abort(&sh.bar_w[q & 1], (q >> 1) & 1, sh.abort_flag))) {
            ptx::tc_fence_after();
            const uint32_t tmem = *sh.tmem_addr;
            const uint32_t wb = ptx::smem_u32(sh.base + ((q & 1) ? pl.o_w1 : pl.o_w0));
            const uint4 *tab = reinterpret_cast<const uint4 *>(sh.base + pl.o_mtab) + iw * (kMtabLayer + kMtab0);
            const int *cnt = reinterpret_cast<const int *>(sh.base + pl.o_mtab +
                                                           16u * kIssuers * (kMtabLayer + kMtab0)) + 2 * iw;
            const uint32_t wlo = wb >> 4;   // weight buffer start in 16-byte units, added to the B entries
            if (l == 0) {
                const int n0 = cnt[1];
                for (int k = 0; k < n0; ++k) {
                    const uint4 e = tab[kMtabLayer + k];
                    ptx::mma_bf16_elect(tmem + (e.z & 0x7FFFFFFFu), ((uint64_t)kDescHi << 32) | e.x,
                                  ((uint64_t)kDescHi << 32) | (e.y + wlo), e.w, e.z >> 31);
                }
            } else {
                // zero this issuer's accumulators: A = B = the zero block, N = its columns
                const int xa = iw * pl.L / kIssuers, xb = (iw + 1) * pl.L / kIssuers;
                const uint64_t z = ((uint64_t)kDescHi << 32) | desc_lo(ptx::smem_u32(sh.base + pl.o_zero), 2048);
                ptx::mma_bf16_elect(tmem + (uint32_t)(xa * C), z, z, ptx::idesc_bf16(128, (xb - xa) * C), 0u);
                const int n = cnt[0];
#pragma unroll 4
                for (int k = 0; k < n; ++k) {
                    const uint4 e = tab[k];
                    if constexpr (F8)
                        ptx::mma_e4m3_elect(tmem + e.z, ((uint64_t)kDescHi << 32) | e.x,
                                            ((uint64_t)kDescHi << 32) | (e.y + wlo), e.w, 1u);
                    else
                        ptx::mma_bf16_elect(tmem + e.z, ((uint64_t)kDescHi << 32) | e.x, ((uint64_t)kDescHi << 32) | (e.y + wlo),
                                      e.w, 1u);
                }
            }
            ptx::mma_commit_elect(&sh.bar_tile[iw]);
            // next layer's weights into the other buffer (last read by layer q - 1's MMAs, completed), after
            // this layer's MMAs are issued
            if (lane == 0 && iw == 0) issue_weight_load(pl, sh, packed, q + 1, st.wbase);
        } else if (lane == 0) {
            raise_abort(sh, err);
        }
    }
    st.wissued = q + 2;
}

// TMEM columns [col, col + C) of this warp's lane quarter into r (no wait).
template <int C>
__device__ __forceinline__ void row_ld(uint32_t taddr, uint32_t (&r)[C / 16][16]) {
#pragma unroll
    for (int hh = 0; hh < C / 16; ++hh) ptx::tmem_ld16_nowait(taddr + (uint32_t)(16 * hh), r[hh]);
}
template <int C>
__device__ __forceinline__ void row_wait(uint32_t (&r)[C / 16][16]) {
    ptx::tmem_wait_ld();
#pragma unroll
    for (int hh = 0; hh < C / 16; ++hh) ptx::reg_fence16(r[hh]);
}

// One output column x of one row (y, g): bias + SiLU to bf16, stored at the
// padded position and its periodic image along y (the MMAs read the x images
// from the columns themselves); or, after the last layer, the head
// contributions of the position. The bf16 stores go to amain (the row's
// address at padded column 0) plus the column's offset, and dimg bytes
// further for the image; the e4m3 stores address act by row index.
template <int C, bool F8 = false>
__device__ __forceinline__ void row_out(const TcPlan &pl, uint32_t act, uint32_t amain, int dimg, float *contrib,
                                        const float *bias, const float *wa, const float (&hb)[C == 16 ? C : 1],
                                        bool last, int x, int y, int yimg, int g, const uint32_t (&r)[C / 16][16],
                                        int *err, const float *scl = nullptr) {
    constexpr int KC = C / 8, HB = C == 16 ? C : 1;
    const int G = pl.G, L = pl.L, Lp = pl.Lp;
    float v[C];
#pragma unroll
    for (int c = 0; c < C; ++c) v[c] = __uint_as_float(r[c >> 4][c & 15]);
    if constexpr (F8) {
        if (!last) {
            // e4m3 outputs (16 channels): SiLU(s v + b) with s the layer's weight scale of the channel (1 in
            // layer 0), computed as z / 2 = (s / 2) v + b / 2 from the halved scales; saturated to +-448, 16
            // bytes a row
            uint32_t w[4];
#pragma unroll
            for (int c4 = 0; c4 < C; c4 += 4) {
                const float4 s4 = scl ? *reinterpret_cast<const float4 *>(scl + c4) : make_float4(.5f, .5f, .5f, .5f);
                const float ss[4] = {s4.x, s4.y, s4.z, s4.w};
                const float2 o01 = ptx::silu_half2(__ffma2_rn(make_float2(ss[0], ss[1]), make_float2(v[c4], v[c4 + 1]),
                                                              make_float2(hb[c4 % HB], hb[(c4 + 1) % HB])));
                const float2 o23 = ptx::silu_half2(__ffma2_rn(make_float2(ss[2], ss[3]),
                                                              make_float2(v[c4 + 2], v[c4 + 3]),
                                                              make_float2(hb[(c4 + 2) % HB], hb[(c4 + 3) % HB])));
                w[c4 / 4] = ptx::pack_e4m3(o01.x, o01.y) | (ptx::pack_e4m3(o23.x, o23.y) << 16);
            }
            // row addresses from the row index (measured faster here than the precomputed form below)
            const int xp = x + 1;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int yp = b == 0 ? y + 1 : yimg;
                if (yp < 0) continue;
                const uint32_t row = (uint32_t)((xp * Lp + yp) * G + g);
                if (!NQS_INDEX_OK(row < (uint32_t)pl.rows_total, err)) continue;
                ptx::st_shared_v4(act + row * 16u, w[0], w[1], w[2], w[3]);
            }
        } else {
            float ca = 0.f, cp = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < C; c4 += 4) {
                const float4 s4 = scl ? *reinterpret_cast<const float4 *>(scl + c4) : make_float4(.5f, .5f, .5f, .5f);
                const float4 xa = *reinterpret_cast<const float4 *>(wa + c4);
                const float4 xq = *reinterpret_cast<const float4 *>(wa + C + c4);
                const float ss[4] = {s4.x, s4.y, s4.z, s4.w};
                const float aa[4] = {xa.x, xa.y, xa.z, xa.w}, pp[4] = {xq.x, xq.y, xq.z, xq.w};
                // z / 2 = (s / 2) v + b / 2, exactly half of s v + b
                const float2 h01 = ptx::silu_half2(__ffma2_rn(make_float2(ss[0], ss[1]), make_float2(v[c4], v[c4 + 1]),
                                                              make_float2(hb[c4 % HB], hb[(c4 + 1) % HB])));
                const float2 h23 = ptx::silu_half2(__ffma2_rn(make_float2(ss[2], ss[3]),
                                                              make_float2(v[c4 + 2], v[c4 + 3]),
                                                              make_float2(hb[(c4 + 2) % HB], hb[(c4 + 3) % HB])));
                const float hv[4] = {h01.x, h01.y, h23.x, h23.y};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    ca = fmaf(aa[k], hv[k], ca);
                    cp = fmaf(pp[k], hv[k], cp);
                }
            }
            const int idx = g * pl.N + y * L + x;
            contrib[idx] = ca;
            contrib[G * pl.N + idx] = cp;
        }
        return;
    }
    if (!last) {
        uint32_t w[C / 2];
#pragma unroll
        for (int c = 0; c < C / 2; ++c) {
            const float h0 = C == 16 ? hb[(2 * c) % HB] : 0.5f * bias[2 * c];
            const float h1 = C == 16 ? hb[(2 * c + 1) % HB] : 0.5f * bias[2 * c + 1];
            const float2 o = ptx::silu_bias2(make_float2(v[2 * c], v[2 * c + 1]), make_float2(h0, h1));
            w[c] = ptx::pack_bf16(o.x, o.y);
        }
        const int xp = x + 1;
        const uint32_t a = amain + (uint32_t)(xp * Lp * G) * 16u;   // row (xp Lp + y + 1) G + g
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int yp = b == 0 ? y + 1 : yimg;
            if (yp < 0) continue;
            if (!NQS_INDEX_OK((uint32_t)((xp * Lp + yp) * G + g) < (uint32_t)pl.rows_total, err)) continue;
            const uint32_t ab = a + (b == 0 ? 0u : (uint32_t)dimg);
#pragma unroll
            for (int kc = 0; kc < KC; ++kc)
                ptx::st_shared_v4(ab + (uint32_t)kc * pl.plane, w[4 * kc], w[4 * kc + 1], w[4 * kc + 2],
                                  w[4 * kc + 3]);
        }
    } else {
        // the tap form's head arithmetic: c = 0 .. C - 1 in order, 16-byte broadcast loads
        float ca = 0.f, cp = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < C; c4 += 4) {
            const float4 xa = *reinterpret_cast<const float4 *>(wa + c4);
            const float4 xq = *reinterpret_cast<const float4 *>(wa + C + c4);
            const float aa[4] = {xa.x, xa.y, xa.z, xa.w}, pp[4] = {xq.x, xq.y, xq.z, xq.w};
            float2 h01, h23;
            if constexpr (C == 16) {   // the halved biases in registers (the same values, as in the tap form)
                h01 = ptx::silu_bias2(make_float2(v[c4], v[c4 + 1]), make_float2(hb[c4], hb[c4 + 1]));
                h23 = ptx::silu_bias2(make_float2(v[c4 + 2], v[c4 + 3]), make_float2(hb[c4 + 2], hb[c4 + 3]));
            } else {
                const float4 b = *reinterpret_cast<const float4 *>(bias + c4);
                h01 = ptx::silu_fast2(make_float2(v[c4], v[c4 + 1]), make_float2(b.x, b.y));
                h23 = ptx::silu_fast2(make_float2(v[c4 + 2], v[c4 + 3]), make_float2(b.z, b.w));
            }
            const float hv[4] = {h01.x, h01.y, h23.x, h23.y};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ca = fmaf(aa[k], hv[k], ca);
                cp = fmaf(pp[k], hv[k], cp);
            }
        }
        // site order [a | phi][g][y * L + x]
        const int idx = g * pl.N + y * L + x;
        contrib[idx] = ca;
        contrib[G * pl.N + idx] = cp;
    }
}

// Epilogue of layer l: once every MMA of the layer has completed, bias +
// SiLU of each output and its bf16 rows (with periodic images) written back
// into the activation buffer, or after the last layer the head contributions.
// Each thread walks its columns with the next column's TMEM load in flight.
template <int C, bool F8 = false>
__device__ bool row_epilogue(const TcPlan &pl, const TcShared &sh, TcState &st, int l, int *err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quarter = warp & 3;
    const bool last = l == pl.n_layers - 1;
    const int G = pl.G, L = pl.L;
    const float *bias = sh.f32 + l * C;
    // halved e4m3 weight scales of layer l >= 1: after its image in the weight buffer it was loaded into (that buffer
    // is refilled only at the next layer's issue, after this epilogue)
    const uint32_t qw = st.wseq + (uint32_t)l;
    const float *scl = F8 && l > 0 ? reinterpret_cast<const float *>(sh.base + ((qw & 1) ? pl.o_w1 : pl.o_w0) +
                                                                      12 * C * C)
                                   : nullptr;
    const float *wa = sh.f32 + pl.n_layers * C;
    const uint32_t act = row_act(pl, sh);
    float *contrib = reinterpret_cast<float *>(sh.base + pl.o_act);
    bool ok = true;
    if (warp < pl.epi) {
        bool got = true;
        for (int i = 0; i < kIssuers; ++i)
            got = got && wait_sleep_or_abort(&sh.bar_tile[i], (st.tphase >> i) & 1u, sh.abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
            ok = false;
        } else {
            ptx::tc_fence_after();
            const uint32_t tmem = *sh.tmem_addr + ((uint32_t)(quarter * 32) << 16);
            const int m = quarter * 32 + lane;
            const bool valid = m < G * L;
            const int y = valid ? m / G : 0, g = valid ? m - y * G : 0;
            const int yimg = y == 0 ? L + 1 : (y == L - 1 ? 0 : -1);
            // this row's store address at padded column 0 and the byte offset of its periodic image along y
            const uint32_t amain = act + (uint32_t)((y + 1) * G + g) * 16u;
            const int dimg = (yimg - (y + 1)) * G * 16;
            const int nh = pl.epi >> 2, h = warp >> 2;
            float hb[C == 16 ? C : 1];
#pragma unroll
            for (int c = 0; c < (C == 16 ? C : 1); ++c) hb[c] = 0.5f * bias[c];
            uint32_t ra[C / 16][16], rb[C / 16][16];
            // columns x = h, h + nh, ... (interleaved between the groups: measured faster than halves)
            if (h < L) {
                row_ld<C>(tmem + (uint32_t)(h * C), ra);
                row_wait<C>(ra);
            }
            for (int x = h; x < L; x += 2 * nh) {
                const bool more = x + nh < L;
                if (more) row_ld<C>(tmem + (uint32_t)((x + nh) * C), rb);
                if (valid) row_out<C, F8>(pl, act, amain, dimg, contrib, bias, wa, hb, last, x, y, yimg, g, ra, err, scl);
                if (!more) break;
                row_wait<C>(rb);
                const bool more2 = x + 2 * nh < L;
                if (more2) row_ld<C>(tmem + (uint32_t)((x + 2 * nh) * C), ra);
                if (valid) row_out<C, F8>(pl, act, amain, dimg, contrib, bias, wa, hb, last, x + nh, y, yimg, g, rb,
                                          err, scl);
                if (more2) row_wait<C>(ra);
            }
        }
    }
    if (!ok) raise_abort(sh, err);
    st.tphase ^= (1u << kIssuers) - 1u;
    ptx::tc_fence_before();
    ptx::fence_async_smem();
    __syncthreads();
    return *(volatile int *)sh.abort_flag == 0;
}

// Evaluate the group's G configurations (sh.spins) in the row form; results
// in sh.res. False if a wait timed out (the block must stop).
template <int C, bool F8 = false>
__device__ bool row_forward(const TcPlan &pl, const TcShared &sh, const unsigned char *packed, TcState &st, int *err) {
    build_rows(pl, sh);
    row_issue<C, F8>(pl, sh, packed, st, 0, err);
    for (int l = 0; l < pl.n_layers; ++l) {
        if (!row_epilogue<C, F8>(pl, sh, st, l, err)) return false;
        if (l + 1 < pl.n_layers) row_issue<C, F8>(pl, sh, packed, st, l + 1, err);
        else head_slot(pl, sh, 0, nullptr, reinterpret_cast<const float *>(sh.base + pl.o_act));
    }
    st.wseq += (uint32_t)pl.n_layers;
    return true;
}

// ---------------------------------------------------------------- kernel prologue / epilogue
// Once per block: barriers (fixed offset 0), tensor memory.
__device__ void tc_init(TcShared &sh, unsigned char *smem, uint32_t tmem_cols, TcState &st) {
    sh.base = smem;
    sh.bar_w = reinterpret_cast<uint64_t *>(smem);
    sh.bar_tile = sh.bar_w + 2;
    sh.tmem_addr = reinterpret_cast<uint32_t *>(smem + 8 * (2 + kMaxSlots * kMaxTiles));
    sh.abort_flag = reinterpret_cast<int *>(smem + 8 * (2 + kMaxSlots * kMaxTiles) + 4);
    if (threadIdx.x == 0) {
        ptx::mbar_init(&sh.bar_w[0], 1);
        ptx::mbar_init(&sh.bar_w[1], 1);
        for (int t = 0; t < kMaxSlots * kMaxTiles; ++t) ptx::mbar_init(&sh.bar_tile[t], 1);
        *sh.abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        ptx::tmem_alloc(sh.tmem_addr, tmem_cols);
        ptx::tmem_relinquish();
    }
    st.tphase = 0;
    st.wseq = 0;
    st.wissued = 0;
    st.wbase = 0;
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
}

// Bind the block to one problem: shared-memory carve-up, parameters,
// destination tables, zeroed buffers, first weight load.
__device__ void tc_bind(const TcPlan &pl, TcShared &sh, const unsigned char *packed, TcState &st) {
    unsigned char *smem = sh.base;
    sh.spins = reinterpret_cast<int8_t *>(smem + pl.o_spins);
    sh.rowtab = reinterpret_cast<const uint2 *>(smem + pl.o_rowtab);
    sh.sitetab = reinterpret_cast<const uint2 *>(smem + pl.o_sitetab);
    sh.f32 = reinterpret_cast<float *>(smem + pl.o_f32);
    sh.res = reinterpret_cast<double *>(smem + pl.o_res);
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
    // zero the activation buffers: rows outside the lattice are read by
    // discarded output rows only, but keep them finite
    for (uint32_t i = threadIdx.x; i < pl.slots * 2 * pl.act_bytes / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem + pl.o_act)[i] = 0u;
    ptx::fence_async_smem();
    __syncthreads();
    st.wbase = st.wissued;
    st.wseq = st.wissued;
    if (threadIdx.x == 0) issue_weight_load(pl, sh, packed, st.wissued, st.wbase);
    st.wissued += 1;
}

// Bind the block to a row-form plan: parameters, site and neighbour tables,
// zeroed activations and zero block, first weight load.
__device__ void row_bind(const TcPlan &pl, TcShared &sh, const unsigned char *packed, TcState &st) {
    unsigned char *smem = sh.base;
    sh.spins = reinterpret_cast<int8_t *>(smem + pl.o_spins);
    sh.rowtab = nullptr;
    sh.sitetab = reinterpret_cast<const uint2 *>(smem + pl.o_sitetab);
    sh.f32 = reinterpret_cast<float *>(smem + pl.o_f32);
    sh.res = reinterpret_cast<double *>(smem + pl.o_res);
    const float *src = reinterpret_cast<const float *>(packed);
    for (uint32_t i = threadIdx.x; i < pl.f32_count; i += blockDim.x) sh.f32[i] = src[i];
    uint2 *sitetab = reinterpret_cast<uint2 *>(smem + pl.o_sitetab);
    for (int s = threadIdx.x; s < pl.N; s += blockDim.x) {
        int pos[4];
        const int n = images(pl.L, pl.Lp, s % pl.L, s / pl.L, pos);
        sitetab[s] = pack4(pos, n);
    }
    // zero the activations (rows no output writes are read only by discarded
    // accumulator rows, but stay finite) and the zero block
    for (uint32_t i = threadIdx.x; i < pl.act_bytes / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(smem + pl.o_act)[i] = 0u;
    for (uint32_t i = threadIdx.x; i < 4096 / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(smem + pl.o_zero)[i] = 0u;
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, iw = warp - pl.epi;
        if (lane == 0 && iw >= 0 && iw < kIssuers) {
            if (pl.C == 16) row_build_mtab<16>(pl, sh, iw);
            else row_build_mtab<32>(pl, sh, iw);
        }
    }
    ptx::fence_async_smem();
    __syncthreads();
    st.wbase = st.wissued;
    st.wseq = st.wissued;
    if (threadIdx.x == 0) issue_weight_load(pl, sh, packed, st.wissued, st.wbase);
    st.wissued += 1;
}

// Wait for prefetched weight loads nobody will consume (before re-binding
// or exiting), so no copy is in flight into the buffers.
__device__ void tc_unbind(TcShared &sh, TcState &st) {
    __syncthreads();
    if (threadIdx.x == 0)
        for (uint32_t q = st.wseq; q < st.wissued; ++q) ptx::mbar_wait(&sh.bar_w[q & 1], (q >> 1) & 1);
    st.wseq = st.wissued;
    __syncthreads();
}

__device__ void tc_fini(TcShared &sh, TcState &st, uint32_t tmem_cols) {
    tc_unbind(sh, st);
    ptx::tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(*sh.tmem_addr, tmem_cols);
    }
}

__device__ void tc_setup(const TcPlan &pl, TcShared &sh, unsigned char *smem, const unsigned char *packed,
                         TcState &st) {
    tc_init(sh, smem, pl.tmem_cols, st);
    tc_bind(pl, sh, packed, st);
}

__device__ void tc_teardown(const TcPlan &pl, TcShared &sh, TcState &st) { tc_fini(sh, st, pl.tmem_cols); }

// ---------------------------------------------------------------- kernels
// Failure-path check: one warp waits, through the kernels' bounded wait, on
// an mbarrier phase that nothing completes; when the limit runs out it sets
// the timeout bit exactly as a stalled pipeline would, and exits.
__global__ void wait_probe_kernel(int *err, long long limit) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        abort_flag = 0;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    const bool got = wait_or_abort(&bar, 0, &abort_flag, limit);
    if (!__all_sync(0xffffffffu, got) && threadIdx.x == 0) atomicOr(err, ERRBIT_TIMEOUT);
}

template <int C>
__global__ void __launch_bounds__(kTcThreads, kMinBlocks<C>) logpsi_tc_kernel(TcPlan pl, const unsigned char *packed,
                                                                   const int8_t *configs, int64_t n, double *out,
                                                                   int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    const int G = pl.G, N = pl.N, per = G * pl.slots;
    for (int64_t b0 = (int64_t)blockIdx.x * per; b0 < n; b0 += (int64_t)gridDim.x * per) {
        const int cnt = (int)min((int64_t)per, n - b0);
        for (int r = threadIdx.x; r < per * N; r += blockDim.x) {
            const int c = r / N;
            sh.spins[r] = configs[(b0 + (c < cnt ? c : 0)) * N + (r - c * N)];
        }
        __syncthreads();
        if (!tc_forward<C>(pl, sh, packed, st, err)) break;
        for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
            const int s = c / G, g = c - s * G;
            out[2 * (b0 + c)] = sh.res[s * 2 * G + g];
            out[2 * (b0 + c) + 1] = sh.res[s * 2 * G + G + g];
        }
        __syncthreads();
    }
    tc_teardown(pl, sh, st);
}

// Local energy of one configuration (Sec. 5.4.1): enumerate its connected
// configurations, evaluate sigma and all of them in groups, then
// E_loc = H_diag + sum_k H_k exp((a'_k - a) + i (phi'_k - phi)) in float64,
// every term of the sample at once, fixed-order block reduction.
// ROWS: the configurations go through the row form (no cones).
template <int C, bool ROWS = false, bool F8 = false>
__device__ bool eloc_sample(const TcPlan &pl, const Problem &p, const TcShared &sh, TcState &st,
                            const unsigned char *packed, const int8_t *cfg, const double *logpsi_s, double *out_s,
                            int *err, unsigned char *cache) {
    const int G = pl.G, N = pl.N, L = pl.L, per = G * pl.slots, chunk = bond_chunk(p);
    unsigned char *ex = sh.base + pl.o_extra;
    int8_t *sigma = reinterpret_cast<int8_t *>(ex);
    int16_t *ci = reinterpret_cast<int16_t *>(ex + al16(N));
    int16_t *cj = ci + chunk;
    double *ch = reinterpret_cast<double *>(ex + al16(N) + al16(4 * chunk));
    int *cum = reinterpret_cast<int *>(ch + chunk);
    EnumScratch *scr = reinterpret_cast<EnumScratch *>(ex + al16(N) + al16(4 * chunk) + al16(8 * chunk) +
                                                       al16(4 * (N + 1)));
    double *ref = reinterpret_cast<double *>(scr + 1);   // a0, phi0
    double *lp = ref + 4;                                 // [chunk + 1][2]: (a, phi) of every list entry
    double *fsum = lp + 2 * (chunk + 1);                  // [258] fixed-order sum scratch
    int16_t *ord = reinterpret_cast<int16_t *>(fsum + 258);   // [chunk] evaluation order of the entries
    int *roll = reinterpret_cast<int *>(ord + ((chunk + 1) & ~1));   // [32] per configuration of a group
    const int recompute = logpsi_s == nullptr;
    // the cone of every connected configuration is evaluated alone when the
    // sample itself is evaluated here (its activations fill the cache)
    const bool cone = !ROWS && cache != nullptr && recompute && pl.slots == 1;
    for (int r = threadIdx.x; r < N; r += blockDim.x) sigma[r] = cfg[r];
    __syncthreads();
    if (p.model == NQS_MODEL_TJ) snake_prefix(p, sigma, cum, *scr);
    if (threadIdx.x == 0 && !recompute) { ref[0] = logpsi_s[0]; ref[1] = logpsi_s[1]; }
    __syncthreads();
    // bonds in chunks (one chunk unless the lattice is large); running float64
    // sums of the diagonal and of the off-diagonal terms, identical in every thread
    double hd_tot = 0.0, sr_tot = 0.0, si_tot = 0.0;
    for (int b0 = 0; b0 < p.n_bonds; b0 += chunk) {
        double hd;
        const int nconn = enumerate_range(p, sigma, b0, min(p.n_bonds, b0 + chunk), ci, cj, ch, &hd, cum, *scr);
        hd_tot += hd;
        const int lead = (recompute && b0 == 0) ? 1 : 0;   // sigma itself evaluated first
        const int n_entries = nconn + lead;
        // evaluation order: the first group (sigma and per - 1 entries) in list
        // order; with cones, the other entries grouped by class (pair in one
        // row, then pair in two rows), stable, so each group shares one band
        const int first = cone ? min(nconn, per - lead) : nconn;
        for (int k = threadIdx.x; k < first; k += blockDim.x) ord[k] = (int16_t)k;
        int base0 = first, n0 = 0;
        for (int cls = 0; cls < 2 && first < nconn; ++cls) {
            int base = cls == 0 ? first : first + n0;
            for (int k0 = first; k0 < nconn; k0 += blockDim.x) {
                const int k = k0 + threadIdx.x;
                int f = 0;
                if (k < nconn) f = ((ci[k] / L) != (cj[k] / L)) == (cls == 1);
                int tot;
                const int off = block_exclusive_scan(f, scr->iscr, &tot);
                if (f) ord[base + off] = (int16_t)k;
                base += tot;
            }
            if (cls == 0) n0 = base - base0;
        }
        __syncthreads();
        for (int e0 = 0; e0 < n_entries; e0 += per) {
            const int cnt = min(per, n_entries - e0);
            // band of this group: all entries of one class (never the group holding sigma)
            Band band = dense_band();
            if (cone && e0 >= lead + first) {
                const int ka = ord[e0 - lead], kb = ord[e0 + cnt - 1 - lead];
                const int ca = (ci[ka] / L) != (cj[ka] / L), cb = (ci[kb] / L) != (cj[kb] / L);
                if (ca == cb) band = Band{ca, ca ? L / 2 - 1 : L / 2, roll};
            }
            if (threadIdx.x < per) {
                int r = 0;
                const int c = threadIdx.x;
                if (band.cls >= 0 && c < cnt) {
                    const int k = ord[e0 + c - lead];
                    const int yi = ci[k] / L, yj = cj[k] / L;
                    const int top = band.cls == 0 ? yi : ((yi + 1) % L == yj ? yi : yj);
                    r = (top - band.top + L) % L;
                }
                roll[c] = r;
            }
            __syncthreads();
            // configuration c of the group: one warp per configuration, lanes over sites (no divisions)
            {
                const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
                for (int c = warp; c < per; c += nwarps) {
                    const int q = e0 + c - lead;   // list position (-1: sigma)
                    const bool own = c >= cnt || q < 0;
                    const int k = own ? 0 : ord[q];
                    const int i = own ? -1 : ci[k], j = own ? -1 : cj[k];
                    const int rl = roll[c] * L;
                    const bool idx_ok = own || NQS_INDEX_OK(k >= 0 && k < nconn && i >= 0 && i < N && j >= 0 && j < N, err);
                    int8_t *dst = sh.spins + c * N;
                    for (int site = lane; site < N; site += 32) {
                        int v;
                        if (own) {
                            v = sigma[site];
                        } else {
                            int s0 = site + rl;   // original site: row + roll (mod L)
                            if (s0 >= N) s0 -= N;
                            v = idx_ok ? sigma[s0 == i ? j : (s0 == j ? i : s0)] : 0;
                        }
                        dst[site] = (int8_t)v;
                    }
                }
            }
            __syncthreads();
            if (ROWS) {
                if (!row_forward<C, F8>(pl, sh, packed, st, err)) return false;
            } else if (!tc_forward<C>(pl, sh, packed, st, err, band, cache, (cone && lead && e0 == 0) ? cache : nullptr)) {
                return false;
            }
            if (threadIdx.x < cnt) {
                const int c = threadIdx.x, sl = c / G, g = c - sl * G;
                const int q = e0 + c - lead;
                const int idx = q < 0 ? 0 : ord[q] + lead;
                lp[2 * idx] = sh.res[sl * 2 * G + g];
                lp[2 * idx + 1] = sh.res[sl * 2 * G + G + g];
            }
            __syncthreads();
        }
        __syncthreads();
        if (lead && threadIdx.x == 0) { ref[0] = lp[0]; ref[1] = lp[1]; }
        __syncthreads();
        // off-diagonal terms in an order independent of the block size
        const double2 tsum = fixed_order_sum2(nconn, [&](int k) {
            const double m = ch[k] * exp(lp[2 * (k + lead)] - ref[0]);
            double sn, cs;
            sincos(lp[2 * (k + lead) + 1] - ref[1], &sn, &cs);
            return make_double2(m * cs, m * sn);
        }, fsum);
        sr_tot += tsum.x;
        si_tot += tsum.y;
    }
    if (threadIdx.x == 0) {
        const double er = hd_tot + sr_tot, ei = si_tot;
        out_s[0] = er;
        out_s[1] = ei;
        if (!isfinite(er) || !isfinite(ei)) atomicOr(err, ERRBIT_NONFINITE);
    }
    __syncthreads();
    return true;
}

template <int C>
__global__ void __launch_bounds__(kTcThreads, kMinBlocks<C>)
    eloc_tc_kernel(TcPlan pl, Problem p, const unsigned char *packed, const int8_t *configs, const double *logpsi,
                   int64_t n, double *out, int *err, unsigned char *cache) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    unsigned char *my_cache = cache ? cache + (size_t)blockIdx.x * sigma_cache_bytes(pl) : nullptr;
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x)
        if (!eloc_sample<C>(pl, p, sh, st, packed, configs + s * p.N, logpsi ? logpsi + 2 * s : nullptr, out + 2 * s,
                            err, my_cache))
            break;
    tc_teardown(pl, sh, st);
}

// Local energies through the row form (plans with L * C <= 256 columns);
// F8: e4m3 operands in layers >= 1 (16 channels).
template <int C, bool F8 = false>
__global__ void __launch_bounds__(kTcThreads, 2)
    eloc_rows_kernel(TcPlan pl, Problem p, const unsigned char *packed, const int8_t *configs, const double *logpsi,
                     int64_t n, double *out, int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_init(sh, smem, pl.tmem_cols, st);
    row_bind(pl, sh, packed, st);
    for (int64_t s = blockIdx.x; s < n; s += gridDim.x)
        if (!eloc_sample<C, true, F8>(pl, p, sh, st, packed, configs + s * p.N, logpsi ? logpsi + 2 * s : nullptr,
                                      out + 2 * s, err, nullptr))
            break;
    tc_teardown(pl, sh, st);
}

// One problem of a grouped local-energy launch.
struct TcRequest {
    TcPlan pl;
    Problem p;
    const unsigned char *packed;
    const int8_t *configs;
    const double *logpsi;
    double *out;
    int64_t n, start;   // samples, index of the first sample in the launch
};

// Local energies of several problems (same channel count) in one launch:
// blocks take samples one at a time from a global counter in problem-major
// order and re-bind their shared-memory plan when the problem changes.
template <int C>
__global__ void __launch_bounds__(kTcThreads, 1) eloc_tc_multi_kernel(const TcRequest *reqs, int nreq, int64_t total,
                                                                       uint32_t tmem_cols, unsigned long long *counter,
                                                                       int *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ long long grab;
    TcShared sh;
    TcState st;
    tc_init(sh, smem, tmem_cols, st);
    int cur = -1;
    TcPlan pl;
    Problem p;
    while (true) {
        if (threadIdx.x == 0) grab = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t g = grab;
        __syncthreads();
        if (g >= total) break;
        int r = 0;
        while (r + 1 < nreq && reqs[r + 1].start <= g) ++r;
        if (r != cur) {
            if (cur >= 0) tc_unbind(sh, st);
            pl = reqs[r].pl;
            p = reqs[r].p;
            tc_bind(pl, sh, reqs[r].packed, st);
            cur = r;
        }
        const int64_t s = g - reqs[r].start;
        const double *lps = reqs[r].logpsi ? reqs[r].logpsi + 2 * s : nullptr;
        if (!eloc_sample<C>(pl, p, sh, st, reqs[r].packed, reqs[r].configs + s * p.N, lps, reqs[r].out + 2 * s, err,
                            nullptr))
            break;
    }
    tc_fini(sh, st, tmem_cols);
}

__device__ __forceinline__ int neighbour_dir_tc(int i, int d, int L) {
    const int x = i % L, y = i / L;
    const int dx = d == 0 ? 1 : (d == 1 ? -1 : 0);
    const int dy = d == 2 ? 1 : (d == 3 ? -1 : 0);
    return ((y + dy + L) % L) * L + (x + dx + L) % L;
}

// Metropolis exchange sampler. Each block owns up to slots * G chains;
// slot s evaluates the proposals of chains s * G ... s * G + G - 1.
template <int C>
__global__ void __launch_bounds__(kTcThreads, 2) sample_tc_kernel(TcPlan pl, const unsigned char *packed,
                                                                   int8_t *chains, int n_chains, int per_block,
                                                                   uint64_t step0, uint64_t seed, int spc,
                                                                   int sweeps_between, int burn_in, int8_t *out_cfg,
                                                                   double *out_logpsi, int *err,
                                                                   unsigned long long *moves) {
    extern __shared__ __align__(128) unsigned char smem[];
    TcShared sh;
    TcState st;
    tc_setup(pl, sh, smem, packed, st);
    const int G = pl.G, N = pl.N, S = pl.slots;
    unsigned char *ex = smem + pl.o_extra;
    int8_t *cur = reinterpret_cast<int8_t *>(ex);                                // [per_block][N]
    // [2][S][G + 1]: by step parity (step q + 1 is built while slower threads may still read step q's)
    int *list2 = reinterpret_cast<int *>(ex + al16(per_block * N));
    double *ca = reinterpret_cast<double *>(ex + al16(per_block * N) + al16(4 * 2 * (S * (G + 1))));
    double *cphi = ca + per_block;
    // proposals of the next kPropWindow steps of every chain of the group,
    // drawn in parallel (they do not depend on the chain state): site i,
    // neighbour j and log u, [step][chain]
    const int W = prop_window(per_block);
    double *wlu = cphi + per_block;
    int *wpi = reinterpret_cast<int *>(wlu + W * per_block);
    int *wpj = wpi + W * per_block;
    // moves and accepted moves of the block, in shared memory after the proposal window (not live in
    // registers across the forward; the address is recomputed where it is used)
    auto scnt = [&]() {
        return reinterpret_cast<unsigned long long *>(smem + pl.o_extra +
                                                      ((al16(per_block * pl.N) + al16(8 * pl.slots * (pl.G + 1)) +
                                                        16 * per_block + 16 * prop_window(per_block) * per_block +
                                                        7) & ~7u));
    };
    if (threadIdx.x == 0) { scnt()[0] = 0; scnt()[1] = 0; }
    // chain groups: group k = blockIdx.x + j * gridDim.x (one pass when the
    // grid covers every group; fewer blocks when the launch is held to an SM share)
    bool ok = true;
    for (int c0 = blockIdx.x * per_block; ok && c0 < n_chains; c0 += gridDim.x * per_block) {
    const int gc = min(per_block, n_chains - c0);
    {
        for (int r = threadIdx.x; r < gc * N; r += blockDim.x) cur[r] = chains[(size_t)c0 * N + r];
        __syncthreads();
        for (int r = threadIdx.x; r < per_block * N; r += blockDim.x) {
            const int c = r / N;
            sh.spins[r] = cur[(c < gc ? c : 0) * N + (r - c * N)];
        }
        __syncthreads();
        ok = tc_forward<C>(pl, sh, packed, st, err);
        for (int c = threadIdx.x; c < gc; c += blockDim.x) {
            const int s = c / G, g = c - s * G;
            ca[c] = sh.res[s * 2 * G + g];
            cphi[c] = sh.res[s * 2 * G + G + g];
        }
        __syncthreads();
    }
    const int n_sweeps = burn_in + spc * sweeps_between;
    const int64_t n_steps = (int64_t)n_sweeps * N;
    for (int sweep = 0; ok && sweep < n_sweeps; ++sweep) {
        for (int q = 0; q < N; ++q) {
            const int64_t gstep = (int64_t)sweep * N + q;
            const int w = (int)(gstep & (int64_t)(W - 1));
            if (w == 0) {   // draw the window (one Philox4x64-10 block per chain and step)
                // every thread has read the previous window (steps without a forward pass no block barrier)
                __syncthreads();
                for (int t = threadIdx.x; t < W * gc; t += blockDim.x) {
                    const int ww = t / gc, c = t - ww * gc;
                    if (gstep + ww >= n_steps) continue;
                    const Philox4 b = philox((uint64_t)(c0 + c), step0 + (uint64_t)(gstep + ww), 0, 0, seed, 0);
                    const int i = (int)mulhi64(b.v[0], (uint64_t)N);
                    wpi[ww * per_block + c] = i;
                    wpj[ww * per_block + c] = neighbour_dir_tc(i, (int)(b.v[1] >> 62), pl.L);
                    const double u = (double)(b.v[2] >> 11) * 0x1.0p-53;
                    wlu[ww * per_block + c] = u > 0.0 ? log(u) : -INFINITY;
                }
                __syncthreads();
            }
            int *pi_s = wpi + w * per_block;
            int *pj_s = wpj + w * per_block;
            if (per_block == 1) {
                // one chain: every thread sees the same state (the last block barrier followed its update), so
                // each one decides whether the proposal changes it, with no list and no barrier; the forward reads
                // the chain with the two sites exchanged
                const int i = pi_s[0], j = pj_s[0];
                if (!NQS_INDEX_OK(i >= 0 && i < N && j >= 0 && j < N, err) || cur[i] == cur[j]) continue;
                if (threadIdx.x == 0) scnt()[0] += 1ull;
                const SwapSrc sw{cur, i, j};
                if (!tc_forward<C>(pl, sh, packed, st, err, dense_band(), nullptr, nullptr, &sw)) { ok = false; break; }
                if (threadIdx.x == 0) {
                    const double an = sh.res[0];
                    const double delta = 2.0 * (an - ca[0]);
                    // u < exp(2 (a' - a)) evaluated as log u < 2 (a' - a), log u drawn with the proposal
                    if (delta >= 0.0 || wlu[w] < delta) {
                        scnt()[1] += 1ull;
                        const int8_t t = cur[i];
                        cur[i] = cur[j];
                        cur[j] = t;
                        ca[0] = an;
                        cphi[0] = sh.res[G];
                    }
                }
                __syncthreads();
                continue;
            }
            int *list = list2 + (int)(gstep & 1) * S * (G + 1);
            if (threadIdx.x < S) {   // per-slot list of chains whose proposal changes the state
                const int s = threadIdx.x;
                int cnt = 0;
                for (int g = 0; g < G; ++g) {
                    const int c = s * G + g;
                    if (c < gc && NQS_INDEX_OK(pi_s[c] >= 0 && pi_s[c] < N && pj_s[c] >= 0 && pj_s[c] < N, err) &&
                        cur[c * N + pi_s[c]] != cur[c * N + pj_s[c]])
                        list[s * (G + 1) + cnt++] = c;
                }
                list[s * (G + 1) + G] = cnt;
            }
            __syncthreads();
            int total = 0;
            for (int s = 0; s < S; ++s) total += list[s * (G + 1) + G];
            if (total == 0) continue;
            if (threadIdx.x == 0) scnt()[0] += (unsigned long long)total;
            for (int r = threadIdx.x; r < per_block * N; r += blockDim.x) {
                const int slot_row = r / N, site = r - slot_row * N;
                const int s = slot_row / G, m = slot_row - s * G;
                const int cnt = list[s * (G + 1) + G];
                const int c = cnt > 0 ? list[s * (G + 1) + (m < cnt ? m : 0)] : 0;
                const int i = cnt > 0 ? pi_s[c] : -1, j = cnt > 0 ? pj_s[c] : -1;
                const int src = site == i ? j : (site == j ? i : site);
                sh.spins[r] = cur[c * N + src];
            }
            __syncthreads();
            if (!tc_forward<C>(pl, sh, packed, st, err)) { ok = false; break; }
            for (int r = threadIdx.x; r < per_block; r += blockDim.x) {
                const int s = r / G, m = r - s * G;
                if (m >= list[s * (G + 1) + G]) continue;
                const int c = list[s * (G + 1) + m];
                const double an = sh.res[s * 2 * G + m];
                const double delta = 2.0 * (an - ca[c]);
                // u < exp(2 (a' - a)) evaluated as log u < 2 (a' - a), log u drawn with the proposal
                if (delta >= 0.0 || wlu[w * per_block + c] < delta) {
                    atomicAdd(&scnt()[1], 1ull);
                    const int i = pi_s[c], j = pj_s[c];
                    const int8_t t = cur[c * N + i];
                    cur[c * N + i] = cur[c * N + j];
                    cur[c * N + j] = t;
                    ca[c] = an;
                    cphi[c] = sh.res[s * 2 * G + G + m];
                }
            }
            __syncthreads();
        }
        if (ok && sweep >= burn_in && (sweep - burn_in + 1) % sweeps_between == 0) {
            const int k = (sweep - burn_in + 1) / sweeps_between - 1;
            for (int r = threadIdx.x; r < gc * N; r += blockDim.x) {
                const int c = r / N, site = r - c * N;
                out_cfg[((size_t)(c0 + c) * spc + k) * N + site] = cur[r];
            }
            for (int c = threadIdx.x; c < gc; c += blockDim.x) {
                out_logpsi[2 * ((size_t)(c0 + c) * spc + k)] = ca[c];
                out_logpsi[2 * ((size_t)(c0 + c) * spc + k) + 1] = cphi[c];
                if (!isfinite(ca[c])) atomicOr(err, ERRBIT_NONFINITE);
            }
            __syncthreads();
        }
    }
    if (ok)
        for (int r = threadIdx.x; r < gc * N; r += blockDim.x) chains[(size_t)c0 * N + r] = cur[r];
    __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0 && moves && scnt()[0]) {
        atomicAdd(&moves[0], scnt()[0]);
        atomicAdd(&moves[1], scnt()[1]);
    }
    tc_teardown(pl, sh, st);
}

// ---------------------------------------------------------------- packing
// fp32 block: biases[l][c], head[2][c]. bf16 block of layer 0: B operand
// [K0 / 8][C][8] with k = tap (J1-J2) or 3 tap + one-hot channel (t-J),
// zero for k >= 9 c_in. bf16 block per layer l >= 1: [9][C / 8][C][8],
// element (tap o, k = c_in, n = c_out); then the same layers again in the
// row form's order [3][C / 8][3][C][8].
__global__ void tc_pack_kernel(Problem p, TcPlan pl, const double *params, unsigned char *packed) {
    const int C = p.C;
    float *f = reinterpret_cast<float *>(packed);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int e = tid; e < p.n_layers * C; e += nth) {
        const int l = e / C, c = e - l * C;
        f[e] = (float)params[layer_offset(p, l) + 9 * layer_cin(p, l) * C + c];
    }
    for (int e = tid; e < 2 * C; e += nth) f[p.n_layers * C + e] = (float)params[head_offset(p) + e];
    __nv_bfloat16 *w0 = reinterpret_cast<__nv_bfloat16 *>(packed + pl.f32_bytes);
    for (int e = tid; e < pl.K0 * C; e += nth) {
        const int n = e / pl.K0, k = e - n * pl.K0;
        float w = 0.f;
        if (k < 9 * p.c_in) {
            const int o = p.c_in == 1 ? k : k / 3, ci = p.c_in == 1 ? 0 : k % 3;
            w = (float)params[(n * p.c_in + ci) * 9 + o];
        }
        w0[((k / 8) * C + n) * 8 + (k % 8)] = __float2bfloat16_rn(w);
    }
    const int per = 9 * C * C;
    for (int e = tid; e < (p.n_layers - 1) * per; e += nth) {
        const int l = 1 + e / per, r = e - (l - 1) * per;
        const int o = r / (C * C), r2 = r - o * C * C, n = r2 / C, k = r2 - n * C;
        const double w = params[layer_offset(p, l) + (n * C + k) * 9 + o];
        __nv_bfloat16 *dst =
            reinterpret_cast<__nv_bfloat16 *>(packed + pl.f32_bytes + pl.w0bytes + (size_t)(l - 1) * pl.wbytes);
        dst[((o * (C / 8) + k / 8) * C + n) * 8 + (k % 8)] = __float2bfloat16_rn((float)w);
        // row-form image of the same layer: [kernel row dy][C / 8][column block j = 1 - dx][C][8], so that
        // one kernel row's three dx taps are one N = 3C operand
        __nv_bfloat16 *dr = reinterpret_cast<__nv_bfloat16 *>(packed + pl.f32_bytes + pl.w0bytes +
                                                               (size_t)(p.n_layers - 1 + l - 1) * pl.wbytes);
        const int dyi = o / 3, j = 2 - o % 3;
        dr[(((dyi * (C / 8) + k / 8) * 3 + j) * C + n) * 8 + (k % 8)] = __float2bfloat16_rn((float)w);
    }
    // e4m3 images of layers >= 1 (layer 0 keeps bf16 operands); the scale of output channel n is the largest
    // |weight| of the channel over 448, the largest e4m3 value
    if (pl.f8bytes == 0) return;
    for (int e = tid; e < (p.n_layers - 1) * C; e += nth) {
        const int l = 1 + e / C, n = e - (l - 1) * C;
        const double *wn = params + layer_offset(p, l) + (size_t)n * C * 9;   // [cin][dy][dx] of channel n
        double m = 0.0;
        for (int k = 0; k < 9 * C; ++k) m = fmax(m, fabs(wn[k]));
        const float sc = m > 0.0 ? (float)m / 448.f : 1.f;
        // row-form image [pair q][K half h][column block j = 1 - dx][C][16 input channels]: kernel row
        // dy = 2 q + h (dy = 3: zero), so one K = 32 operand holds two kernel rows; then the scales
        unsigned char *dst = packed + pl.f32_bytes + pl.w0bytes + 2 * (size_t)(p.n_layers - 1) * pl.wbytes +
                             (size_t)(l - 1) * pl.f8bytes;
        reinterpret_cast<float *>(dst + 12 * C * C)[n] = 0.5f * sc;   // halved, as the epilogue uses it
        for (int q = 0; q < 2; ++q)
            for (int h = 0; h < 2; ++h)
                for (int j = 0; j < 3; ++j) {
                    const int dy = 2 * q + h, dxi = 2 - j;
                    unsigned short *row = reinterpret_cast<unsigned short *>(dst + (((q * 2 + h) * 3 + j) * C + n) * 16);
                    for (int k = 0; k < 16; k += 2) {
                        const float w0 = dy < 3 ? (float)wn[k * 9 + dy * 3 + dxi] / sc : 0.f;
                        const float w1 = dy < 3 ? (float)wn[(k + 1) * 9 + dy * 3 + dxi] / sc : 0.f;
                        row[k / 2] = (unsigned short)ptx::pack_e4m3(w0, w1);
                    }
                }
    }
}

// ---------------------------------------------------------------- host planning
// Packed image: fp32 block (biases [n_layers][C], head [2][C]), bf16 layer 0,
// bf16 tap-form and row-form images of layers >= 1, and with 16 channels the
// e4m3 row-form images of layers >= 1, each followed by its fp32 weight
// scales [C], halved.
void plan_weights(const Problem &p, TcPlan &pl) {
    pl.K0 = p.c_in == 1 ? 16 : 32;
    pl.f32_count = p.n_layers * p.C + 2 * p.C;
    pl.f32_bytes = al16(pl.f32_count * 4);
    pl.w0bytes = (uint32_t)pl.K0 * p.C * 2u;
    pl.wbytes = 9u * p.C * p.C * 2u;
    pl.wstride = pl.wbytes;
    pl.f8bytes = p.C == 16 ? 12u * p.C * p.C + 4u * p.C : 0u;   // [pair][K half][j][C][16], scales [C]
}

int eloc_extra(const Problem &p);

// Row-form plan (local energies): one group of G = min(16, 128 / L)
// configurations per block, the L x C accumulator columns of a layer in
// tensor memory, two blocks per SM. Needs L * C <= 256.
bool make_row_plan(const Problem &p, size_t max_smem, int extra_bytes, TcPlan *out, std::string *why, int G = 0) {
    if (p.L * p.C > 256) { *why = "row form needs L * C <= 256 accumulator columns"; return false; }
    // MMA lists: 3 (dy) x (columns per issuer + 2) x (C / 16) per layer, columns x (K0 / 16) for layer 0
    const int per_issuer = (p.L + kIssuers - 1) / kIssuers;
    if (3 * (per_issuer + 2) * (p.C / 16) > kMtabLayer || per_issuer * 2 > kMtab0) {
        *why = "row form: MMA list too long";
        return false;
    }
    TcPlan pl{};
    pl.rows = 1;
    pl.ctas = 2;
    pl.epi = kMaxEpiWarps;
    pl.L = p.L;
    pl.Lp = p.L + 2;
    pl.N = p.N;
    pl.G = G > 0 ? std::min(G, 128 / p.L) : std::min(16, 128 / p.L);
    pl.C = p.C;
    pl.KC = p.C / 8;
    pl.c_in = p.c_in;
    pl.n_layers = p.n_layers;
    pl.slots = 1;
    plan_weights(p, pl);
    pl.wimg = (uint32_t)(p.n_layers - 1) * pl.wbytes;
    pl.n_tiles = 1;
    // the last A operand read starts at ((L + 1) Lp + 2) G and spans 128 rows; the im2col of layer 0 takes L x 128
    pl.rows_total = std::max(pl.Lp * pl.Lp * pl.G + 128, p.L * 128);
    pl.rows_total = (pl.rows_total + 7) & ~7;
    pl.rbuf = pl.rows_total;
    pl.plane = (uint32_t)pl.rows_total * 16u;
    pl.act_bytes = pl.plane * (uint32_t)std::max(pl.KC, pl.K0 / 8);
    pl.slot_cols = (uint32_t)(p.L * p.C);
    uint32_t cols = 32;
    while (cols < pl.slot_cols) cols <<= 1;
    pl.tmem_cols = cols;
    uint32_t o = kBarBytes;
    pl.o_bar = 0;
    pl.o_act = o; o = al16(o + pl.act_bytes);
    pl.o_zero = o; o = al16(o + 4096);
    pl.o_w0 = o; o = al16(o + pl.wbytes);
    pl.o_w1 = o; o = al16(o + pl.wbytes);
    pl.o_f32 = o; o = al16(o + pl.f32_count * 4);
    pl.o_sitetab = o; o = al16(o + 8 * p.N);
    pl.o_mtab = o; o = al16(o + kMtabBytes);
    pl.o_spins = o; o = al16(o + pl.G * p.N);
    pl.o_res = o; o = al16(o + 16 * pl.G);
    pl.o_extra = o; o = al16(o + extra_bytes);
    const uint32_t sm_bytes = 233472u;   // 228 KB per SM, 1 KB reserved per block
    while (cols * (sm_bytes / (o + 1024u)) > 512u) o += 1024u;
    pl.total = o;
    if (cols * 2u > 512u) { *why = "tensor-memory columns do not fit two blocks"; return false; }
    if (2u * (pl.total + 1024u) > sm_bytes) { *why = "row form: two blocks do not fit the SM's shared memory"; return false; }
    if (pl.total > max_smem) { *why = "shared memory plan exceeds the per-block limit"; return false; }
    // the contributions of the head ([2][G][Lp^2] floats) reuse the activation buffer
    if ((size_t)8 * pl.G * pl.Lp * pl.Lp > pl.act_bytes) { *why = "head contributions exceed the buffer"; return false; }
    *out = pl;
    return true;
}

// Whether the local-energy launch uses the row form (NQS_TC_ROWS=0 turns it
// off, NQS_TC_ROWS=G forces G configurations per group: tuning and A/B
// comparisons).
bool use_row_form(const Problem &p, size_t max_smem, TcPlan *out) {
    const char *e = getenv("NQS_TC_ROWS");
    int G = 0;
    if (e) {
        G = atoi(e);
        if (G == 0) return false;
    }
    std::string why;
    return make_row_plan(p, max_smem, eloc_extra(p), out, &why, G);
}

bool make_plan(const Problem &p, int G, int slots, int ctas, size_t max_smem, int extra_bytes, TcPlan *out,
               std::string *why) {
    TcPlan pl{};
    pl.ctas = ctas;
    pl.epi = kMaxEpiWarps;
    pl.L = p.L;
    pl.Lp = p.L + 2;
    pl.N = p.N;
    pl.G = G;
    pl.C = p.C;
    pl.KC = p.C / 8;
    pl.c_in = p.c_in;
    pl.n_layers = p.n_layers;
    pl.slots = slots;
    plan_weights(p, pl);
    pl.count_out = (p.L - 1) * pl.Lp + p.L;
    pl.r0 = (pl.Lp + 1) * G;
    pl.n_tiles = (pl.count_out * G + 127) / 128;
    const int reach = (pl.Lp + 1) * G;
    pl.rbuf = std::max(pl.r0 + pl.n_tiles * 128 + reach, pl.Lp * pl.Lp * G);
    pl.rbuf = (pl.rbuf + 7) & ~7;
    pl.plane = (uint32_t)pl.rbuf * 16u;
    pl.act_bytes = pl.plane * (uint32_t)std::max(pl.KC, pl.K0 / 8);
    pl.slot_cols = (uint32_t)(pl.n_tiles * p.C);
    uint32_t cols = 32;
    while (cols < (uint32_t)slots * pl.slot_cols) cols <<= 1;
    pl.tmem_cols = cols;
    uint32_t o = kBarBytes;
    pl.o_bar = 0;
    pl.o_act = o; o = al16(o + (uint32_t)slots * 2u * pl.act_bytes);
    pl.o_w0 = o; o = al16(o + pl.wbytes);
    pl.o_w1 = o; o = al16(o + pl.wbytes);
    pl.o_f32 = o; o = al16(o + pl.f32_count * 4);
    pl.o_rowtab = o; o = al16(o + 8 * pl.n_tiles * 128);
    pl.o_sitetab = o; o = al16(o + 8 * p.N);
    pl.o_spins = o; o = al16(o + slots * G * p.N);
    pl.o_res = o; o = al16(o + 16 * slots * G);
    pl.o_extra = o; o = al16(o + extra_bytes);
    // co-resident blocks must not ask for more than the SM's 512 TMEM
    // columns together: pad shared memory to cap residency
    const uint32_t sm_bytes = 233472u;   // 228 KB per SM, 1 KB reserved per block
    while (cols * (sm_bytes / (o + 1024u)) > 512u) o += 1024u;
    pl.total = o;
    if (cols * (uint32_t)ctas > 512) { *why = "tensor-memory tiles do not fit in 512 columns"; return false; }
    if ((uint32_t)ctas * (pl.total + 1024u) > sm_bytes) { *why = "shared memory plan exceeds the per-SM share"; return false; }
    if (pl.n_tiles > kMaxTiles) { *why = "more than 16 row tiles per group"; return false; }
    if (pl.rbuf >= (int)kNone) { *why = "row index range exceeds 16 bits"; return false; }
    if (pl.total > max_smem) { *why = "shared memory plan exceeds the per-block limit"; return false; }
    *out = pl;
    return true;
}

int eloc_extra(const Problem &p) {
    const int chunk = bond_chunk(p);
    return (int)(al16(p.N) + al16(4 * chunk) + al16(8 * chunk) + al16(4 * (p.N + 1)) + sizeof(EnumScratch) +
                 4 * sizeof(double) + 16 * (chunk + 1) + 8 * 258 + 2 * ((chunk + 1) & ~1) + 4 * 32);
}

int sample_extra(const Problem &p, int G, int slots) {
    const int per = G * slots;
    return (int)(al16(per * p.N) + al16(4 * 2 * (slots * (G + 1))) + 16 * per + 16 * prop_window(per) * per + 24);
}

// Relative throughput of a one-slot plan: useful rows per computed row,
// with a fixed cost of four tiles per forward (inputs, head, barriers).
double plan_score(const Problem &p, const TcPlan &pl) {
    return (double)(p.N * pl.G) / (double)(pl.n_tiles * 128 + 4 * 128);
}

// NQS_TC_PLAN="G,slots[,blocks per SM]" forces a plan (tuning); ignored if
// infeasible or if the launch allows fewer blocks per SM.
bool forced_plan(int *G, int *slots, int *ctas) {
    const char *s = getenv("NQS_TC_PLAN");
    *ctas = 1;
    if (!s) return false;
    const int k = sscanf(s, "%d,%d,%d", G, slots, ctas);
    return k >= 2 && *G >= 1 && *G <= 16 && *slots >= 1 && *slots <= kMaxSlots && *ctas >= 1 && *ctas <= 2;
}

bool best_plan(const Problem &p, size_t max_smem, bool eloc, int gmax, int max_ctas, TcPlan *out, std::string *why) {
    int fg, fs, fc;
    if (forced_plan(&fg, &fs, &fc) && fc <= max_ctas &&
        make_plan(p, fg, fs, fc, max_smem, eloc ? eloc_extra(p) : 0, out, why))
        return true;
    // 16 channels: two co-resident blocks per SM with the largest group that
    // fits, when that group has at least 3 configurations (measured on GB300,
    // 6 layers: 1.32x at 10x10 J1-J2 with groups of 8, 1.13x at 12x12 t-J
    // with groups of 3 over the one-block plan; slower with groups of 2, as
    // at 16x16)
    if (p.C == 16 && max_ctas >= 2) {
        for (int G = gmax; G >= 3; --G) {
            std::string w;
            if (make_plan(p, G, 1, 2, max_smem, eloc ? eloc_extra(p) : 0, out, &w)) return true;
        }
    }
    // best one-slot plan; then two slots of the same G when they fit and a
    // slot has few tiles (measured on GB300: the epilogue tail after the last
    // MMA of a layer is then a large share of the layer, and the second slot
    // hides it; with many tiles the extra shared memory costs more than it saves)
    double best = -1.0;
    bool found = false;
    for (int G = 1; G <= gmax; ++G) {
        TcPlan pl;
        std::string w;
        if (!make_plan(p, G, 1, 1, max_smem, eloc ? eloc_extra(p) : 0, &pl, &w)) {
            if (!found) *why = w;
            continue;
        }
        const double sc = plan_score(p, pl);
        if (sc > best + 1e-9) { best = sc; *out = pl; found = true; }
    }
    if (found && out->n_tiles <= 8) {
        TcPlan two;
        std::string w;
        if (make_plan(p, out->G, 2, 1, max_smem, eloc ? eloc_extra(p) : 0, &two, &w)) *out = two;
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
    return allow_dynamic_smem(kernel, pl.total, env);
}

}  // namespace

bool tc_supported(const Problem &p, std::string *why) {
    if (p.net != NQS_NET_SILU) { *why = "the tensor-core path runs the SiLU network family"; return false; }
    if (p.C != 16 && p.C != 32) { *why = "the tensor-core path needs 16 or 32 channels"; return false; }
    return true;
}

size_t tc_packed_bytes(const Problem &p) {
    TcPlan pl{};
    plan_weights(p, pl);
    // tap and row images, e4m3 row images
    return pl.f32_bytes + pl.w0bytes + 2 * (size_t)(p.n_layers - 1) * pl.wbytes + (size_t)(p.n_layers - 1) * pl.f8bytes;
}

int launch_tc_pack(const Problem &p, const double *p64, void *packed, const LaunchEnv &env) {
    std::string why;
    if (!tc_supported(p, &why)) { *env.msg = why; return NQS_ERR_UNSUPPORTED; }
    TcPlan pl{};
    plan_weights(p, pl);
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
    if (!tc_supported(p, &why) || !best_plan(p, env.max_smem, false, 16, 2, &pl, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    const int64_t per = pl.G * pl.slots;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, (int64_t)env.num_sms * pl.ctas));
    NQS_TC_DISPATCH(p.C, {
        auto k = logpsi_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, 32 * (pl.epi + kIssuers), pl.total, env.stream>>>(pl, (const unsigned char *)packed, configs, n, out, env.err);
    });
    return check(env, "logpsi_tc_kernel");
}

// Bytes of the per-block cache of sample activations the E_loc launch
// uses to evaluate connected configurations on their cones only (0: the
// plan evaluates them densely). Cones are used with one-block-per-SM plans:
// measured on GB300 (E_loc, cones vs dense) 1.06x t-J 12x12 (32 channels),
// 1.12x 16x16 (32 channels), 1.13x 16x16 (16 channels), 1.25x 24x24; with
// two blocks per SM (10x10, 8x8, t-J 12x12 with 16 channels) the fixed
// per-layer costs of a band (the fill, a shorter tile pipeline) outweigh
// the saved tiles (0.93-0.98x). NQS_TC_DENSE=1 turns the cones off,
// NQS_TC_CONES=1 forces them wherever a plan allows (tuning).
size_t tc_eloc_cache_bytes(const Problem &p, size_t max_smem, int num_sms, int64_t n) {
    std::string why;
    TcPlan pl;
    if (n <= 0 || !tc_supported(p, &why) || use_row_form(p, max_smem, &pl) ||
        !best_plan(p, max_smem, true, 16, 2, &pl, &why))
        return 0;
    const char *d = getenv("NQS_TC_DENSE"), *f = getenv("NQS_TC_CONES");
    const bool force = f && f[0] == '1';
    if (pl.slots != 1 || p.n_layers < 2 || (d && d[0] == '1') || (pl.ctas != 1 && !force)) return 0;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)num_sms * pl.ctas));
    return (size_t)grid * sigma_cache_bytes(pl);
}

int launch_eloc_tc(const Problem &p, const double *, const void *packed, const int8_t *configs,
                   const double *logpsi, int64_t n, double *out, void *cache, size_t cache_bytes,
                   const LaunchEnv &env, bool f8) {
    if (n == 0) return NQS_OK;
    std::string why;
    TcPlan pl;
    if (!tc_supported(p, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    if (f8) {
        // e4m3 operands: the row form with 16 channels; the sample's log psi is always recomputed, so that
        // every ratio of the local energy is taken in the same arithmetic
        if (p.C != 16 || !use_row_form(p, env.max_smem, &pl)) {
            *env.msg = "e4m3 local energies need the row form with 16 channels";
            return NQS_ERR_UNSUPPORTED;
        }
        pl.f8 = 1;
        pl.wimg = 2u * (uint32_t)(p.n_layers - 1) * pl.wbytes;
        pl.wstride = pl.f8bytes;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)env.num_sms * pl.ctas));
        auto k = eloc_rows_kernel<16, true>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, 32 * (pl.epi + kIssuers), pl.total, env.stream>>>(pl, p, (const unsigned char *)packed, configs,
                                                                    nullptr, n, out, env.err);
        return check(env, "eloc_rows_kernel (e4m3)");
    }
    if (use_row_form(p, env.max_smem, &pl)) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)env.num_sms * pl.ctas));
        NQS_TC_DISPATCH(p.C, {
            auto k = eloc_rows_kernel<CC>;
            if (int rc = prep(k, pl, env)) return rc;
            k<<<grid, 32 * (pl.epi + kIssuers), pl.total, env.stream>>>(pl, p, (const unsigned char *)packed, configs,
                                                                        logpsi, n, out, env.err);
        });
        return check(env, "eloc_rows_kernel");
    }
    if (!best_plan(p, env.max_smem, true, 16, 2, &pl, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)env.num_sms * pl.ctas));
    const size_t need = tc_eloc_cache_bytes(p, env.max_smem, env.num_sms, n);
    unsigned char *c = (need > 0 && cache && cache_bytes >= need) ? (unsigned char *)cache : nullptr;
    NQS_TC_DISPATCH(p.C, {
        auto k = eloc_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, 32 * (pl.epi + kIssuers), pl.total, env.stream>>>(pl, p, (const unsigned char *)packed, configs,
                                                                    logpsi, n, out, env.err, c);
    });
    return check(env, "eloc_tc_kernel");
}

size_t tc_multi_table_bytes(int count) { return 256 + sizeof(TcRequest) * (size_t)count; }

int launch_eloc_tc_multi(const TcMultiItem *items, int count, void *dev_table, int max_blocks, const LaunchEnv &env) {
    if (count <= 0) return NQS_OK;
    const int C = items[0].p.C;
    std::vector<TcRequest> reqs((size_t)count);
    uint32_t smem = 0, cols = 32;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        const Problem &p = items[i].p;
        std::string why;
        TcPlan pl;
        if (p.C != C || !tc_supported(p, &why) || !best_plan(p, env.max_smem, true, 16, 1, &pl, &why)) {
            *env.msg = p.C != C ? std::string("grouped local energy needs one channel count per launch") : why;
            return NQS_ERR_UNSUPPORTED;
        }
        reqs[i].pl = pl;
        reqs[i].p = p;
        reqs[i].packed = (const unsigned char *)items[i].packed;
        reqs[i].configs = items[i].configs;
        reqs[i].logpsi = items[i].logpsi;
        reqs[i].out = items[i].out;
        reqs[i].n = items[i].n;
        reqs[i].start = total;
        total += items[i].n;
        smem = std::max(smem, pl.total);
        cols = std::max(cols, pl.tmem_cols);
    }
    if (total == 0) return NQS_OK;
    while (cols * (233472u / (smem + 1024u)) > 512u) smem += 1024u;
    if (smem > env.max_smem) { *env.msg = "grouped plan exceeds the shared-memory limit"; return NQS_ERR_UNSUPPORTED; }
    unsigned long long *counter = (unsigned long long *)dev_table;
    TcRequest *dreqs = (TcRequest *)((unsigned char *)dev_table + 256);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), env.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dreqs, reqs.data(), sizeof(TcRequest) * (size_t)count, cudaMemcpyHostToDevice, env.stream);
    if (e != cudaSuccess) { *env.msg = std::string("grouped table: ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
    const int cap = max_blocks > 0 ? std::min(max_blocks, env.num_sms) : env.num_sms;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(total, cap));
    NQS_TC_DISPATCH(C, {
        auto k = eloc_tc_multi_kernel<CC>;
        if (int rc = allow_dynamic_smem(k, smem, env)) return rc;
        k<<<grid, kTcThreads, smem, env.stream>>>(dreqs, count, total, cols, counter, env.err);
    });
    return check(env, "eloc_tc_multi_kernel");
}

namespace {

// Sampler plan: one chain per block, with as many co-resident blocks per SM
// as fit (three, two or one); chains beyond one wave of blocks run in later
// waves that the hardware schedules as blocks retire. A forward of one
// configuration is latency-bound and co-resident blocks overlap their layer
// boundaries: measured on GB300, two blocks of one chain were 1.3-1.4x faster
// than one block of two chains, and for 512 to 4,096 chains one chain per
// block (three blocks per SM where they fit) ran 1.3-1.8x faster at 10x10,
// 1.2-2.0x at t-J 12x12 and 1.3-1.7x at 16x16 with 32 channels than the
// earlier plans of 3 to 10 chains per block at one block per SM (the chains
// are the same bit for bit: a configuration's log psi does not depend on its
// row in the tile).
bool sample_plan(const Problem &p, size_t max_smem, TcPlan *out, std::string *why) {
    int fg = 0, fs = 0, fc = 1;
    const char *force = getenv("NQS_TC_SAMPLE");   // "G,slots,blocks per SM" (tuning)
    const bool forced = force && sscanf(force, "%d,%d,%d", &fg, &fs, &fc) == 3 && fc >= 1 && fc <= 3 && fg >= 1;
    if (!forced) {
        // the kernel is compiled for two blocks of kTcThreads threads, so it uses at most 96 registers a thread
        // (65,536 / 640, in steps of 8); a launch of fewer threads leaves room for a third block
        constexpr int kRegsCap = 65536 / (2 * kTcThreads) / 8 * 8;
        for (int ctas = 3; ctas >= 1; --ctas)
            if (make_plan(p, 1, 1, ctas, max_smem, sample_extra(p, 1, 1), out, why)) {
                // one epilogue warp per TMEM lane quarter (measured 8 % faster than eight warps)
                if (out->n_tiles <= 4) out->epi = 4;
                if (ctas * 32 * (out->epi + kIssuers) * kRegsCap > 65536) continue;
                return true;
            }
        return false;
    }
    for (int ctas = fc; ctas >= 1; --ctas) {   // fewer blocks per SM if the forced count does not fit
        const int slots = std::min(std::max(fs, 1), kMaxSlots);
        for (int G = std::min(fg, 16); G >= 1; --G)
            if (make_plan(p, G, slots, ctas, max_smem, sample_extra(p, G, slots), out, why)) {
                // a sampler group is one or a few tiles: one epilogue warp per
                // TMEM lane quarter (measured 8 % faster than eight warps)
                if (out->slots * out->n_tiles <= 4) out->epi = 4;
                return true;
            }
    }
    return false;
}

// Sampler grid: one block per chain group, or, when the groups outnumber the
// co-resident blocks and a group holds several chains or the context is held
// to an SM share, the co-resident blocks, each taking several groups in turn.
int64_t sample_grid(const TcPlan &pl, int64_t n_chains, int num_sms, bool sm_limited) {
    const int64_t per = (int64_t)pl.G * pl.slots, groups = (n_chains + per - 1) / per;
    if (per == 1 && !sm_limited) return groups;
    return std::min<int64_t>(groups, (int64_t)num_sms * pl.ctas);
}

}  // namespace

int launch_sample_tc(const Problem &p, const double *, const void *packed, int8_t *chains, int n_chains,
                     uint64_t step0, uint64_t seed, int spc, int sweeps_between, int burn_in, int8_t *out_cfg,
                     double *out_logpsi, const LaunchEnv &env) {
    std::string why;
    TcPlan pl;
    if (!tc_supported(p, &why) || !sample_plan(p, env.max_smem, &pl, &why)) {
        *env.msg = why;
        return NQS_ERR_UNSUPPORTED;
    }
    const int per_block = pl.G * pl.slots;
    const int grid = (int)sample_grid(pl, n_chains, env.num_sms, env.sm_limited);
    NQS_TC_DISPATCH(p.C, {
        auto k = sample_tc_kernel<CC>;
        if (int rc = prep(k, pl, env)) return rc;
        k<<<grid, 32 * (pl.epi + kIssuers), pl.total, env.stream>>>(pl, (const unsigned char *)packed, chains,
                                                                    n_chains, per_block, step0, seed, spc,
                                                                    sweeps_between, burn_in, out_cfg, out_logpsi,
                                                                    env.err, env.moves);
    });
    return check(env, "sample_tc_kernel");
}

int launch_wait_probe(int64_t iterations, const LaunchEnv &env) {
    wait_probe_kernel<<<1, 32, 0, env.stream>>>(env.err, (long long)iterations);
    return check(env, "wait_probe_kernel");
}

int tc_describe_plan(const Problem &p, int kind, int64_t n, size_t max_smem, int num_sms, int32_t *out,
                     std::string *why) {
    TcPlan pl;
    bool ok = tc_supported(p, why);
    if (ok) {
        if (kind == 2) ok = sample_plan(p, max_smem, &pl, why);
        else if (kind == 1 && use_row_form(p, max_smem, &pl)) ok = true;
        else ok = best_plan(p, max_smem, kind == 1, 16, 2, &pl, why);
    }
    if (!ok) return NQS_ERR_UNSUPPORTED;
    const int64_t per = (int64_t)pl.G * pl.slots, cap = (int64_t)num_sms * pl.ctas;
    int64_t grid;
    if (kind == 2) grid = sample_grid(pl, n, num_sms, false);
    else if (kind == 1) grid = std::max<int64_t>(1, std::min<int64_t>(n, cap));
    else grid = std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, cap));
    out[0] = pl.G;
    out[1] = pl.slots;
    out[2] = pl.ctas;
    out[3] = pl.epi;
    out[4] = pl.n_tiles;
    out[5] = (int32_t)pl.total;
    out[6] = (int32_t)pl.tmem_cols;
    out[7] = (int32_t)grid;
    out[8] = pl.rows;
    return NQS_OK;
}

}  // namespace nqs
