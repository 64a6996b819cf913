// Device helpers shared by the kernels: problem description, lattice
// geometry, Philox4x64-10, block-wide scans/reductions in a fixed order, and
// the enumeration of connected configurations (Eq. 2, Eq. 3).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nqs.h"

namespace nqs {

// Device-side error bits latched in the context (read by nqs_sync).
enum : int { ERRBIT_NONFINITE = 1, ERRBIT_TIMEOUT = 2, ERRBIT_BOUNDS = 4 };

// Index check of the checked build (NQS_CHECK): false, with the bounds bit set, when cond fails; the caller then
// skips the access. In the default build it is the constant true and compiles away.
#ifdef NQS_CHECK
#define NQS_INDEX_OK(cond, err) ((cond) ? true : (atomicOr((err), ERRBIT_BOUNDS), false))
#else
#define NQS_INDEX_OK(cond, err) true
#endif

struct Problem {
    int model;      // NQS_MODEL_J1J2 / NQS_MODEL_TJ
    int L, N;
    int c_in;       // 1 (J1-J2) or 3 (t-J)
    int C;          // channels
    int n_layers;
    double J1, J2, t, J;
    int sign_rule;
    int P;          // parameter count
    int n_bonds;    // 4N (J1-J2) or 2N (t-J)
    int n_up, n_down;
    int net;        // NQS_NET_SILU, NQS_NET_CNN1, NQS_NET_CNN2
};

// Offset of layer l's weights in the flat parameter vector; its bias
// follows at + 9 * cin * C.
__host__ __device__ inline int layer_offset(const Problem &p, int l) {
    if (l == 0) return 0;
    int first = 9 * p.c_in * p.C + p.C;
    return first + (l - 1) * (9 * p.C * p.C + p.C);
}
__host__ __device__ inline int layer_cin(const Problem &p, int l) { return l == 0 ? p.c_in : p.C; }
__host__ __device__ inline int head_offset(const Problem &p) { return layer_offset(p, p.n_layers); }

__device__ __forceinline__ int wrap(int v, int L) { v %= L; return v < 0 ? v + L : v; }
__device__ __forceinline__ int site_at(int x, int y, int L) { return wrap(y, L) * L + wrap(x, L); }

// Bond b of the bond list: site-major, then direction (x+1), (y+1),
// (x+1, y+1), (x+1, y-1); the t-J model uses only the first two.
__device__ __forceinline__ void bond_sites(const Problem &p, int b, int &i, int &j, bool &nnn) {
    const int per = (p.model == NQS_MODEL_J1J2) ? 4 : 2;
    i = b / per;
    const int d = b - i * per;
    const int x = i % p.L, y = i / p.L;
    const int dx = (d == 1) ? 0 : 1;
    const int dy = (d == 0) ? 0 : (d == 3 ? -1 : 1);
    j = site_at(x + dx, y + dy, p.L);
    nnn = d >= 2;
}

// Snake (boustrophedon) position of a site, and the site at a position.
__device__ __forceinline__ int snake_pos(int i, int L) {
    const int x = i % L, y = i / L;
    return y * L + ((y & 1) ? (L - 1 - x) : x);
}
__device__ __forceinline__ int snake_site(int p, int L) {
    const int y = p / L, xs = p - y * L;
    return y * L + ((y & 1) ? (L - 1 - xs) : xs);
}

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon et al., SC'11): ten rounds of two 64x64 -> 128-bit
// multiplications with a Feistel-like word permutation, key bumped by the
// Weyl constants between rounds.
struct Philox4 { uint64_t v[4]; };

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ Philox4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                   uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = mulhi64(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = mulhi64(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
    Philox4 out;
    out.v[0] = c0; out.v[1] = c1; out.v[2] = c2; out.v[3] = c3;
    return out;
}

// ---------------------------------------------------------------- block helpers
// Sum of one double per thread over the block, in a fixed tree order
// (result valid in every thread). scratch: >= 32 doubles of shared memory.
__device__ inline double block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = lane < nw ? scratch[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) scratch[32] = w;
    }
    __syncthreads();
    const double r = scratch[32];
    __syncthreads();
    return r;
}

// Sum over k < n of the pairs value(k) = (x, y), in an order that does not
// depend on the block size: item k goes to partial sum k mod 128 (items in
// increasing k), then warp 0 adds the 128 partials in a fixed tree. Needs
// blockDim.x >= 32; scratch: >= 258 doubles of shared memory. Result valid in
// every thread.
template <typename F>
__device__ inline double2 fixed_order_sum2(int n, F value, double *scratch) {
    for (int v = threadIdx.x; v < 128; v += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int k = v; k < n; k += 128) {
            const double2 t = value(k);
            x += t.x;
            y += t.y;
        }
        scratch[v] = x;
        scratch[128 + v] = y;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int l = threadIdx.x;
        double x = (scratch[l] + scratch[l + 32]) + (scratch[l + 64] + scratch[l + 96]);
        double y = (scratch[128 + l] + scratch[160 + l]) + (scratch[192 + l] + scratch[224 + l]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (l == 0) { scratch[256] = x; scratch[257] = y; }
    }
    __syncthreads();
    const double2 r = make_double2(scratch[256], scratch[257]);
    __syncthreads();
    return r;
}

// Exclusive prefix sum of one int flag per thread over the block; returns
// the thread's offset and writes the block total to *total. scratch: >= 33 ints.
__device__ inline int block_exclusive_scan(int v, int *scratch, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? scratch[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    const int off = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();
    return off;
}

// ---------------------------------------------------------------- enumeration
// Connected configurations of the configuration in `sigma` (shared memory,
// int8 [N]), in bond order: the swapped pairs go to ci/cj, the matrix
// elements to ch, the count is returned; the diagonal element goes to *hdiag.
// cum_snake: shared int scratch [N + 1] (t-J only). scratch: >= 33 ints and
// >= 33 doubles. All threads of the block must call this.
struct EnumScratch { int iscr[34]; double dscr[34]; };

// Diagonal element H_{sigma sigma} from integer sums over bonds (exact, so it
// does not depend on how the bonds are split among threads). J1-J2 (Eq. of
// the J1-J2 model): s1 = sum over NN bonds of s_i s_j, s2 = the same over NNN
// bonds, with s = +-1, giving (J1 s1 + J2 s2) / 4. t-J: s1 = sum of s_i s_j
// over NN bonds holding two electrons, s2 = the number of those bonds, giving
// J (s1 / 4 - s2 / 4).
__device__ __forceinline__ double diagonal_element(const Problem &p, int s1, int s2) {
    if (p.model == NQS_MODEL_J1J2) return 0.25 * (p.J1 * (double)s1 + p.J2 * (double)s2);
    return p.J * (0.25 * (double)s1 - 0.25 * (double)s2);
}

__device__ inline int enumerate_connected(const Problem &p, const int8_t *sigma, int16_t *ci, int16_t *cj,
                                          double *ch, double *hdiag, int *cum_snake, EnumScratch &es) {
    const int N = p.N;
    if (p.model == NQS_MODEL_TJ) {
        // cum_snake[q] = electrons at snake positions < q
        int base = 0;
        for (int q0 = 0; q0 < N; q0 += blockDim.x) {
            const int q = q0 + threadIdx.x;
            const int occ = (q < N) ? (sigma[snake_site(q, p.L)] != 0) : 0;
            int tot;
            const int off = block_exclusive_scan(occ, es.iscr, &tot);
            if (q < N) cum_snake[q] = base + off;
            base += tot;
        }
        if (threadIdx.x == 0) cum_snake[N] = base;
        __syncthreads();
    }
    int d1 = 0, d2 = 0;   // integer sums of s_i s_j (see diagonal_element)
    int count = 0;
    for (int b0 = 0; b0 < p.n_bonds; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        int flag = 0;
        int i = 0, j = 0;
        double h = 0.0;
        if (b < p.n_bonds) {
            bool nnn;
            bond_sites(p, b, i, j, nnn);
            const int si = sigma[i], sj = sigma[j];
            if (p.model == NQS_MODEL_J1J2) {
                const double Jb = nnn ? p.J2 : p.J1;
                if (nnn) d2 += si * sj; else d1 += si * sj;
                if (si != sj) {
                    flag = 1;
                    h = 0.5 * Jb;
                    if (p.sign_rule && !nnn) h = -h;
                }
            } else {
                if (si != 0 && sj != 0) {
                    d1 += si * sj;
                    d2 += 1;
                    if (si != sj) { flag = 1; h = 0.5 * p.J; }
                } else if ((si == 0) != (sj == 0)) {
                    flag = 1;
                    int pi = snake_pos(i, p.L), pj = snake_pos(j, p.L);
                    const int lo = pi < pj ? pi : pj, hi = pi < pj ? pj : pi;
                    const int between = cum_snake[hi] - cum_snake[lo + 1];
                    h = (between & 1) ? p.t : -p.t;
                }
            }
        }
        int tot;
        const int off = block_exclusive_scan(flag, es.iscr, &tot);
        if (flag) {
            ci[count + off] = (int16_t)i;
            cj[count + off] = (int16_t)j;
            ch[count + off] = h;
        }
        count += tot;
    }
    int t1, t2;
    block_exclusive_scan(d1, es.iscr, &t1);
    block_exclusive_scan(d2, es.iscr, &t2);
    if (hdiag) *hdiag = diagonal_element(p, t1, t2);
    __syncthreads();
    return count;
}

// Electron counts along the snake path for the t-J hop signs:
// cum_snake[q] = electrons at snake positions < q (q = 0..N). All threads.
__device__ inline void snake_prefix(const Problem &p, const int8_t *sigma, int *cum_snake, EnumScratch &es) {
    int base = 0;
    for (int q0 = 0; q0 < p.N; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const int occ = (q < p.N) ? (sigma[snake_site(q, p.L)] != 0) : 0;
        int tot;
        const int off = block_exclusive_scan(occ, es.iscr, &tot);
        if (q < p.N) cum_snake[q] = base + off;
        base += tot;
    }
    if (threadIdx.x == 0) cum_snake[p.N] = base;
    __syncthreads();
}

// Connected configurations from bonds [b_begin, b_end) only, in bond order
// (same rules as enumerate_connected); *hdiag receives the diagonal part of
// those bonds. For t-J, cum_snake must hold snake_prefix of sigma.
__device__ inline int enumerate_range(const Problem &p, const int8_t *sigma, int b_begin, int b_end, int16_t *ci,
                                      int16_t *cj, double *ch, double *hdiag, const int *cum_snake, EnumScratch &es) {
    int d1 = 0, d2 = 0;   // integer sums of s_i s_j (see diagonal_element)
    int count = 0;
    for (int b0 = b_begin; b0 < b_end; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        int flag = 0;
        int i = 0, j = 0;
        double h = 0.0;
        if (b < b_end) {
            bool nnn;
            bond_sites(p, b, i, j, nnn);
            const int si = sigma[i], sj = sigma[j];
            if (p.model == NQS_MODEL_J1J2) {
                const double Jb = nnn ? p.J2 : p.J1;
                if (nnn) d2 += si * sj; else d1 += si * sj;
                if (si != sj) {
                    flag = 1;
                    h = 0.5 * Jb;
                    if (p.sign_rule && !nnn) h = -h;
                }
            } else {
                if (si != 0 && sj != 0) {
                    d1 += si * sj;
                    d2 += 1;
                    if (si != sj) { flag = 1; h = 0.5 * p.J; }
                } else if ((si == 0) != (sj == 0)) {
                    flag = 1;
                    const int pi = snake_pos(i, p.L), pj = snake_pos(j, p.L);
                    const int lo = pi < pj ? pi : pj, hi = pi < pj ? pj : pi;
                    h = ((cum_snake[hi] - cum_snake[lo + 1]) & 1) ? p.t : -p.t;
                }
            }
        }
        int tot;
        const int off = block_exclusive_scan(flag, es.iscr, &tot);
        if (flag) {
            ci[count + off] = (int16_t)i;
            cj[count + off] = (int16_t)j;
            ch[count + off] = h;
        }
        count += tot;
    }
    int t1, t2;
    block_exclusive_scan(d1, es.iscr, &t1);
    block_exclusive_scan(d2, es.iscr, &t2);
    if (hdiag) *hdiag = diagonal_element(p, t1, t2);
    __syncthreads();
    return count;
}

__device__ __forceinline__ double silu_d(double z) { return z / (1.0 + exp(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }

}  // namespace nqs
