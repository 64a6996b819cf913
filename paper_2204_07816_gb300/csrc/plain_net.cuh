// Network evaluation on CUDA cores in type T (double or float): the
// periodic 3x3 convolution stack with SiLU and the sum-pooled two-output
// head (Eq. 1 wave function; periodic padding of Sec. 5.4.2 folded into the
// neighbour index arithmetic). One thread block evaluates G configurations
// at a time with every activation in shared memory.
#pragma once

#include "common.cuh"
#include "paper_net.cuh"

namespace nqs {

template <typename T> __device__ __forceinline__ T silu_t(T z);
template <> __device__ __forceinline__ double silu_t<double>(double z) { return silu_d(z); }
template <> __device__ __forceinline__ float silu_t<float>(float z) { return silu_f(z); }

// Shared-memory carve-up of one plain evaluator (sizes in bytes, 16-aligned).
struct PlainLayout {
    size_t act;     // one activation buffer: G * C * N * sizeof(T)
    size_t w;       // staged weights of one layer: (9 * C * C + C) * sizeof(T)
    size_t hbar;    // G * C * sizeof(T)
    size_t total;   // 2 * act + w + hbar + 2 * G * sizeof(double)
    int G;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

template <typename T>
__host__ __device__ inline PlainLayout plain_layout(const Problem &p, int G) {
    PlainLayout l;
    l.act = align16((size_t)G * p.C * p.N * sizeof(T));
    l.w = align16((size_t)(9 * p.C * p.C + p.C) * sizeof(T));
    l.hbar = align16((size_t)G * p.C * sizeof(T));
    l.total = 2 * l.act + l.w + l.hbar + align16(2 * (size_t)G * sizeof(double));
    l.G = G;
    return l;
}

template <typename T>
struct PlainNet {
    T *act0, *act1, *w, *hbar;
    double *a, *phi;   // [G] results

    __device__ void bind(unsigned char *base, const PlainLayout &l) {
        act0 = reinterpret_cast<T *>(base);
        act1 = reinterpret_cast<T *>(base + l.act);
        w = reinterpret_cast<T *>(base + 2 * l.act);
        hbar = reinterpret_cast<T *>(base + 2 * l.act + l.w);
        a = reinterpret_cast<double *>(base + 2 * l.act + l.w + l.hbar);
        phi = a + l.G;
    }
};

// Evaluate (a, phi) for the G configurations in spins[g * N + site]
// (shared memory). params: layer weights in type T (flat layout);
// params64: the float64 vector (head read in float64). Results in net.a,
// net.phi. All threads of the block must call.
// PN: the paper's CNN1 / CNN2 (p.net), a separate instantiation so that the
// SiLU kernels carry none of its code (it cost them registers: measured
// 1.6-2.3x slower FP32 local energies and sampling when the families shared
// one kernel).
template <typename T, int CB, bool PN = false>
__device__ void plain_forward(const Problem &p, const T *__restrict__ params, const double *__restrict__ params64,
                              const int8_t *spins, int G, PlainNet<T> &net) {
    if constexpr (PN) {
        paper_forward<T>(p, params, spins, G, net.act0, net.act1, net.a, net.phi);
        return;
    }
    const int N = p.N, L = p.L, C = p.C;
    // input encoding: J1-J2 one channel (+-1), t-J one-hot (hole, up, down)
    for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
        const int g = r / N, s = r - g * N;
        const int v = spins[r];
        if (p.c_in == 1) {
            net.act0[g * N + s] = (T)v;
        } else {
            T *base = net.act0 + (size_t)g * 3 * N + s;
            base[0] = (T)(v == 0);
            base[N] = (T)(v == 1);
            base[2 * N] = (T)(v == -1);
        }
    }
    T *in = net.act0, *out = net.act1;
    for (int l = 0; l < p.n_layers; ++l) {
        const int cin = layer_cin(p, l);
        const int off = layer_offset(p, l);
        __syncthreads();
        // stage weights as w[(o * cin + c) * C + co], o = ky * 3 + kx; bias after
        for (int e = threadIdx.x; e < 9 * cin * C; e += blockDim.x) {
            const int co = e / (9 * cin);
            const int rem = e - co * 9 * cin;
            const int c = rem / 9, o = rem - c * 9;
            net.w[(o * cin + c) * C + co] = params[off + e];
        }
        for (int e = threadIdx.x; e < C; e += blockDim.x) net.w[9 * cin * C + e] = params[off + 9 * cin * C + e];
        __syncthreads();
        const T *bias = net.w + 9 * cin * C;
        for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
            const int g = r / N, s = r - g * N;
            const int x = s % L, y = s / L;
            int nb[9];
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) nb[ky * 3 + kx] = site_at(x + kx - 1, y + ky - 1, L);
            const T *ing = in + (size_t)g * cin * N;
            for (int cb = 0; cb < C; cb += CB) {
                T acc[CB];
#pragma unroll
                for (int q = 0; q < CB; ++q) acc[q] = bias[cb + q];
                for (int o = 0; o < 9; ++o) {
                    for (int c = 0; c < cin; ++c) {
                        const T v = ing[c * N + nb[o]];
                        const T *wr = net.w + (o * cin + c) * C + cb;
#pragma unroll
                        for (int q = 0; q < CB; ++q) acc[q] = fma(wr[q], v, acc[q]);
                    }
                }
                T *og = out + (size_t)g * C * N + s;
#pragma unroll
                for (int q = 0; q < CB; ++q) og[(cb + q) * N] = silu_t<T>(acc[q]);
            }
        }
        T *t = in; in = out; out = t;
    }
    __syncthreads();
    // head: hbar[g][c] = sum over sites (one warp per (g, c), fixed order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int task = warp; task < G * C; task += nw) {
        const T *h = in + (size_t)task * N;
        T v = 0;
        for (int s = lane; s < N; s += 32) v += h[s];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) net.hbar[task] = v;
    }
    __syncthreads();
    const int ho = head_offset(p);
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        double sa = 0.0, sp = 0.0;
        for (int c = 0; c < C; ++c) {
            const double hb = (double)net.hbar[g * C + c];
            sa = fma(params64[ho + c], hb, sa);
            sp = fma(params64[ho + C + c], hb, sp);
        }
        net.a[g] = sa;
        net.phi[g] = sp;
    }
    __syncthreads();
}

}  // namespace nqs
