// The paper's two network families (Sec. 5.2, "Neural network innovations")
// on CUDA cores in type T (double or float), forward and per-sample
// backward. The paper describes them in words; the reading implemented here:
//
//   encode   CNN1: the input channels of the SiLU family (sigma = +-1, or the
//            one-hot (hole, up, down) of t-J); CNN2: X[c][s] = E[v(s)][c],
//            v = 0/1 for down/up (J1-J2), 0/1/2 for hole/up/down (t-J)
//   block b  U = periodic 3x3 convolution of X (cross-correlation) + beta_b
//            CNN1: V[c][j] = max(U[c][2j], U[c][2j+1])       (1-D max-pooling over
//                  the row-major site order, window 2, stride 2), then
//                  Y[o][2j+t] = gamma_b[o] + sum_c T_b[c][o][t] V[c][j]
//                  (transposed convolution, kernel 2, stride 2)
//            CNN2: V[c][s] = max(U[c][s], U[c][(s+1) mod N]) (stride 1, the first
//                  neuron copied to the end), then
//                  Y[o][s] = gamma_b[o] + sum_c T_b[c][o][0] V[c][s] + T_b[c][o][1] V[c][(s-1) mod N]
//   output   CNN1: the last block's transposed convolution has one channel;
//            CNN2: a final periodic 3x3 convolution to one channel (+ beta_f);
//            W(S) = product of that channel's N neurons z_s:
//            a = sum_s log|z_s|, phi = pi (number of negative z_s mod 2)
//
// Max-pooling ties go to the window's first element. The local derivatives
// are real: d a / d theta = sum_s (1 / z_s) d z_s / d theta, d phi = 0.
// Flat parameter layout (float64 vector):
//   CNN1: per block W[C][C_b][3][3], beta[C], T[C][C_o][2], gamma[C_o]
//         (C_b = c_in for the first block, else C; C_o = 1 for the last, else C)
//   CNN2: E[n_states][C]; per block W[C][C][3][3], beta[C], T[C][C][2], gamma[C];
//         W_f[1][C][3][3], beta_f[1]
#pragma once

#include "common.cuh"

namespace nqs {

__host__ __device__ inline int paper_states(const Problem &p) { return p.c_in == 1 ? 2 : 3; }

// Embedding row of a site value (CNN2).
__device__ __forceinline__ int paper_state(const Problem &p, int v) {
    if (p.c_in == 1) return v > 0 ? 1 : 0;
    return v == 0 ? 0 : (v == 1 ? 1 : 2);
}

// Parameter offsets of block b: W, beta, T, gamma; C_b inputs, C_o outputs of the transposed convolution.
struct PaperBlock {
    int w, beta, t, gamma, cin, cout;
};

__host__ __device__ inline PaperBlock paper_block(const Problem &p, int b) {
    const int C = p.C, B = p.n_layers;
    const bool cnn1 = p.net == NQS_NET_CNN1;
    int off = cnn1 ? 0 : paper_states(p) * C;
    PaperBlock k{};
    for (int i = 0; i <= b; ++i) {
        const int cin = cnn1 ? (i == 0 ? p.c_in : C) : C;
        const int cout = (cnn1 && i == B - 1) ? 1 : C;
        k.w = off; off += 9 * C * cin;
        k.beta = off; off += C;
        k.t = off; off += 2 * C * cout;
        k.gamma = off; off += cout;
        k.cin = cin;
        k.cout = cout;
    }
    return k;
}

// Offset of the final convolution's weights (CNN2): W_f[9 C], then beta_f.
__host__ __device__ inline int paper_final(const Problem &p) {
    const PaperBlock k = paper_block(p, p.n_layers - 1);
    return k.gamma + k.cout;
}

__host__ __device__ inline int paper_param_count(const Problem &p) {
    if (p.net == NQS_NET_CNN1) {
        const PaperBlock k = paper_block(p, p.n_layers - 1);
        return k.gamma + k.cout;
    }
    return paper_final(p) + 9 * p.C + 1;
}

__device__ __forceinline__ int paper_nb(int s, int k, int L) {
    const int x = s % L, y = s / L;
    return site_at(x + k % 3 - 1, y + k / 3 - 1, L);
}

// out[g][o][s] = beta[o] + sum_{c, k} W[(o cin + c) 9 + k] in[g][c][nb(s, k)], g < G, o < cout.
template <typename T>
__device__ void paper_conv(const T *__restrict__ W, const T *__restrict__ beta, const T *in, int cin, int cout, int G,
                           int N, int L, T *out) {
    for (int r = threadIdx.x; r < G * cout * N; r += blockDim.x) {
        const int g = r / (cout * N), rem = r - g * cout * N, o = rem / N, s = rem - o * N;
        T acc = beta[o];
        const T *ig = in + (size_t)g * cin * N;
        for (int c = 0; c < cin; ++c)
            for (int k = 0; k < 9; ++k) acc = fma(W[(o * cin + c) * 9 + k], ig[c * N + paper_nb(s, k, L)], acc);
        out[r] = acc;
    }
}

// V = max-pooling of U ([g][C][N] -> [g][C][M], M = N/2 for CNN1, N for CNN2).
template <typename T>
__device__ void paper_pool(bool cnn1, const T *U, int G, int C, int N, T *V) {
    const int M = cnn1 ? N / 2 : N;
    for (int r = threadIdx.x; r < G * C * M; r += blockDim.x) {
        const int gc = r / M, j = r - gc * M;
        const T *u = U + (size_t)gc * N;
        const T u0 = u[cnn1 ? 2 * j : j], u1 = u[cnn1 ? 2 * j + 1 : (j + 1 == N ? 0 : j + 1)];
        V[r] = u0 >= u1 ? u0 : u1;
    }
}

// Y[g][o][s] of the transposed convolution of V ([g][C][M]).
template <typename T>
__device__ void paper_tconv(bool cnn1, const T *__restrict__ Tw, const T *__restrict__ gamma, const T *V, int C,
                            int cout, int G, int N, T *Y) {
    const int M = cnn1 ? N / 2 : N;
    for (int r = threadIdx.x; r < G * cout * N; r += blockDim.x) {
        const int g = r / (cout * N), rem = r - g * cout * N, o = rem / N, s = rem - o * N;
        const T *vg = V + (size_t)g * C * M;
        T acc = gamma[o];
        if (cnn1) {
            const int j = s >> 1, t = s & 1;
            for (int c = 0; c < C; ++c) acc = fma(Tw[(c * cout + o) * 2 + t], vg[c * M + j], acc);
        } else {
            const int sm = s == 0 ? N - 1 : s - 1;
            for (int c = 0; c < C; ++c) {
                acc = fma(Tw[(c * cout + o) * 2], vg[c * M + s], acc);
                acc = fma(Tw[(c * cout + o) * 2 + 1], vg[c * M + sm], acc);
            }
        }
        Y[r] = acc;
    }
}

// Input of the first block for G configurations ([g][channels][N]).
template <typename T>
__device__ void paper_encode(const Problem &p, const T *__restrict__ params, const int8_t *spins, int G, T *X) {
    const int N = p.N, C = p.C;
    if (p.net == NQS_NET_CNN1) {
        for (int r = threadIdx.x; r < G * N; r += blockDim.x) {
            const int g = r / N, s = r - g * N;
            const int v = spins[r];
            if (p.c_in == 1) {
                X[(size_t)g * N + s] = (T)v;
            } else {
                T *base = X + (size_t)g * 3 * N + s;
                base[0] = (T)(v == 0);
                base[N] = (T)(v == 1);
                base[2 * N] = (T)(v == -1);
            }
        }
    } else {
        for (int r = threadIdx.x; r < G * C * N; r += blockDim.x) {
            const int g = r / (C * N), rem = r - g * C * N, c = rem / N, s = rem - c * N;
            X[r] = params[paper_state(p, spins[g * N + s]) * C + c];
        }
    }
}

// (a, phi) of G configurations from their output neurons z[g][N] (one warp
// per configuration: lanes over sites in order, then an xor tree).
template <typename T>
__device__ void paper_product(const T *z, int G, int N, double *a, double *phi) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int g = warp; g < G; g += nw) {
        double la = 0.0;
        int neg = 0;
        for (int s = lane; s < N; s += 32) {
            const double v = (double)z[(size_t)g * N + s];
            la += log(fabs(v));
            neg += v < 0.0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            la += __shfl_xor_sync(0xffffffffu, la, o);
            neg += __shfl_xor_sync(0xffffffffu, neg, o);
        }
        if (lane == 0) {
            a[g] = la;
            phi[g] = (neg & 1) ? 3.141592653589793 : 0.0;
        }
    }
}

// Forward of G configurations with two [G][C][N] buffers X, Y (contents
// destroyed); results in a[g], phi[g]. All threads of the block must call.
template <typename T>
__device__ void paper_forward(const Problem &p, const T *__restrict__ params, const int8_t *spins, int G, T *X, T *Y,
                              double *a, double *phi) {
    const int N = p.N, L = p.L, C = p.C, B = p.n_layers;
    const bool cnn1 = p.net == NQS_NET_CNN1;
    paper_encode<T>(p, params, spins, G, X);
    for (int b = 0; b < B; ++b) {
        const PaperBlock k = paper_block(p, b);
        __syncthreads();
        paper_conv<T>(params + k.w, params + k.beta, X, k.cin, C, G, N, L, Y);   // U
        __syncthreads();
        paper_pool<T>(cnn1, Y, G, C, N, X);                                      // V
        __syncthreads();
        paper_tconv<T>(cnn1, params + k.t, params + k.gamma, X, C, k.cout, G, N, Y);
        T *t = X; X = Y; Y = t;                                                  // X: block output
    }
    __syncthreads();
    if (!cnn1) {
        const int f = paper_final(p);
        paper_conv<T>(params + f, params + f + 9 * C, X, C, 1, G, N, L, Y);
        T *t = X; X = Y; Y = t;
        __syncthreads();
    }
    paper_product<T>(X, G, N, a, phi);
    __syncthreads();
}

// Per-block working set of the backward (elements of T): block inputs, the
// pre-pooling values and the pooled values of every block, the final input
// (CNN2), the output neurons and two gradient buffers.
__host__ __device__ inline size_t paper_grad_per_block(const Problem &p) {
    return (size_t)(3 * p.n_layers + 3) * p.C * p.N + p.N;
}

// Backward of one configuration. VJP = false: Oa = d a / d theta, Op = 0.
// VJP = true: acc[k] += ga d a / d theta_k (gp multiplies d phi = 0).
// Every parameter's gradient is one thread's sum over sites in order.
template <typename T, bool VJP>
__device__ void paper_grad_sample(const Problem &p, const T *__restrict__ params, const int8_t *cfg, double *Oa,
                                  double *Op, double ga, double *acc, T *base) {
    const int N = p.N, L = p.L, C = p.C, B = p.n_layers, P = p.P;
    const bool cnn1 = p.net == NQS_NET_CNN1;
    const int M = cnn1 ? N / 2 : N;
    T *Xs = base;                                   // [B][C][N] block inputs
    T *Us = Xs + (size_t)B * C * N;                 // [B][C][N] before pooling
    T *Vs = Us + (size_t)B * C * N;                 // [B][C][N] pooled ([C][M] used)
    T *Xf = Vs + (size_t)B * C * N;                 // [C][N] input of the final convolution (CNN2)
    T *z = Xf + (size_t)C * N;                      // [N] output neurons
    T *ga_buf = z + N;                              // [C][N]
    T *gb_buf = ga_buf + (size_t)C * N;             // [C][N]
    auto put = [&](int k, T v) {
        if (VJP) acc[k] += ga * (double)v;
        else Oa[k] = (double)v;
    };
    if (!VJP)
        for (int k = threadIdx.x; k < P; k += blockDim.x) Op[k] = 0.0;
    // ---------------- forward, keeping every block's values
    paper_encode<T>(p, params, cfg, 1, Xs);
    for (int b = 0; b < B; ++b) {
        const PaperBlock k = paper_block(p, b);
        T *Xb = Xs + (size_t)b * C * N, *Ub = Us + (size_t)b * C * N, *Vb = Vs + (size_t)b * C * N;
        __syncthreads();
        paper_conv<T>(params + k.w, params + k.beta, Xb, k.cin, C, 1, N, L, Ub);
        __syncthreads();
        paper_pool<T>(cnn1, Ub, 1, C, N, Vb);
        __syncthreads();
        T *Yout = b + 1 < B ? Xs + (size_t)(b + 1) * C * N : (cnn1 ? z : Xf);
        paper_tconv<T>(cnn1, params + k.t, params + k.gamma, Vb, C, k.cout, 1, N, Yout);
    }
    __syncthreads();
    if (!cnn1) {
        const int f = paper_final(p);
        paper_conv<T>(params + f, params + f + 9 * C, Xf, C, 1, 1, N, L, z);
        __syncthreads();
    }
    // ---------------- backward; g = d a / d (current tensor)
    T *g = ga_buf, *gn = gb_buf;
    for (int s = threadIdx.x; s < N; s += blockDim.x) g[s] = T(1) / z[s];
    __syncthreads();
    if (!cnn1) {
        // final convolution (one output channel): dW_f[c][k], dbeta_f, then g over its input Xf
        const int f = paper_final(p);
        for (int e = threadIdx.x; e < 9 * C + 1; e += blockDim.x) {
            T v = 0;
            if (e < 9 * C) {
                const int c = e / 9, k = e - c * 9;
                for (int s = 0; s < N; ++s) v = fma(g[s], Xf[c * N + paper_nb(s, k, L)], v);
            } else {
                for (int s = 0; s < N; ++s) v += g[s];
            }
            put(f + e, v);
        }
        // adjoint of the padded convolution: input site s' collects the outputs s = s' - d_k that read it
        for (int r = threadIdx.x; r < C * N; r += blockDim.x) {
            const int c = r / N, s = r - c * N;
            T v = 0;
            for (int k = 0; k < 9; ++k) v = fma(params[f + c * 9 + k], g[paper_nb(s, 8 - k, L)], v);
            gn[r] = v;
        }
        __syncthreads();
        T *t = g; g = gn; gn = t;
    }
    for (int b = B - 1; b >= 0; --b) {
        const PaperBlock k = paper_block(p, b);
        const T *Xb = Xs + (size_t)b * C * N, *Ub = Us + (size_t)b * C * N, *Vb = Vs + (size_t)b * C * N;
        const int co = k.cout;
        // transposed convolution: dgamma, dT; gV (into gn, [C][M])
        for (int e = threadIdx.x; e < co + 2 * C * co; e += blockDim.x) {
            T v = 0;
            if (e < co) {
                for (int s = 0; s < N; ++s) v += g[e * N + s];
                put(k.gamma + e, v);
            } else {
                const int q = e - co, c = q / (2 * co), rem = q - c * 2 * co, o = rem / 2, t = rem - o * 2;
                if (cnn1) {
                    for (int j = 0; j < M; ++j) v = fma(g[o * N + 2 * j + t], Vb[c * M + j], v);
                } else {
                    for (int s = 0; s < N; ++s)
                        v = fma(g[o * N + s], Vb[c * M + (t == 0 ? s : (s == 0 ? N - 1 : s - 1))], v);
                }
                put(k.t + (c * co + o) * 2 + t, v);
            }
        }
        for (int r = threadIdx.x; r < C * M; r += blockDim.x) {
            const int c = r / M, j = r - c * M;
            T v = 0;
            for (int o = 0; o < co; ++o) {
                if (cnn1) {
                    v = fma(params[k.t + (c * co + o) * 2], g[o * N + 2 * j], v);
                    v = fma(params[k.t + (c * co + o) * 2 + 1], g[o * N + 2 * j + 1], v);
                } else {
                    v = fma(params[k.t + (c * co + o) * 2], g[o * N + j], v);
                    v = fma(params[k.t + (c * co + o) * 2 + 1], g[o * N + (j + 1 == N ? 0 : j + 1)], v);
                }
            }
            gn[r] = v;   // gV[c][j]
        }
        __syncthreads();
        // max-pooling: gU[c][s] (into g) from gV (gn); the window's first element wins ties
        for (int r = threadIdx.x; r < C * N; r += blockDim.x) {
            const int c = r / N, s = r - c * N;
            const T *u = Ub + (size_t)c * N;
            T v = 0;
            if (cnn1) {
                const int j = s >> 1;
                const bool first = u[2 * j] >= u[2 * j + 1];
                if ((s & 1) == (first ? 0 : 1)) v = gn[c * M + j];
            } else {
                const int sn = s + 1 == N ? 0 : s + 1, sp = s == 0 ? N - 1 : s - 1;
                if (u[s] >= u[sn]) v += gn[c * N + s];          // window s picked s
                if (!(u[sp] >= u[s])) v += gn[c * N + sp];      // window s - 1 picked s
            }
            g[r] = v;
        }
        __syncthreads();
        // convolution: dW[o][c][k], dbeta[o]; gX (into gn) through the adjoint of the periodic padding
        const int cin = k.cin;
        for (int e = threadIdx.x; e < 9 * C * cin + C; e += blockDim.x) {
            T v = 0;
            if (e < 9 * C * cin) {
                const int o = e / (9 * cin), rem = e - o * 9 * cin, c = rem / 9, kk = rem - c * 9;
                for (int s = 0; s < N; ++s) v = fma(g[o * N + s], Xb[c * N + paper_nb(s, kk, L)], v);
                put(k.w + e, v);
            } else {
                const int o = e - 9 * C * cin;
                for (int s = 0; s < N; ++s) v += g[o * N + s];
                put(k.beta + o, v);
            }
        }
        if (b > 0 || !cnn1) {
            for (int r = threadIdx.x; r < cin * N; r += blockDim.x) {
                const int c = r / N, s = r - c * N;
                T v = 0;
                for (int o = 0; o < C; ++o)
                    for (int kk = 0; kk < 9; ++kk)
                        v = fma(params[k.w + (o * cin + c) * 9 + kk], g[o * N + paper_nb(s, 8 - kk, L)], v);
                gn[r] = v;
            }
        }
        __syncthreads();
        T *t = g; g = gn; gn = t;
    }
    if (!cnn1) {
        // embedding rows: dE[state][c] = sum of gX[c][s] over the sites in that state
        const int ns = paper_states(p);
        for (int e = threadIdx.x; e < ns * C; e += blockDim.x) {
            const int st = e / C, c = e - st * C;
            T v = 0;
            for (int s = 0; s < N; ++s)
                if (paper_state(p, cfg[s]) == st) v += g[c * N + s];
            put(e, v);
        }
    }
    __syncthreads();
}

}  // namespace nqs
