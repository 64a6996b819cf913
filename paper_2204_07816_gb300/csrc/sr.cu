// Stochastic reconfiguration solve (Sec. 3.2; Sec. 5.4.1 "Distributed SR
// computation"). The paper builds the covariance matrix S explicitly and
// factorises it; here S is never formed:
//   (S + eps I) x = Ohat^T (Ohat x - mean) / n + eps x
// with Ohat the real-stacked [2n, P] matrix of local derivatives, and the
// system is solved by conjugate gradient, its vectors and scalars in
// float64 and its two passes over O per iteration in double-float (default)
// or float64 arithmetic (below). Every reduction runs in a fixed order, so
// results do not depend on what else runs on the GPU.
//
// Sample-space form (run_sr_woodbury): the same delta is
//   delta = Ohat^T y,   (Ohat Ohat^T / n + eps I) y = Ehat / n,
// since (Ohat^T Ohat / n + eps I)^-1 Ohat^T = Ohat^T (Ohat Ohat^T / n + eps I)^-1.
// The 2n x 2n matrix is formed (centred Gram matrix, lower triangle) and
// factorised by a blocked right-looking Cholesky, as the paper factorises S.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace nqs {

namespace {

// scalar slots in the workspace
enum : int { S_ERE = 0, S_EIM, S_RS, S_FNORM, S_DONE, S_ITER, S_MEANRE, S_MEANIM, S_WBRES, S_WIDE, S_COUNT = 16 };
// P-vector kernels of a CG iteration run on ceil(P / kPvThreads) blocks (a grid that depends on P only, so the
// partial sums and their fixed-order reduction do not depend on the device)
constexpr int kPvThreads = 256;

constexpr int kRowWarps = 8;    // rows per block in the row GEMV
constexpr int kColThreads = 256;
constexpr int kVecThreads = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// A float64 as a double-float h + l (the S.x passes below read vectors in this form).
__device__ __forceinline__ float2 df_of(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// Block-wide fixed-order sum (blockDim.x == kVecThreads).
__device__ double vec_block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double w = 0.0;
    if (warp == 0) {
        w = warp_sum(sh[lane]);
        if (lane == 0) sh[32] = w;
    }
    __syncthreads();
    w = sh[32];
    __syncthreads();
    return w;
}

// <E> and the centred energies Ehat = [Re(E - <E>); Im(E - <E>)] (into y).
__global__ void __launch_bounds__(kVecThreads) energy_kernel(const double *eloc, int64_t n, double *y, double *sc) {
    __shared__ double sh[33];
    double pr = 0.0, pi = 0.0;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) { pr += eloc[2 * s]; pi += eloc[2 * s + 1]; }
    const double er = vec_block_sum(pr, sh) / (double)n;
    const double ei = vec_block_sum(pi, sh) / (double)n;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
        y[s] = eloc[2 * s] - er;
        y[n + s] = eloc[2 * s + 1] - ei;
    }
    if (threadIdx.x == 0) {
        sc[S_ERE] = er;
        sc[S_EIM] = ei;
        sc[S_DONE] = 0.0;
        sc[S_ITER] = 0.0;
        sc[S_WIDE] = 0.0;
    }
}

// y[r] = Ohat[r, :] . v  (one warp per row, lanes strided over columns)
__global__ void __launch_bounds__(kRowWarps * 32) gemv_rows_kernel(const double *__restrict__ O, const double *__restrict__ v,
                                                                   int64_t rows, int P, double *__restrict__ y,
                                                                   const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    if (r >= rows) return;
    const double *row = O + r * (int64_t)P;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int k = lane;
    for (; k + 96 < P; k += 128) {
        a0 = fma(row[k], v[k], a0);
        a1 = fma(row[k + 32], v[k + 32], a1);
        a2 = fma(row[k + 64], v[k + 64], a2);
        a3 = fma(row[k + 96], v[k + 96], a3);
    }
    for (; k < P; k += 32) a0 = fma(row[k], v[k], a0);
    const double s = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) y[r] = s;
}

// ---------------------------------------------------------------- double-float S.x passes
// GB300 runs float64 FMAs at 1/64 of its float32 rate, and one float64 FMA
// per element of O kept the FP64 pipe 82-86 % busy in the passes above while
// HBM ran at half its bandwidth. The conjugate gradient therefore splits O
// once per solve, in the pass that computes the force, into double-floats
// (each element the unevaluated sum h + l of two floats, stored as a plane of
// h and a plane of l), and its S.x passes multiply-add in double-float
// arithmetic on the float32 pipes; float64 returns only for the row or column
// totals. Products keep about 46 bits (the split truncates at 2^-46 of the
// element, the l * l term is dropped) and every accumulation is a
// renormalised double-float add, so a dot product's error stays near 1e-15 of
// the sum of its terms' magnitudes (float64: about 1e-17). Where every
// element of O is a float (the float32 and bf16 local derivatives are), every
// l is zero: the split pass records whether any l is not, the l plane is
// written (by a second pass over O) only then, and otherwise the passes read
// the h plane alone, half the bytes, with the same results.

// a + b, both double-floats: two-sum of the high parts, then renormalised.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    const float u = __fadd_rn(t, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, u);
    return make_float2(h, __fsub_rn(u, __fsub_rn(h, s)));
}

// acc + (ah + al) q for q = q.x + q.y: the exact product of the high parts (its
// rounding error by one FMA) plus the two cross terms.
__device__ __forceinline__ float2 df_fma(float ah, float al, float2 q, float2 acc) {
    const float p = __fmul_rn(ah, q.x);
    float e = fmaf(ah, q.x, -p);
    e = fmaf(ah, q.y, e);
    e = fmaf(al, q.x, e);
    return df_add(acc, make_float2(p, e));
}

__device__ __forceinline__ double df_value(float2 a) { return (double)a.x + (double)a.y; }

// A float64 (its two 32-bit words, w.x low, w.y high) as h + l by integer
// operations, which leave the FP64 pipe to the force's FMAs in the same pass:
// h carries the sign, the exponent rebiased and the top 23 mantissa bits, l
// the next 23 bits (bits 28 .. 6 of the low word) as an integer float times
// +-2^(E - 1069); |a - h - l| < 2^-46 |a|, and l = 0 exactly when a is a
// float (its low 29 mantissa bits are zero). |a| < 2^-80 (zero, subnormals:
// nothing an entry of O could add to a sum of O(1) terms) gives 0;
// |a| >= 2^128, Inf and NaN give NaN.
__device__ __forceinline__ float2 df_split_bits(uint2 w) {
    const uint32_t sgn = w.y & 0x80000000u, t = w.y & 0x7FFFFFFFu;
    const float h = __uint_as_float((((t - (896u << 20)) << 3) | (w.x >> 29)) | sgn);
    const float m = __fsub_rn(__uint_as_float(0x4B000000u | ((w.x >> 6) & 0x7FFFFFu)), 8388608.f);
    const float l = __fmul_rn(m, __uint_as_float((((t - (942u << 20)) >> 20) << 23) | sgn));
    const bool tiny = t < (943u << 20), huge = t >= (1151u << 20);
    return huge ? make_float2(__int_as_float(0x7FC00000), 0.f) : (tiny ? make_float2(0.f, 0.f) : make_float2(h, l));
}

// The force pass: zpart[chunk][k] = sum over the chunk's rows r of O[r, k] y[r]
// in float64, in gemv_cols_kernel's order (the same sums), and every element
// of O split into h + l with h written to the plane Oh (row stride Pp = P
// rounded up to a multiple of 4, the pad columns zero); sc[S_WIDE] = 1 if any
// l is not zero, and split_low_kernel then writes the l plane.
__global__ void __launch_bounds__(kColThreads) gemv_cols_split_kernel(const double *__restrict__ O,
                                                                      const double *__restrict__ y, int64_t rows, int P,
                                                                      int Pp, int64_t chunk_rows,
                                                                      double *__restrict__ zpart,
                                                                      float *__restrict__ Oh, double *sc) {
    if (sc[S_DONE] != 0.0) return;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
    const int64_t r1 = rows < r0 + chunk_rows ? rows : r0 + chunk_rows;
    bool wide = false;
    if (k < P) {
        const uint2 *col = reinterpret_cast<const uint2 *>(O) + k;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int64_t r = r0;
        for (; r + 3 < r1; r += 4) {
            uint2 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = __ldcs(col + (r + u) * P);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 d = df_split_bits(w[u]);
                __stcs(Oh + (r + u) * Pp + k, d.x);
                wide |= d.y != 0.f;
            }
            a0 = fma(__hiloint2double((int)w[0].y, (int)w[0].x), y[r], a0);
            a1 = fma(__hiloint2double((int)w[1].y, (int)w[1].x), y[r + 1], a1);
            a2 = fma(__hiloint2double((int)w[2].y, (int)w[2].x), y[r + 2], a2);
            a3 = fma(__hiloint2double((int)w[3].y, (int)w[3].x), y[r + 3], a3);
        }
        for (; r < r1; ++r) {
            const uint2 w = __ldcs(col + r * P);
            const float2 d = df_split_bits(w);
            __stcs(Oh + r * Pp + k, d.x);
            wide |= d.y != 0.f;
            a0 = fma(__hiloint2double((int)w.y, (int)w.x), y[r], a0);
        }
        zpart[(int64_t)blockIdx.y * P + k] = (a0 + a1) + (a2 + a3);
    } else if (k < Pp) {
        for (int64_t r = r0; r < r1; ++r) Oh[r * Pp + k] = 0.f;
    }
    // the same value from every writer
    if (__any_sync(0xffffffffu, wide) && (threadIdx.x & 31) == 0) sc[S_WIDE] = 1.0;
}

// The l plane, only when the force pass found an l that is not zero (O not
// made of floats): every element split again, the pad columns zero. Rows
// r = blockIdx.y, blockIdx.y + gridDim.y, ...
__global__ void __launch_bounds__(kColThreads) split_low_kernel(const double *__restrict__ O, int64_t rows, int P,
                                                                int Pp, float *__restrict__ Ol, const double *sc) {
    if (sc[S_DONE] != 0.0 || sc[S_WIDE] == 0.0) return;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    if (k >= Pp) return;
    const uint2 *col = reinterpret_cast<const uint2 *>(O) + k;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y)
        __stcs(Ol + r * Pp + k, k < P ? df_split_bits(__ldcs(col + r * P)).y : 0.f);
}

// acc[j] += x[j] q[j] for the four columns of a float4 group (l parts zero
// unless W).
template <bool W>
__device__ __forceinline__ void df_fma4(float2 (&acc)[4], float4 h, float4 l, float2 q0, float2 q1, float2 q2,
                                        float2 q3) {
    acc[0] = df_fma(h.x, W ? l.x : 0.f, q0, acc[0]);
    acc[1] = df_fma(h.y, W ? l.y : 0.f, q1, acc[1]);
    acc[2] = df_fma(h.z, W ? l.z : 0.f, q2, acc[2]);
    acc[3] = df_fma(h.w, W ? l.w : 0.f, q3, acc[3]);
}

// y[r] = O[r, :] . v from the planes (one warp per row; lane i takes the float4
// column groups i, i + 32, ...; accumulator j the j-th column of each group;
// W: read the l plane too). The next U groups of each lane are loaded before
// the current ones are consumed, so a warp keeps its loads in flight while it
// computes. v holds Pp double-floats (zero past P). The order of every sum
// does not depend on W or U, so a zero l plane gives the same y either way.
template <bool W, int U>
__device__ __forceinline__ void rows_df(const float *__restrict__ Oh, const float *__restrict__ Ol,
                                        const float2 *__restrict__ v, int64_t r, int Pp, double *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int n4 = Pp >> 2;
    const float4 *rh = reinterpret_cast<const float4 *>(Oh + r * (int64_t)Pp);
    const float4 *rl = reinterpret_cast<const float4 *>(Ol + r * (int64_t)Pp);
    const float4 *v4 = reinterpret_cast<const float4 *>(v);   // two double-floats each
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = make_float2(0.f, 0.f);
    int c = lane;
    float4 oh[U], ol[U];
    if (c + 32 * (U - 1) < n4) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            oh[u] = __ldcs(rh + c + 32 * u);
            ol[u] = W ? __ldcs(rl + c + 32 * u) : zero4;
        }
    }
    while (c + 32 * (U - 1) < n4) {
        const int cn = c + 32 * U;
        const bool more = cn + 32 * (U - 1) < n4;
        float4 nh[U], nl[U];
        if (more) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                nh[u] = __ldcs(rh + cn + 32 * u);
                nl[u] = W ? __ldcs(rl + cn + 32 * u) : zero4;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 qa = v4[2 * (c + 32 * u)], qb = v4[2 * (c + 32 * u) + 1];
            df_fma4<W>(acc, oh[u], ol[u], make_float2(qa.x, qa.y), make_float2(qa.z, qa.w), make_float2(qb.x, qb.y),
                       make_float2(qb.z, qb.w));
        }
        c = cn;
        if (!more) break;
#pragma unroll
        for (int u = 0; u < U; ++u) { oh[u] = nh[u]; ol[u] = nl[u]; }
    }
    for (; c < n4; c += 32) {
        const float4 qa = v4[2 * c], qb = v4[2 * c + 1];
        df_fma4<W>(acc, __ldcs(rh + c), W ? __ldcs(rl + c) : zero4, make_float2(qa.x, qa.y), make_float2(qa.z, qa.w),
                   make_float2(qb.x, qb.y), make_float2(qb.z, qb.w));
    }
    const double s = warp_sum(df_value(df_add(df_add(acc[0], acc[1]), df_add(acc[2], acc[3]))));
    if (lane == 0) y[r] = s;
}

// ... and the block's partial sums of y over its real rows (r < n) and its
// imaginary rows, in row order, into ypart[2 blockIdx.x + half].
__global__ void __launch_bounds__(kRowWarps * 32) gemv_rows_df_kernel(const float *__restrict__ Oh,
                                                                      const float *__restrict__ Ol,
                                                                      const float2 *__restrict__ v, int64_t rows,
                                                                      int Pp, double *__restrict__ y,
                                                                      double *__restrict__ ypart, const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    const int64_t r0 = (int64_t)blockIdx.x * kRowWarps;
    const int64_t r = r0 + (threadIdx.x >> 5);
    if (r < rows) {
        if (sc[S_WIDE] != 0.0) rows_df<true, 2>(Oh, Ol, v, r, Pp, y);
        else rows_df<false, 2>(Oh, Ol, v, r, Pp, y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t n = rows / 2;
        double h0 = 0.0, h1 = 0.0;
        for (int64_t q = r0; q < r0 + kRowWarps && q < rows; ++q) (q < n ? h0 : h1) += y[q];
        ypart[2 * blockIdx.x] = h0;
        ypart[2 * blockIdx.x + 1] = h1;
    }
}

// zpart[chunk][k] = sum over the chunk's rows r of O[r, k] y[r] from the
// planes, for the four columns k = 4 c4 ... 4 c4 + 3 of one thread (one
// accumulator each, rows in order; the next U rows are loaded before the
// current ones are consumed); W: read the l plane too.
template <bool W, int U>
__device__ __forceinline__ void cols_df(const float *__restrict__ Oh, const float *__restrict__ Ol,
                                        const float2 *__restrict__ y, int64_t rows, int P, int Pp,
                                        int64_t chunk_rows, int c4, double *__restrict__ zpart) {
    const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
    const int64_t r1 = rows < r0 + chunk_rows ? rows : r0 + chunk_rows;
    const int64_t s4 = Pp >> 2;   // row stride in float4
    const float4 *ch = reinterpret_cast<const float4 *>(Oh) + c4;
    const float4 *cl = reinterpret_cast<const float4 *>(Ol) + c4;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = make_float2(0.f, 0.f);
    int64_t r = r0;
    float4 oh[U], ol[U];
    if (r + U - 1 < r1) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            oh[u] = __ldcs(ch + (r + u) * s4);
            ol[u] = W ? __ldcs(cl + (r + u) * s4) : zero4;
        }
    }
    while (r + U - 1 < r1) {
        const int64_t rn = r + U;
        const bool more = rn + U - 1 < r1;
        float4 nh[U], nl[U];
        if (more) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                nh[u] = __ldcs(ch + (rn + u) * s4);
                nl[u] = W ? __ldcs(cl + (rn + u) * s4) : zero4;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float2 q = y[r + u];
            df_fma4<W>(acc, oh[u], ol[u], q, q, q, q);
        }
        r = rn;
        if (!more) break;
#pragma unroll
        for (int u = 0; u < U; ++u) { oh[u] = nh[u]; ol[u] = nl[u]; }
    }
    for (; r < r1; ++r) {
        const float2 q = y[r];
        df_fma4<W>(acc, __ldcs(ch + r * s4), W ? __ldcs(cl + r * s4) : zero4, q, q, q, q);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (4 * c4 + j < P) zpart[(int64_t)blockIdx.y * P + 4 * c4 + j] = df_value(acc[j]);
}

// The column pass's float-plane form with Blackwell's packed float32
// instructions (add / mul / fma .f32x2): the four columns' accumulators as
// two pairs of double-floats (S01, C01), (S23, C23), each lane the same IEEE
// operation as df_fma's, so every sum is bitwise cols_df<false, U>'s with
// half the float32 instructions. a - b is formed as fma(b, -1, a) (one
// rounding of the exact difference, as the subtraction).
__device__ __forceinline__ float2 df_sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void df_fma_pair(float2 &S, float2 &C, float2 h, float2 qh, float2 ql) {
    const float2 p = __fmul2_rn(h, qh);
    float2 e = __ffma2_rn(h, qh, __fmul2_rn(p, make_float2(-1.f, -1.f)));
    e = __ffma2_rn(h, ql, e);
    const float2 sum = __fadd2_rn(S, p);
    const float2 bb = df_sub2(sum, S);
    const float2 t = __fadd2_rn(df_sub2(S, df_sub2(sum, bb)), df_sub2(p, bb));
    const float2 u = __fadd2_rn(t, __fadd2_rn(C, e));
    const float2 hi = __fadd2_rn(sum, u);
    C = df_sub2(u, df_sub2(hi, sum));
    S = hi;
}

template <int U>
__device__ __forceinline__ void cols_df_packed(const float *__restrict__ Oh, const float2 *__restrict__ y,
                                               int64_t rows, int P, int Pp, int64_t chunk_rows, int c4,
                                               double *__restrict__ zpart) {
    const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
    const int64_t r1 = rows < r0 + chunk_rows ? rows : r0 + chunk_rows;
    const int64_t s4 = Pp >> 2;
    const float4 *ch = reinterpret_cast<const float4 *>(Oh) + c4;
    float2 S01 = make_float2(0.f, 0.f), C01 = S01, S23 = S01, C23 = S01;
    int64_t r = r0;
    float4 oh[U];
    if (r + U - 1 < r1) {
#pragma unroll
        for (int u = 0; u < U; ++u) oh[u] = __ldcs(ch + (r + u) * s4);
    }
    while (r + U - 1 < r1) {
        const int64_t rn = r + U;
        const bool more = rn + U - 1 < r1;
        float4 nh[U];
        if (more) {
#pragma unroll
            for (int u = 0; u < U; ++u) nh[u] = __ldcs(ch + (rn + u) * s4);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float2 q = y[r + u];
            const float2 qh = make_float2(q.x, q.x), ql = make_float2(q.y, q.y);
            df_fma_pair(S01, C01, make_float2(oh[u].x, oh[u].y), qh, ql);
            df_fma_pair(S23, C23, make_float2(oh[u].z, oh[u].w), qh, ql);
        }
        r = rn;
        if (!more) break;
#pragma unroll
        for (int u = 0; u < U; ++u) oh[u] = nh[u];
    }
    for (; r < r1; ++r) {
        const float2 q = y[r];
        const float4 o = __ldcs(ch + r * s4);
        df_fma_pair(S01, C01, make_float2(o.x, o.y), make_float2(q.x, q.x), make_float2(q.y, q.y));
        df_fma_pair(S23, C23, make_float2(o.z, o.w), make_float2(q.x, q.x), make_float2(q.y, q.y));
    }
    const float2 a[4] = {make_float2(S01.x, C01.x), make_float2(S01.y, C01.y), make_float2(S23.x, C23.x),
                         make_float2(S23.y, C23.y)};
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (4 * c4 + j < P) zpart[(int64_t)blockIdx.y * P + 4 * c4 + j] = df_value(a[j]);
}

__global__ void __launch_bounds__(kColThreads) gemv_cols_df_kernel(const float *__restrict__ Oh,
                                                                   const float *__restrict__ Ol,
                                                                   const float2 *__restrict__ y, int64_t rows, int P,
                                                                   int Pp, int64_t chunk_rows,
                                                                   double *__restrict__ zpart, const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    const int c4 = blockIdx.x * kColThreads + threadIdx.x;
    if (c4 >= (Pp >> 2)) return;
    if (sc[S_WIDE] != 0.0) cols_df<true, 4>(Oh, Ol, y, rows, P, Pp, chunk_rows, c4, zpart);
    else cols_df_packed<8>(Oh, y, rows, P, Pp, chunk_rows, c4, zpart);
}

// Subtract the mean of each half of y (real rows, imaginary rows).
__global__ void __launch_bounds__(kVecThreads) center_kernel(double *y, int64_t n, double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    double pr = 0.0, pi = 0.0;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) { pr += y[s]; pi += y[n + s]; }
    const double mr = vec_block_sum(pr, sh) / (double)n;
    const double mi = vec_block_sum(pi, sh) / (double)n;
    for (int64_t s = threadIdx.x; s < n; s += blockDim.x) { y[s] -= mr; y[n + s] -= mi; }
}

// zpart[chunk][k] = sum over the chunk's rows r of Ohat[r, k] y[r]
__global__ void __launch_bounds__(kColThreads) gemv_cols_kernel(const double *__restrict__ O, const double *__restrict__ y,
                                                                int64_t rows, int P, int64_t chunk_rows,
                                                                double *__restrict__ zpart, const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    const int k = blockIdx.x * kColThreads + threadIdx.x;
    if (k >= P) return;
    const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
    const int64_t r1 = std::min<int64_t>(rows, r0 + chunk_rows);
    const double *col = O + k;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t r = r0;
    for (; r + 3 < r1; r += 4) {
        a0 = fma(col[r * P], y[r], a0);
        a1 = fma(col[(r + 1) * P], y[r + 1], a1);
        a2 = fma(col[(r + 2) * P], y[r + 2], a2);
        a3 = fma(col[(r + 3) * P], y[r + 3], a3);
    }
    for (; r < r1; ++r) a0 = fma(col[r * P], y[r], a0);
    zpart[(int64_t)blockIdx.y * P + k] = (a0 + a1) + (a2 + a3);
}

// Fixed-order sum of one double per thread over a kPvThreads block (result in every thread).
__device__ double pv_block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double w = 0.0;
    if (warp == 0) {
        w = warp_sum(lane < kPvThreads / 32 ? sh[lane] : 0.0);
        if (lane == 0) sh[32] = w;
    }
    __syncthreads();
    w = sh[32];
    __syncthreads();
    return w;
}

// Sum of the nb block partials part[0 .. nb), in a fixed order (every thread).
__device__ double pv_partials(const double *part, int nb, double *sh) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
    return pv_block_sum(v, sh);
}

// y minus the mean of each half (the means from the row pass's nb block
// partials, summed in a fixed order by every block), and the result as
// double-floats into yf; one element per thread.
__global__ void __launch_bounds__(kPvThreads) center_df_kernel(double *y, int64_t n, const double *ypart, int nb,
                                                                float2 *yf, const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    double pr = 0.0, pi = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) { pr += ypart[2 * b]; pi += ypart[2 * b + 1]; }
    const double mr = pv_block_sum(pr, sh) / (double)n;
    const double mi = pv_block_sum(pi, sh) / (double)n;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 2 * n) {
        const double a = y[q] - (q < n ? mr : mi);
        y[q] = a;
        yf[q] = df_of(a);
    }
}

// CG step, part 1: Ap = sum_chunks zpart / n + eps p; block partials of p . Ap.
__global__ void __launch_bounds__(kPvThreads) cg_ap_kernel(const double *zpart, int nchunks, int P, int64_t n,
                                                            double eps, const double *p, double *Ap, double *part,
                                                            const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    double pap = 0.0;
    if (k < P) {
        double z = 0.0;
        for (int c = 0; c < nchunks; ++c) z += zpart[(int64_t)c * P + k];
        double a = z / (double)n + eps * p[k];
        // an S.x product out of range (the double-float passes overflow past the float range, about 3.4e38) must
        // not pass as a step: Inf becomes NaN, which reaches alpha, the residual and the non-finite status
        if (!isfinite(a)) a = __longlong_as_double(0x7ff8000000000000LL);
        Ap[k] = a;
        pap = p[k] * a;
    }
    pap = pv_block_sum(pap, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = pap;
}

// Part 2: alpha = rs / (p . Ap); x += alpha p; r -= alpha Ap; block partials of r . r.
__global__ void __launch_bounds__(kPvThreads) cg_xr_kernel(int P, const double *p, const double *Ap, double *x,
                                                            double *r, const double *part, double *part2,
                                                            const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    const double alpha = sc[S_RS] / pv_partials(part, gridDim.x, sh);
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    double rn = 0.0;
    if (k < P) {
        x[k] = fma(alpha, p[k], x[k]);
        const double rk = fma(-alpha, Ap[k], r[k]);
        r[k] = rk;
        rn = rk * rk;
    }
    rn = pv_block_sum(rn, sh);
    if (threadIdx.x == 0) part2[blockIdx.x] = rn;
}

// Part 3: beta = (r . r) / rs; p = r + beta p (also as double-floats into pf, if not null).
__global__ void __launch_bounds__(kPvThreads) cg_dir_kernel(int P, const double *r, double *p, const double *part2,
                                                             const double *sc, float2 *pf) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    const double beta = pv_partials(part2, gridDim.x, sh) / sc[S_RS];
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    if (k < P) {
        const double v = fma(beta, p[k], r[k]);
        p[k] = v;
        if (pf) pf[k] = df_of(v);
    }
}

// Part 4 (one block): iteration count, rs = r . r, convergence.
__global__ void __launch_bounds__(kPvThreads) cg_scalars_kernel(int nb, double rtol, int max_iter,
                                                                 const double *part2, double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    const double rn = pv_partials(part2, nb, sh);
    if (threadIdx.x == 0) {
        const double it = sc[S_ITER] + 1.0;
        sc[S_ITER] = it;
        sc[S_RS] = rn;
        if (sqrt(rn) <= rtol * sc[S_FNORM] || it >= (double)max_iter || !isfinite(rn)) sc[S_DONE] = 1.0;
    }
}

// CG start: F = sum_chunks zpart / n; x = 0; r = p = F; block partials of |F|^2.
// pf (nullable) receives p as double-floats.
__global__ void __launch_bounds__(kPvThreads) cg_init_kernel(const double *zpart, int nchunks, int P, int64_t n,
                                                              double *x, double *r, double *p, double *part,
                                                              float2 *pf) {
    __shared__ double sh[33];
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    double acc = 0.0;
    if (k < P) {
        double f = 0.0;
        for (int c = 0; c < nchunks; ++c) f += zpart[(int64_t)c * P + k];
        f /= (double)n;
        x[k] = 0.0;
        r[k] = f;
        p[k] = f;
        if (pf) pf[k] = df_of(f);
        acc = f * f;
    } else if (pf && k < ((P + 3) & ~3)) {
        pf[k] = make_float2(0.f, 0.f);   // the pad the vectorised row pass reads up to the plane stride
    }
    acc = pv_block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// CG start (one block): rs = |F|^2, |F|, nothing to do if F = 0.
__global__ void __launch_bounds__(kPvThreads) cg_init_scalars_kernel(int nb, const double *part, double *sc) {
    __shared__ double sh[33];
    const double rs = pv_partials(part, nb, sh);
    if (threadIdx.x == 0) {
        sc[S_RS] = rs;
        sc[S_FNORM] = sqrt(rs);
        sc[S_DONE] = (rs == 0.0) ? 1.0 : 0.0;
    }
}

// ---------------------------------------------------------------- sample-space (Woodbury) form
constexpr int kWb = 64;          // tile edge of the Gram matrix, Cholesky block size
constexpr int kWbK = 16;         // K chunk staged in shared memory by the tile kernel
constexpr int kWbThreads = 256;  // 16 x 16 threads, 4 x 4 outputs each

// Lower-triangular tile number t -> (row tile, column tile), column <= row.
__device__ __forceinline__ void tri_tile(int64_t t, int *bi, int *bj) {
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
    while ((int64_t)i * (i + 1) / 2 > t) --i;
    *bi = i;
    *bj = (int)(t - (int64_t)i * (i + 1) / 2);
}

// kGram: A[i, j] = sum_k Oc[i, k] Oc[j, k] / n + eps [i == j] over k < P, for
//   the lower tiles, Oc = O minus the column mean of its half (rows < n: real
//   parts, rows >= n: imaginary parts).
// !kGram (trailing update of Cholesky step kb): A[i, j] -= sum_k L[i, k] L[j, k]
//   over the 64 columns of block kb, for the lower tiles right of and below
//   block kb.
template <bool kGram>
__global__ void __launch_bounds__(kWbThreads) wb_tile_kernel(const double *__restrict__ X, int64_t ldx, int64_t K,
                                                             const double *__restrict__ mu, int64_t n, double eps,
                                                             double *A, int64_t m, int kb) {
    __shared__ double sa[kWbK][kWb + 1];
    __shared__ double sb[kWbK][kWb + 1];
    int bi, bj;
    tri_tile(blockIdx.x, &bi, &bj);
    if (!kGram) { bi += kb + 1; bj += kb + 1; }
    const int64_t i0 = (int64_t)bi * kWb, j0 = (int64_t)bj * kWb;
    const int64_t k_begin = kGram ? 0 : (int64_t)kb * kWb;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += kWbK) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = threadIdx.x + e * kWbThreads;   // 0 .. 1023
            const int r = idx >> 4, c = idx & 15;
            const int64_t k = k0 + c;
            double va = 0.0, vb = 0.0;
            if (k < K) {
                const int64_t ri = i0 + r, rj = j0 + r;
                if (ri < m) {
                    va = X[ri * ldx + k_begin + k];
                    if (kGram) va -= mu[(ri >= n ? K : 0) + k];
                }
                if (rj < m) {
                    vb = X[rj * ldx + k_begin + k];
                    if (kGram) vb -= mu[(rj >= n ? K : 0) + k];
                }
            }
            sa[c][r] = va;
            sb[c][r] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kWbK; ++c) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sa[c][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sb[c][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + ty + 16 * a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx + 16 * b;
            if (j >= m || j > i) continue;
            if (kGram) A[i * m + j] = acc[a][b] / (double)n + (i == j ? eps : 0.0);
            else A[i * m + j] -= acc[a][b];
        }
    }
}

// Cholesky of the diagonal block kb (already updated by the earlier steps), in
// shared memory, column by column. A pivot that is not positive becomes NaN,
// which reaches delta and is reported as a non-finite result.
__global__ void __launch_bounds__(kWbThreads) wb_potrf_kernel(double *A, int64_t m, int kb) {
    __shared__ double s[kWb][kWb + 1];
    const int64_t o = (int64_t)kb * kWb;
    const int nb = (int)std::min<int64_t>(kWb, m - o);
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int i = idx / nb, j = idx % nb;
        s[i][j] = j <= i ? A[(o + i) * m + o + j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = s[j][j];
            s[j][j] = d > 0.0 ? sqrt(d) : __longlong_as_double(0x7ff8000000000000LL);
        }
        __syncthreads();
        const double piv = s[j][j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) s[i][j] /= piv;
        __syncthreads();
        const int w = nb - j - 1;
        for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
            const int i = j + 1 + idx / w, k = j + 1 + idx % w;
            if (k <= i) s[i][k] = fma(-s[i][j], s[k][j], s[i][k]);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int i = idx / nb, j = idx % nb;
        if (j <= i) A[(o + i) * m + o + j] = s[i][j];
    }
}

// Panel below the diagonal block kb: L[i, block kb] = A[i, block kb] L_kk^-T,
// one thread per row (forward substitution along the row).
__global__ void __launch_bounds__(kWb) wb_trsm_kernel(double *A, int64_t m, int kb) {
    __shared__ double row[kWb][kWb + 1];
    const int64_t o = (int64_t)kb * kWb;
    const int64_t i = o + (int64_t)(blockIdx.x + 1) * kWb + threadIdx.x;
    const double *Lkk = A + o * m + o;
    if (i < m) {
        double *ai = A + i * m + o;
        for (int j = 0; j < kWb; ++j) {
            double v = ai[j];
            for (int l = 0; l < j; ++l) v = fma(-row[threadIdx.x][l], __ldg(Lkk + (int64_t)j * m + l), v);
            v /= __ldg(Lkk + (int64_t)j * m + j);
            row[threadIdx.x][j] = v;
        }
        for (int j = 0; j < kWb; ++j) ai[j] = row[threadIdx.x][j];
    }
}

// Forward substitution L z = b, block kb: solve the diagonal block in place.
__global__ void __launch_bounds__(kWb) wb_fwd_diag_kernel(const double *A, int64_t m, int kb, double *b) {
    __shared__ double z[kWb];
    const int64_t o = (int64_t)kb * kWb;
    const int nb = (int)std::min<int64_t>(kWb, m - o);
    const int t = threadIdx.x;
    if (t < nb) z[t] = b[o + t];
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (t == j) z[j] /= A[(o + j) * m + o + j];
        __syncthreads();
        if (t > j && t < nb) z[t] = fma(-A[(o + t) * m + o + j], z[j], z[t]);
        __syncthreads();
    }
    if (t < nb) b[o + t] = z[t];
}

// ... then b[i] -= L[i, block kb] . z[block kb] for the rows below (one warp per row).
__global__ void __launch_bounds__(kRowWarps * 32) wb_fwd_update_kernel(const double *A, int64_t m, int kb, double *b) {
    const int64_t o = (int64_t)kb * kWb;
    const int64_t i = o + kWb + (int64_t)blockIdx.x * kRowWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= m) return;
    const double *li = A + i * m + o;
    double v = fma(li[lane], b[o + lane], li[lane + 32] * b[o + lane + 32]);
    v = warp_sum(v);
    if (lane == 0) b[i] -= v;
}

// Back substitution L^T y = z, block kb: solve the diagonal block in place.
__global__ void __launch_bounds__(kWb) wb_bwd_diag_kernel(const double *A, int64_t m, int kb, double *b) {
    __shared__ double y[kWb];
    const int64_t o = (int64_t)kb * kWb;
    const int nb = (int)std::min<int64_t>(kWb, m - o);
    const int t = threadIdx.x;
    if (t < nb) y[t] = b[o + t];
    __syncthreads();
    for (int j = nb - 1; j >= 0; --j) {
        if (t == j) y[j] /= A[(o + j) * m + o + j];
        __syncthreads();
        if (t < j) y[t] = fma(-A[(o + j) * m + o + t], y[j], y[t]);
        __syncthreads();
    }
    if (t < nb) b[o + t] = y[t];
}

// ... then b[i] -= sum_l L[o + l, i] y[o + l] for the rows above (one thread per row).
__global__ void __launch_bounds__(256) wb_bwd_update_kernel(const double *A, int64_t m, int kb, double *b) {
    const int64_t o = (int64_t)kb * kWb;
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= o) return;
    const int nb = (int)std::min<int64_t>(kWb, m - o);
    double v = 0.0;
    for (int l = 0; l < nb; ++l) v = fma(A[(o + l) * m + i], b[o + l], v);
    b[i] -= v;
}

// b = v / n (the right-hand side Ehat / n), and the all-(1/n) vector used for the column means.
__global__ void wb_rhs_kernel(const double *v, int64_t m, int64_t n, double *b, double *ones) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        b[i] = v[i] / (double)n;
        ones[i] = 1.0 / (double)n;
    }
}

// Refinement right-hand side: r = Ehat / n - (Oc Oc^T y / n + eps y), with t = Oc Oc^T y.
__global__ void wb_refine_rhs_kernel(const double *ehat, const double *t, const double *y, int64_t m, int64_t n,
                                     double eps, double *r) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = ehat[i] / (double)n - fma(eps, y[i], t[i] / (double)n);
}

// y += dy, and yc = y (to be centred).
__global__ void wb_add_copy_kernel(double *y, const double *dy, int64_t m, double *yc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = dy ? y[i] + dy[i] : y[i];
        y[i] = v;
        yc[i] = v;
    }
}

// out[k] = sum over chunks of zpart[c][k] (fixed order).
__global__ void wb_chunk_sum_kernel(const double *zpart, int nchunks, int P, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    double z = 0.0;
    for (int c = 0; c < nchunks; ++c) z += zpart[(int64_t)c * P + k];
    out[k] = z;
}

// Block partials of |Ap - F|^2, then the one-block total into sc[S_WBRES].
__global__ void __launch_bounds__(kPvThreads) wb_resid_kernel(int P, const double *Ap, const double *F, double *part) {
    __shared__ double sh[33];
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    double d = 0.0;
    if (k < P) { d = Ap[k] - F[k]; d *= d; }
    d = pv_block_sum(d, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = d;
}

__global__ void __launch_bounds__(kPvThreads) wb_resid_total_kernel(int nb, const double *part, double *sc) {
    __shared__ double sh[33];
    const double v = pv_partials(part, nb, sh);
    if (threadIdx.x == 0) sc[S_WBRES] = v;
}

__global__ void update_kernel(double *params, const double *x, int P, double lr) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) params[k] -= lr * x[k];
}

// Row chunks of a column pass with col_blocks blocks across the columns: about
// eight blocks per SM, at least 64 rows a chunk, at most 256 chunks.
int chunks_for_blocks(int64_t rows, int col_blocks, int num_sms) {
    int64_t want = std::max<int64_t>(1, (int64_t)num_sms * 8 / col_blocks);
    want = std::min<int64_t>(want, std::max<int64_t>(1, rows / 64));
    return (int)std::min<int64_t>(want, 256);
}

int chunks_for(int64_t rows, int P, int num_sms) {
    return chunks_for_blocks(rows, (P + kColThreads - 1) / kColThreads, num_sms);
}

}  // namespace

size_t sr_workspace_doubles(int64_t n, int P, int sx_fp64) {
    // y [2n], Ap, r, p [P], zpart [256][P] upper bound, scalars, two block-partial arrays, then the double-float
    // copies of p [Pp] and y [2n] and O's two float planes [2n][Pp] (Pp = P rounded up to a multiple of 4; one
    // double's room per double-float) from a 16-byte boundary, the row pass's partial sums [2 ceil(2n / 8)]
    // (the float64 passes need none of the double-float part)
    const size_t Pp = (size_t)((P + 3) & ~3);
    const size_t base = 2 * (size_t)n + 3 * (size_t)P + 256 * (size_t)P + S_COUNT +
                        2 * (size_t)((P + kPvThreads - 1) / kPvThreads);
    if (sx_fp64) return base;
    return base + 1 + Pp + 2 * (size_t)n + 2 * (size_t)n * Pp + 2 * (size_t)((2 * n + kRowWarps - 1) / kRowWarps);
}

int run_sr_solve(const Problem &pr, const double *O, const double *eloc, int64_t n, double eps, double rtol,
                 int max_iter, double lr, double *delta, double *params, int apply, double *ws, int *iters_out,
                 double *resid_out, double *energy_out, int sx_fp64, const LaunchEnv &env) {
    const int P = pr.P;
    const int64_t rows = 2 * n;
    const int nchunks = chunks_for(rows, P, env.num_sms);
    const int64_t chunk_rows = (rows + nchunks - 1) / nchunks;
    double *y = ws;
    double *Ap = y + 2 * n;
    double *r = Ap + P;
    double *p = r + P;
    double *zpart = p + P;
    double *sc = zpart + (size_t)256 * P;
    const int pvb = (P + kPvThreads - 1) / kPvThreads;
    double *part = sc + S_COUNT;
    double *part2 = part + pvb;
    // double-float copies of p [Pp] and y [2n], then O as planes of h and of l [2n][Pp] each (written by the
    // force pass), from a 16-byte boundary for the float4 loads
    const int Pp = (P + 3) & ~3;
    float2 *pf = reinterpret_cast<float2 *>((reinterpret_cast<uintptr_t>(part2 + pvb) + 15) & ~(uintptr_t)15);
    float2 *yf = pf + Pp;
    float *Oh = reinterpret_cast<float *>(yf + 2 * n);
    float *Ol = Oh + (size_t)rows * Pp;
    double *ypart = reinterpret_cast<double *>(Ol + (size_t)rows * Pp);   // [rgrid][2]
    cudaStream_t s = env.stream;
    const dim3 cgrid((P + kColThreads - 1) / kColThreads, nchunks);
    const int rgrid = (int)((rows + kRowWarps - 1) / kRowWarps);
    const int cgb = (int)((rows + kPvThreads - 1) / kPvThreads);
    // the double-float column pass: four columns a thread
    const int dcb = (Pp / 4 + kColThreads - 1) / kColThreads;
    const int nch_df = chunks_for_blocks(rows, dcb, env.num_sms);
    const int64_t chunk_df = (rows + nch_df - 1) / nch_df;
    const dim3 dgrid(dcb, nch_df);

    energy_kernel<<<1, kVecThreads, 0, s>>>(eloc, n, y, sc);
    if (sx_fp64) gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
    else {
        gemv_cols_split_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, Pp, chunk_rows, zpart, Oh, sc);
        split_low_kernel<<<dim3((Pp + kColThreads - 1) / kColThreads, (unsigned)std::min<int64_t>(rows, 1024)),
                           kColThreads, 0, s>>>(O, rows, P, Pp, Ol, sc);
    }
    cg_init_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, nchunks, P, n, delta, r, p, part, sx_fp64 ? nullptr : pf);
    cg_init_scalars_kernel<<<1, kPvThreads, 0, s>>>(pvb, part, sc);
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR setup launch failed"; return NQS_ERR_CUDA; }
    *env.launches += sx_fp64 ? 4 : 5;

    double host_sc[S_COUNT];
    int done_iters = 0;
    // iterations launched between host checks: the caller's hint (*iters_out on entry: the previous solve's
    // count) plus two, so a solve like the last one needs one check; then doubling. Launches past convergence
    // return at once (device flag), so the hint changes no result.
    int batch = iters_out && *iters_out > 0 ? std::min(std::max(*iters_out + 2, 4), 64) : 4;
    while (max_iter > 0) {
        for (int b = 0; b < batch; ++b) {
            if (sx_fp64) {
                gemv_rows_kernel<<<rgrid, kRowWarps * 32, 0, s>>>(O, p, rows, P, y, sc);
                center_kernel<<<1, kVecThreads, 0, s>>>(y, n, sc);
                gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
            } else {
                gemv_rows_df_kernel<<<rgrid, kRowWarps * 32, 0, s>>>(Oh, Ol, pf, rows, Pp, y, ypart, sc);
                center_df_kernel<<<cgb, kPvThreads, 0, s>>>(y, n, ypart, rgrid, yf, sc);
                gemv_cols_df_kernel<<<dgrid, kColThreads, 0, s>>>(Oh, Ol, yf, rows, P, Pp, chunk_df, zpart, sc);
            }
            cg_ap_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, sx_fp64 ? nchunks : nch_df, P, n, eps, p, Ap, part, sc);
            cg_xr_kernel<<<pvb, kPvThreads, 0, s>>>(P, p, Ap, delta, r, part, part2, sc);
            cg_dir_kernel<<<pvb, kPvThreads, 0, s>>>(P, r, p, part2, sc, sx_fp64 ? nullptr : pf);
            cg_scalars_kernel<<<1, kPvThreads, 0, s>>>(pvb, rtol, max_iter, part2, sc);
        }
        done_iters += batch;
        *env.launches += 7 * batch;
        cudaError_t e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { *env.msg = std::string("SR loop: ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
        if (host_sc[S_DONE] != 0.0 || done_iters >= max_iter + batch) break;
        batch = std::min(batch * 2, 64);
    }
    if (max_iter <= 0) {
        cudaError_t e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { *env.msg = std::string("SR: ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
    }
    const int iters = (int)host_sc[S_ITER];
    const double fnorm = host_sc[S_FNORM];
    const double resid = fnorm > 0.0 ? std::sqrt(host_sc[S_RS]) / fnorm : 0.0;
    if (iters_out) *iters_out = iters;
    if (resid_out) *resid_out = resid;
    if (energy_out) { energy_out[0] = host_sc[S_ERE]; energy_out[1] = host_sc[S_EIM]; }
    // a non-finite force, residual or energy (a NaN or Inf in O or E_loc) means delta is not a step: the
    // parameters are left as they are
    if (!std::isfinite(fnorm) || !std::isfinite(resid) || !std::isfinite(host_sc[S_ERE])) {
        *env.msg = "SR: non-finite force, residual or energy (parameters not updated)";
        return NQS_ERR_NONFINITE;
    }
    if (apply) {
        update_kernel<<<(P + 255) / 256, 256, 0, s>>>(params, delta, P, lr);
        ++*env.launches;
    }
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR update launch failed"; return NQS_ERR_CUDA; }
    if (fnorm > 0.0 && resid > rtol) {
        *env.msg = "SR: conjugate gradient reached max_iter before the tolerance";
        return NQS_ERR_NOT_CONVERGED;
    }
    return NQS_OK;
}

size_t sr_woodbury_workspace_doubles(int64_t n, int P) {
    // A [2n x 2n], column means [2P], ehat, b, t, yc, r [2n], zpart [256][P], F, Ap, two scratch
    // P-vectors, scalars, two block-partial arrays
    const size_t m = 2 * (size_t)n;
    return m * m + 2 * (size_t)P + 5 * m + 256 * (size_t)P + 4 * (size_t)P + S_COUNT +
           2 * (size_t)((P + kPvThreads - 1) / kPvThreads);
}

int run_sr_woodbury(const Problem &pr, const double *O, const double *eloc, int64_t n, double eps, double lr,
                    int refine_steps, double *delta, double *params, int apply, double *ws, double *resid_out,
                    double *energy_out, const LaunchEnv &env) {
    const int P = pr.P;
    const int64_t m = 2 * n;
    const int T = (int)((m + kWb - 1) / kWb);
    double *A = ws;
    double *mu = A + (size_t)m * m;
    double *ehat = mu + 2 * (size_t)P;
    double *b = ehat + m;
    double *t = b + m;
    double *yc = t + m;
    double *r = yc + m;
    double *zpart = r + m;
    double *F = zpart + (size_t)256 * P;
    double *Ap = F + P;
    double *tmp1 = Ap + P;
    double *tmp2 = tmp1 + P;
    double *sc = tmp2 + P;
    const int pvb = (P + kPvThreads - 1) / kPvThreads;
    double *part = sc + S_COUNT;
    double *part2 = part + pvb;
    cudaStream_t s = env.stream;
    int64_t launches = 0;
    const int nch_half = chunks_for(n, P, env.num_sms);
    const int64_t chunk_half = (n + nch_half - 1) / nch_half;
    const int nch = chunks_for(m, P, env.num_sms);
    const int64_t chunk_rows = (m + nch - 1) / nch;
    const int colb = (P + kColThreads - 1) / kColThreads;
    const int sumb = (P + 255) / 256;
    const int vecb = (int)std::min<int64_t>((m + 255) / 256, 4096);

    // <E>, Ehat; b = Ehat / n; column means of each half of O
    energy_kernel<<<1, kVecThreads, 0, s>>>(eloc, n, ehat, sc);
    wb_rhs_kernel<<<vecb, 256, 0, s>>>(ehat, m, n, b, t);
    gemv_cols_kernel<<<dim3(colb, nch_half), kColThreads, 0, s>>>(O, t, n, P, chunk_half, zpart, sc);
    wb_chunk_sum_kernel<<<sumb, 256, 0, s>>>(zpart, nch_half, P, mu);
    gemv_cols_kernel<<<dim3(colb, nch_half), kColThreads, 0, s>>>(O + (size_t)n * P, t, n, P, chunk_half, zpart, sc);
    wb_chunk_sum_kernel<<<sumb, 256, 0, s>>>(zpart, nch_half, P, mu + P);
    launches += 6;
    // A = Ohat Ohat^T / n + eps I (lower tiles)
    const int64_t tiles = (int64_t)T * (T + 1) / 2;
    wb_tile_kernel<true><<<(unsigned)tiles, kWbThreads, 0, s>>>(O, P, P, mu, n, eps, A, m, 0);
    ++launches;
    // A = L L^T, blocked right-looking
    for (int kb = 0; kb < T; ++kb) {
        wb_potrf_kernel<<<1, kWbThreads, 0, s>>>(A, m, kb);
        ++launches;
        const int below = T - kb - 1;
        if (below > 0) {
            wb_trsm_kernel<<<below, kWb, 0, s>>>(A, m, kb);
            const int64_t ut = (int64_t)below * (below + 1) / 2;
            wb_tile_kernel<false><<<(unsigned)ut, kWbThreads, 0, s>>>(A, m, kWb, nullptr, n, 0.0, A, m, kb);
            launches += 2;
        }
    }
    // L z = v, then L^T y = z (in place)
    auto chol_solve = [&](double *v) {
        for (int kb = 0; kb < T; ++kb) {
            wb_fwd_diag_kernel<<<1, kWb, 0, s>>>(A, m, kb, v);
            ++launches;
            const int64_t rows_below = m - (int64_t)(kb + 1) * kWb;
            if (rows_below > 0) {
                wb_fwd_update_kernel<<<(unsigned)((rows_below + kRowWarps - 1) / kRowWarps), kRowWarps * 32, 0,
                                       s>>>(A, m, kb, v);
                ++launches;
            }
        }
        for (int kb = T - 1; kb >= 0; --kb) {
            wb_bwd_diag_kernel<<<1, kWb, 0, s>>>(A, m, kb, v);
            ++launches;
            if (kb > 0) {
                wb_bwd_update_kernel<<<(unsigned)(((int64_t)kb * kWb + 255) / 256), 256, 0, s>>>(A, m, kb, v);
                ++launches;
            }
        }
    };
    // delta = Ohat^T y = O^T (y minus its half means); dy (nullable) is added to y first
    auto delta_of = [&](const double *dy) {
        wb_add_copy_kernel<<<vecb, 256, 0, s>>>(b, dy, m, yc);
        center_kernel<<<1, kVecThreads, 0, s>>>(yc, n, sc);
        gemv_cols_kernel<<<dim3(colb, nch), kColThreads, 0, s>>>(O, yc, m, P, chunk_rows, zpart, sc);
        wb_chunk_sum_kernel<<<sumb, 256, 0, s>>>(zpart, nch, P, delta);
        launches += 4;
    };
    chol_solve(b);
    delta_of(nullptr);
    // iterative refinement in the sample space: r = Ehat / n - A y with A y = Oc delta / n + eps y
    // (evaluated from O, not from the factor), then y += A^-1 r
    for (int it = 0; it < refine_steps; ++it) {
        gemv_rows_kernel<<<(unsigned)((m + kRowWarps - 1) / kRowWarps), kRowWarps * 32, 0, s>>>(O, delta, m, P, t,
                                                                                                sc);
        center_kernel<<<1, kVecThreads, 0, s>>>(t, n, sc);
        wb_refine_rhs_kernel<<<vecb, 256, 0, s>>>(ehat, t, b, m, n, eps, r);
        launches += 3;
        chol_solve(r);
        delta_of(r);
    }
    // residual of the parameter-space system: |(S + eps I) delta - F| / |F|
    gemv_cols_kernel<<<dim3(colb, nch), kColThreads, 0, s>>>(O, ehat, m, P, chunk_rows, zpart, sc);
    cg_init_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, nch, P, n, tmp1, F, tmp2, part, nullptr);
    cg_init_scalars_kernel<<<1, kPvThreads, 0, s>>>(pvb, part, sc);
    // (S_DONE is set when F = 0; delta is then 0 and the kernels below skip)
    gemv_rows_kernel<<<(unsigned)((m + kRowWarps - 1) / kRowWarps), kRowWarps * 32, 0, s>>>(O, delta, m, P, t, sc);
    center_kernel<<<1, kVecThreads, 0, s>>>(t, n, sc);
    gemv_cols_kernel<<<dim3(colb, nch), kColThreads, 0, s>>>(O, t, m, P, chunk_rows, zpart, sc);
    cg_ap_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, nch, P, n, eps, delta, Ap, part2, sc);
    wb_resid_kernel<<<pvb, kPvThreads, 0, s>>>(P, Ap, F, part);
    wb_resid_total_kernel<<<1, kPvThreads, 0, s>>>(pvb, part, sc);
    launches += 9;
    *env.launches += launches;
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR (sample-space) launch failed"; return NQS_ERR_CUDA; }
    double host_sc[S_COUNT];
    cudaError_t e = cudaMemcpyAsync(host_sc, sc, sizeof(host_sc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { *env.msg = std::string("SR (sample-space): ") + cudaGetErrorString(e); return NQS_ERR_CUDA; }
    const double fnorm = host_sc[S_FNORM];
    const double resid = fnorm > 0.0 ? std::sqrt(host_sc[S_WBRES]) / fnorm : 0.0;
    if (resid_out) *resid_out = resid;
    if (energy_out) { energy_out[0] = host_sc[S_ERE]; energy_out[1] = host_sc[S_EIM]; }
    if (!std::isfinite(resid) || !std::isfinite(host_sc[S_ERE])) {
        *env.msg = "SR (sample-space): non-finite result (a Cholesky pivot was not positive)";
        return NQS_ERR_NONFINITE;
    }
    if (apply) {
        update_kernel<<<(P + 255) / 256, 256, 0, s>>>(params, delta, P, lr);
        ++*env.launches;
        if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR update launch failed"; return NQS_ERR_CUDA; }
    }
    return NQS_OK;
}

}  // namespace nqs
