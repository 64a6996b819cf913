// Stochastic reconfiguration solve in float64 (Sec. 3.2; Sec. 5.4.1
// "Distributed SR computation"). The paper builds the covariance matrix
// S explicitly and factorises it; here S is never formed:
//   (S + eps I) x = Ohat^T (Ohat x - mean) / n + eps x
// with Ohat the real-stacked [2n, P] matrix of local derivatives, and the
// system is solved by conjugate gradient. Every reduction runs in a fixed
// order, so results do not depend on what else runs on the GPU.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace nqs {

namespace {

// scalar slots in the workspace
enum : int { S_ERE = 0, S_EIM, S_RS, S_FNORM, S_DONE, S_ITER, S_MEANRE, S_MEANIM, S_COUNT = 16 };
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
        const double a = z / (double)n + eps * p[k];
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

// Part 3: beta = (r . r) / rs; p = r + beta p.
__global__ void __launch_bounds__(kPvThreads) cg_dir_kernel(int P, const double *r, double *p, const double *part2,
                                                             const double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    const double beta = pv_partials(part2, gridDim.x, sh) / sc[S_RS];
    const int k = blockIdx.x * kPvThreads + threadIdx.x;
    if (k < P) p[k] = fma(beta, p[k], r[k]);
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
__global__ void __launch_bounds__(kPvThreads) cg_init_kernel(const double *zpart, int nchunks, int P, int64_t n,
                                                              double *x, double *r, double *p, double *part) {
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
        acc = f * f;
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

__global__ void update_kernel(double *params, const double *x, int P, double lr) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) params[k] -= lr * x[k];
}

int chunks_for(int64_t rows, int P, int num_sms) {
    const int col_blocks = (P + kColThreads - 1) / kColThreads;
    int64_t want = std::max<int64_t>(1, (int64_t)num_sms * 8 / col_blocks);
    want = std::min<int64_t>(want, std::max<int64_t>(1, rows / 64));
    return (int)std::min<int64_t>(want, 256);
}

}  // namespace

size_t sr_workspace_doubles(int64_t n, int P) {
    // y [2n], Ap, r, p [P], zpart [256][P] upper bound, scalars, two block-partial arrays
    return 2 * (size_t)n + 3 * (size_t)P + 256 * (size_t)P + S_COUNT + 2 * (size_t)((P + kPvThreads - 1) / kPvThreads);
}

int run_sr_solve(const Problem &pr, const double *O, const double *eloc, int64_t n, double eps, double rtol,
                 int max_iter, double lr, double *delta, double *params, int apply, double *ws, int *iters_out,
                 double *resid_out, double *energy_out, const LaunchEnv &env) {
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
    cudaStream_t s = env.stream;
    const dim3 cgrid((P + kColThreads - 1) / kColThreads, nchunks);
    const int rgrid = (int)((rows + kRowWarps - 1) / kRowWarps);

    energy_kernel<<<1, kVecThreads, 0, s>>>(eloc, n, y, sc);
    gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
    cg_init_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, nchunks, P, n, delta, r, p, part);
    cg_init_scalars_kernel<<<1, kPvThreads, 0, s>>>(pvb, part, sc);
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR setup launch failed"; return NQS_ERR_CUDA; }
    *env.launches += 4;

    double host_sc[S_COUNT];
    int done_iters = 0;
    int batch = 4;
    while (max_iter > 0) {
        for (int b = 0; b < batch; ++b) {
            gemv_rows_kernel<<<rgrid, kRowWarps * 32, 0, s>>>(O, p, rows, P, y, sc);
            center_kernel<<<1, kVecThreads, 0, s>>>(y, n, sc);
            gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
            cg_ap_kernel<<<pvb, kPvThreads, 0, s>>>(zpart, nchunks, P, n, eps, p, Ap, part, sc);
            cg_xr_kernel<<<pvb, kPvThreads, 0, s>>>(P, p, Ap, delta, r, part, part2, sc);
            cg_dir_kernel<<<pvb, kPvThreads, 0, s>>>(P, r, p, part2, sc);
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
    if (apply) {
        update_kernel<<<(P + 255) / 256, 256, 0, s>>>(params, delta, P, lr);
        ++*env.launches;
    }
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR update launch failed"; return NQS_ERR_CUDA; }
    if (!std::isfinite(resid) || !std::isfinite(host_sc[S_ERE])) {
        *env.msg = "SR: non-finite residual or energy";
        return NQS_ERR_NONFINITE;
    }
    if (fnorm > 0.0 && resid > rtol) {
        *env.msg = "SR: conjugate gradient reached max_iter before the tolerance";
        return NQS_ERR_NOT_CONVERGED;
    }
    return NQS_OK;
}

}  // namespace nqs
