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

// F = sum_chunks zpart / n; x = 0; r = p = F; rs = |r|^2.
__global__ void __launch_bounds__(kVecThreads) cg_init_kernel(const double *zpart, int nchunks, int P, int64_t n,
                                                              double *x, double *r, double *p, double rtol, double *sc) {
    __shared__ double sh[33];
    double acc = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double f = 0.0;
        for (int c = 0; c < nchunks; ++c) f += zpart[(int64_t)c * P + k];
        f /= (double)n;
        x[k] = 0.0;
        r[k] = f;
        p[k] = f;
        acc = fma(f, f, acc);
    }
    const double rs = vec_block_sum(acc, sh);
    if (threadIdx.x == 0) {
        sc[S_RS] = rs;
        sc[S_FNORM] = sqrt(rs);
        sc[S_DONE] = (rs == 0.0) ? 1.0 : 0.0;
    }
}

// One CG update given z = Ohat^T y_c in zpart.
__global__ void __launch_bounds__(kVecThreads) cg_step_kernel(const double *zpart, int nchunks, int P, int64_t n,
                                                              double eps, double rtol, int max_iter, double *x,
                                                              double *r, double *p, double *Ap, double *sc) {
    if (sc[S_DONE] != 0.0) return;
    __shared__ double sh[33];
    double pap = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double z = 0.0;
        for (int c = 0; c < nchunks; ++c) z += zpart[(int64_t)c * P + k];
        const double a = z / (double)n + eps * p[k];
        Ap[k] = a;
        pap = fma(p[k], a, pap);
    }
    pap = vec_block_sum(pap, sh);
    const double rs = sc[S_RS];
    const double alpha = rs / pap;
    double rn = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        x[k] = fma(alpha, p[k], x[k]);
        const double rk = fma(-alpha, Ap[k], r[k]);
        r[k] = rk;
        rn = fma(rk, rk, rn);
    }
    rn = vec_block_sum(rn, sh);
    const double beta = rn / rs;
    for (int k = threadIdx.x; k < P; k += blockDim.x) p[k] = fma(beta, p[k], r[k]);
    if (threadIdx.x == 0) {
        const double it = sc[S_ITER] + 1.0;
        sc[S_ITER] = it;
        sc[S_RS] = rn;
        if (sqrt(rn) <= rtol * sc[S_FNORM] || it >= (double)max_iter || !isfinite(rn)) sc[S_DONE] = 1.0;
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
    // y [2n], Ap, r, p [P], zpart [256][P] upper bound, scalars
    return 2 * (size_t)n + 3 * (size_t)P + 256 * (size_t)P + S_COUNT;
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
    cudaStream_t s = env.stream;
    const dim3 cgrid((P + kColThreads - 1) / kColThreads, nchunks);
    const int rgrid = (int)((rows + kRowWarps - 1) / kRowWarps);

    energy_kernel<<<1, kVecThreads, 0, s>>>(eloc, n, y, sc);
    gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
    cg_init_kernel<<<1, kVecThreads, 0, s>>>(zpart, nchunks, P, n, delta, r, p, rtol, sc);
    if (cudaGetLastError() != cudaSuccess) { *env.msg = "SR setup launch failed"; return NQS_ERR_CUDA; }
    *env.launches += 3;

    double host_sc[S_COUNT];
    int done_iters = 0;
    int batch = 4;
    while (max_iter > 0) {
        for (int b = 0; b < batch; ++b) {
            gemv_rows_kernel<<<rgrid, kRowWarps * 32, 0, s>>>(O, p, rows, P, y, sc);
            center_kernel<<<1, kVecThreads, 0, s>>>(y, n, sc);
            gemv_cols_kernel<<<cgrid, kColThreads, 0, s>>>(O, y, rows, P, chunk_rows, zpart, sc);
            cg_step_kernel<<<1, kVecThreads, 0, s>>>(zpart, nchunks, P, n, eps, rtol, max_iter, delta, r, p, Ap, sc);
        }
        done_iters += batch;
        *env.launches += 4 * batch;
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
