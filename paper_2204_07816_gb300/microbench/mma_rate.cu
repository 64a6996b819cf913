// Microbenchmark: cycles per tcgen05.mma (M=128, K=16, bf16, no swizzle) as
// a function of N and of the number of issuing threads, with the same
// descriptor and instruction encodings as the library. All operands lie in
// bounds in shared memory. Build and run on a GB300:
//   nvcc -std=c++17 -O3 -gencode arch=compute_103a,code=sm_103a \
//        -o mma_rate paper_2204_07816_gb300/microbench/mma_rate.cu && ./mma_rate
#include <cstdio>
#include <cstdint>
#include "../csrc/tc_ptx.cuh"
using namespace nqs;

template <int N>
__global__ void k_rate(int nmma, int issuers, long long *out) {
    extern __shared__ __align__(128) unsigned char smem[];
    // A: 128 rows x 32 B = 4 KB per plane pair, use 64 KB region; B: N rows x 32 B
    const uint32_t A = ptx::smem_u32(smem), B = ptx::smem_u32(smem + 65536);
    __shared__ uint64_t bar[4];
    __shared__ uint32_t taddr;
    for (int i = threadIdx.x; i < (65536 + 16384) / 4; i += blockDim.x) reinterpret_cast<uint32_t *>(smem)[i] = 0;
    if (threadIdx.x == 0) { for (int i = 0; i < 4; ++i) ptx::mbar_init(&bar[i], 1); ptx::fence_mbar_init(); }
    ptx::fence_async_smem();
    __syncthreads();
    if (threadIdx.x < 32) { ptx::tmem_alloc(&taddr, 512); ptx::tmem_relinquish(); }
    ptx::tc_fence_before(); __syncthreads(); ptx::tc_fence_after();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long t0 = clock64();
    if (lane == 0 && warp < issuers) {
        const uint32_t idesc = ptx::idesc_bf16(128, N);
        const uint32_t plane = 128 * 16 * 4;   // rows 0..511 per plane (in bounds)
        for (int i = 0; i < nmma; ++i) {
            const uint32_t row = (uint32_t)((i * 7) % 256);
            const uint64_t ad = ptx::smem_desc(A + row * 16, plane, 128);
            const uint64_t bd = ptx::smem_desc(B, N * 16, 128);
            ptx::mma_bf16(taddr + (uint32_t)(warp * 128 % 512) * 0 + (uint32_t)((warp * N) % 256), ad, bd, idesc, i > 0);
        }
        ptx::mma_commit(&bar[warp]);
        ptx::mbar_wait(&bar[warp], 0);
    }
    __syncthreads();
    long long t1 = clock64();
    if (threadIdx.x == 0) out[0] = t1 - t0;
    ptx::tc_fence_before(); __syncthreads();
    if (threadIdx.x < 32) { ptx::tc_fence_after(); ptx::tmem_dealloc(taddr, 512); }
}

template <int N>
void run(int issuers) {
    long long *d, h = 0;
    cudaMalloc(&d, 8);
    auto k = k_rate<N>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536 + 16384);
    const int nmma = 2048;
    k<<<1, 128, 65536 + 16384>>>(nmma, issuers, d);
    cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(&h, d, 8, cudaMemcpyDeviceToHost);
    printf("N=%3d issuers=%d: %s  %.1f cycles per MMA (%.0f MACs/clk)\n", N, issuers, cudaGetErrorString(e),
           (double)h / (nmma * issuers), 128.0 * N * 16 * nmma * issuers / h);
    cudaFree(d);
}

int main() {
    for (int is = 1; is <= 4; is *= 2) { run<16>(is); run<32>(is); run<48>(is); run<64>(is); run<128>(is); run<256>(is); }
    return 0;
}
