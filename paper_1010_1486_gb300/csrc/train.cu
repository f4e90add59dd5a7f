// train.cu -- training of the learned a0 proposal on the GPU: forward and
// backward passes of the MLP + rational-quadratic spline negative
// log-likelihood, with the two hidden-layer contractions of each pass on the
// 5th-generation tensor cores (BF16 operands, FP32 accumulation in tensor
// memory), and an Adam update.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "su2_device.cuh"
#include "su2_internal.h"
#include "tc05.cuh"

namespace su2 {

constexpr uint32_t kMbarPolls = 1u << 26;

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Self-test: D (128 x 32, FP32) = A (128 x K, BF16) * B (32 x K, BF16)^T on the
// tensor cores, K = 16 or 32, for comparison with a host reference.
__global__ void __launch_bounds__(128) mma_selftest_kernel(const uint16_t *__restrict__ A,
                                                           const uint16_t *__restrict__ B, int K,
                                                           float *__restrict__ D, unsigned int *__restrict__ err)
{
    __shared__ __align__(128) unsigned char sA[128 * 32 * 2];
    __shared__ __align__(128) unsigned char sB[32 * 32 * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    for (int k = 0; k < K; ++k) *(uint16_t *)(sA + tc::tile_offset(t, k, K)) = A[t * K + k];
    if (t < 32)
        for (int k = 0; k < K; ++k) *(uint16_t *)(sB + tc::tile_offset(t, k, K)) = B[t * K + k];
    tc::fence_smem_to_async();
    if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_base;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int j = 0; j < K / 16; ++j) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + 256u * j, 128u, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + 256u * j, 128u, sbo);
            tc::mma_bf16(taddr, ad, bd, idesc, j > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    bool ok = tc::mbar_wait(&mbar, 0, kMbarPolls);
    if (!ok) ok = tc::mbar_wait(&mbar, 0, kMbarPolls);  // second bounded wait before giving up
    tc::fence_after_sync();
    if (ok) {
        float v[32];
        tc::tmem_load32(taddr + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
        for (int n = 0; n < 32; ++n) D[t * 32 + n] = v[n];
    } else if ((t & 31) == 0) {
        atomicAdd(err, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

}  // namespace su2

using namespace su2;

extern "C" su2_status su2_selftest_mma(const uint16_t *A, const uint16_t *B, int K, float *D)
{
    if (!A || !B || !D || (K != 16 && K != 32)) return SU2_E_INVAL;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    const size_t bytesA = 128 * (size_t)K * 2, bytesB = 32 * (size_t)K * 2, bytesD = 128 * 32 * 4;
    char *buf = (char *)device_alloc(bytesA + bytesB + bytesD + 512, dev, nullptr);
    if (!buf) return SU2_E_NOMEM;
    uint16_t *dA = (uint16_t *)buf;
    uint16_t *dB = (uint16_t *)(buf + ((bytesA + 255) & ~(size_t)255));
    float *dD = (float *)((char *)dB + ((bytesB + 255) & ~(size_t)255));
    unsigned int *dErr = (unsigned int *)((char *)dD + bytesD);
    su2_status st = SU2_OK;
    cudaError_t e = cudaMemcpy(dA, A, bytesA, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, bytesB, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        mma_selftest_kernel<<<1, 128>>>(dA, dB, K, dD, dErr);
        e = cudaGetLastError();
    }
    unsigned int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, bytesD, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, dErr, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_fail(e, "su2_selftest_mma");
    else if (err) {
        set_last_error("tensor-core self-test: completion wait gave up");
        st = SU2_E_DEVICE_TIMEOUT;
    }
    device_free(buf, bytesA + bytesB + bytesD + 512, dev, nullptr);
    cudaDeviceSynchronize();
    return st;
}
