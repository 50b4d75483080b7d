// mlp.cu -- tensor-core (tcgen05) kernels of the learned displacement model.
//
// This unit starts with the verification hook of the tensor-core tile: the
// product of BF16 operands accumulated in FP32 tensor memory, checked by the
// tests against a CPU product.
#include <string>

#include "kernels.cuh"
#include "tc.cuh"
#include "trime.h"

namespace trime {

// D (M x N, FP32) = A (M x K) * B^T (B: N x K), BF16 bits; one CTA per 128 rows
__global__ void __launch_bounds__(tc::kTcThreads) k_tc_gemm(const uint16_t* __restrict__ A,
                                                            const uint16_t* __restrict__ B, float* __restrict__ D,
                                                            int N, int K, uint32_t ncols, int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    int tid = threadIdx.x, warp = tid >> 5;
    uint8_t* sA = smem;
    uint8_t* sB = smem + (size_t)128 * K * 2;
    if (warp == 0) tc::tmem_alloc(&tslot, ncols);
    if (tid == 0) tc::mbar_init(&bar, 1);
    const uint16_t* Ab = A + (size_t)blockIdx.x * 128 * K;
    for (int i = tid; i < 128 * K; i += tc::kTcThreads) {
        int r = i / K, k = i - r * K;
        *reinterpret_cast<uint16_t*>(sA + tc::kmajor_offset(r, k, K)) = Ab[i];
    }
    for (int i = tid; i < N * K; i += tc::kTcThreads) {
        int r = i / K, k = i - r * K;
        *reinterpret_cast<uint16_t*>(sB + tc::kmajor_offset(r, k, K)) = B[i];
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tbase = tslot;
    if (tid == 0) tc::gemm_issue(tbase, sA, sB, N, K, false, &bar);
    bool ok = tc::mbar_wait(&bar, 0);
    ok = __all_sync(0xffffffffu, ok);
    tc::fence_after_sync();
    if (ok) {
        int row = blockIdx.x * 128 + warp * 32 + (tid & 31);
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; q++) D[(size_t)row * N + c + q] = v[q];
        }
    } else {
        if ((tid & 31) == 0) atomicExch(err, 1);
        tc::mbar_wait(&bar, 0);  // give the MMAs a second bounded chance before the memory goes away
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

}  // namespace trime

using namespace trime;

extern "C" int mesh_tc_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int32_t M, int32_t N, int32_t K) {
    if (M <= 0 || M % 128 || N < 16 || N > 256 || N % 16 || K < 16 || K > 256 || K % 16)
        return set_error(TRIME_EINVAL, "M must be a positive multiple of 128, N and K multiples of 16 in [16, 256]");
    if (!A || !B || !D) return set_error(TRIME_EINVAL, "NULL pointer");
    uint16_t *dA = nullptr, *dB = nullptr;
    float* dD = nullptr;
    int* derr = nullptr;
    size_t na = (size_t)M * K, nb = (size_t)N * K, nd = (size_t)M * N;
    cudaError_t e = cudaMalloc(&dA, na * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dB, nb * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dD, nd * 4);
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(dA);
        cudaFree(dB);
        cudaFree(dD);
        cudaFree(derr);
        return set_error(TRIME_ENOMEM, "cudaMalloc failed");
    }
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    size_t smem = (size_t)(128 + N) * K * 2;
    int herr = 0;
    e = cudaMemcpy(dA, A, na * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, nb * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_tc_gemm<<<M / 128, tc::kTcThreads, smem>>>(dA, dB, dD, N, K, ncols, derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, nd * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    if (e != cudaSuccess) return set_error(TRIME_ECUDA, (std::string("tc gemm: ") + cudaGetErrorString(e)).c_str());
    if (herr) return set_error(TRIME_ETIMEOUT, "tensor-core wait ran out");
    return TRIME_OK;
}
