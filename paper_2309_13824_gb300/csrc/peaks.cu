// peaks.cu -- measured issue peaks of the FP32 and FP64 pipes (the roofline
// denominators of the kernels bound by plain arithmetic, not by memory or
// tensor cores).  Every thread runs 8 independent chains of fused
// multiply-adds; the grid fills every SM several times over.
#include <string>

#include "kernels.cuh"
#include "trime.h"

namespace trime {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T* out, T b, T c, int iters) {
    T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
            a0 = fma(a0, b, c);
            a1 = fma(a1, b, c);
            a2 = fma(a2, b, c);
            a3 = fma(a3, b, c);
            a4 = fma(a4, b, c);
            a5 = fma(a5, b, c);
            a6 = fma(a6, b, c);
            a7 = fma(a7, b, c);
        }
    }
    T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains alive
}

template <typename T>
static int time_chain(int blocks, int iters, double& tflops, T* out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return set_error(TRIME_ECUDA, "event creation failed");
    k_fma_chain<T><<<blocks, 256>>>(out, (T)0.999999, (T)1e-7, iters / 8);  // warm-up
    cudaEventRecord(e0);
    k_fma_chain<T><<<blocks, 256>>>(out, (T)0.999999, (T)1e-7, iters);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(TRIME_ECUDA, cudaGetErrorString(e));
    double flops = 2.0 * 8 * 16 * (double)iters * 256.0 * (double)blocks;
    tflops = flops / (ms * 1e-3) / 1e12;
    return 0;
}

}  // namespace trime

using namespace trime;

extern "C" int mesh_measure_pipe_peaks(double* fp32_tflops, double* fp64_tflops, int32_t* sm_count,
                                       int32_t* sm_clock_khz) {
    if (!fp32_tflops || !fp64_tflops) return set_error(TRIME_EINVAL, "NULL pointer");
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return set_error(TRIME_ECUDA, "device query failed");
    int clk = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
    if (sm_count) *sm_count = prop.multiProcessorCount;
    if (sm_clock_khz) *sm_clock_khz = clk;
    void* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * 65536) != cudaSuccess) return set_error(TRIME_ENOMEM, "cudaMalloc failed");
    int blocks = prop.multiProcessorCount * 8;
    int rc = time_chain<float>(blocks, 4096, *fp32_tflops, (float*)out);
    if (!rc) rc = time_chain<double>(blocks, 256, *fp64_tflops, (double*)out);
    cudaFree(out);
    return rc;
}
