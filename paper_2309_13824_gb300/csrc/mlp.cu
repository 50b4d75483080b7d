// mlp.cu -- the learned displacement model on the tensor cores (tcgen05).
//
// A 3-layer perceptron (48 BF16 inputs, two hidden layers of 64 ReLU units,
// 2 outputs) proposes, for every point, its displacement over the next
// iterations of the plain method divided by h_i, from local features: the
// offsets of its 16 nearest points times 1 / h_i, ln(h_i / h_avg), the sizing
// gradient, the boundary flag and the move in use.  The paper's method has no
// learned part; plain iterations stay the fallback and judge the proposals.
// Two more features carry the point's last move times 1 / h_i, so the model can
// extrapolate the trajectory it is on.
//
// Every product runs on the tensor cores: one CTA of 128 threads takes 128
// samples, stages each operand in shared memory in the K-major core-matrix
// layout (tc.cuh) and accumulates in tensor memory.  Training fuses the
// forward pass, the backward pass and the weight-gradient products; weight
// gradients accumulate in tensor memory across the CTA's tiles (the bias
// gradients come from a row of ones appended to the transposed activations)
// and are added to global memory once per CTA.
#include <algorithm>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc.cuh"
#include "treat.cuh"
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


// ------------------------------------------------------------------ shared helpers
namespace {
constexpr int kRows = 128;  // samples per tile = tensor-memory lanes
constexpr uint32_t kSzW1 = kMlpHid * kMlpIn * 2;
constexpr uint32_t kSzW2 = kMlpHid * kMlpHid * 2;
constexpr uint32_t kSzW3 = kMlpOutPad * kMlpHid * 2;
constexpr uint32_t kSzX = kRows * kMlpIn * 2;
constexpr uint32_t kSzH = kRows * kMlpHid * 2;
constexpr uint32_t kSzT = kRows * kRows * 2;        // transposed activations, 128 rows x 128 samples
constexpr uint32_t kSzY = kRows * kMlpOutPad * 2;
constexpr uint16_t kBf16One = 0x3F80;
constexpr size_t kFwdSmem = kSzW1 + kSzW2 + kSzW3 + kSzX + kSzH;
constexpr size_t kGradSmem = kSzW1 + 2 * kSzW2 + 2 * kSzW3 + kSzX + 2 * kSzH + 3 * kSzT + 2 * kSzY;
}  // namespace

__device__ __forceinline__ void put_bf16(uint8_t* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void put_bits(uint8_t* base, uint32_t off, uint16_t v) {
    *reinterpret_cast<uint16_t*>(base + off) = v;
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// the B operands of the forward pass
__device__ void stage_fwd_weights(const MlpDev& w, uint8_t* sW1, uint8_t* sW2, uint8_t* sW3) {
    for (int i = threadIdx.x; i < kMlpHid * kMlpIn; i += kRows)
        put_bits(sW1, tc::kmajor_offset(i / kMlpIn, i % kMlpIn, kMlpIn), w.w1[i]);
    for (int i = threadIdx.x; i < kMlpHid * kMlpHid; i += kRows)
        put_bits(sW2, tc::kmajor_offset(i / kMlpHid, i % kMlpHid, kMlpHid), w.w2[i]);
    for (int i = threadIdx.x; i < kMlpOutPad * kMlpHid; i += kRows)
        put_bits(sW3, tc::kmajor_offset(i / kMlpHid, i % kMlpHid, kMlpHid), w.w3[i]);
}

// this thread's sample row of X into the K-major tile (zeros past the end)
__device__ __forceinline__ void stage_x_row(const uint16_t* X, int src, uint8_t* sX, int r) {
    const uint4* g = reinterpret_cast<const uint4*>(X + (size_t)(src < 0 ? 0 : src) * kMlpIn);
#pragma unroll
    for (int c = 0; c < kMlpIn / 8; c++) {
        uint4 v = src >= 0 ? g[c] : make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(sX + tc::kmajor_offset(r, 8 * c, kMlpIn)) = v;
    }
}

// 64 accumulator columns of this thread's lane, plus bias
__device__ __forceinline__ void load_row64(uint32_t taddr, const float* bias, float* z) {
#pragma unroll
    for (int c = 0; c < 4; c++) tc::tmem_ld16(taddr + 16 * c, z + 16 * c);
#pragma unroll
    for (int u = 0; u < kMlpHid; u++) z[u] += bias[u];
}

// relu(z) as BF16 into row r of a K-major 128 x 64 tile
__device__ __forceinline__ void store_relu_row(const float* z, uint8_t* sH, int r) {
#pragma unroll
    for (int c = 0; c < 8; c++) {
        uint4 v;
        v.x = pack2(fmaxf(z[8 * c], 0.f), fmaxf(z[8 * c + 1], 0.f));
        v.y = pack2(fmaxf(z[8 * c + 2], 0.f), fmaxf(z[8 * c + 3], 0.f));
        v.z = pack2(fmaxf(z[8 * c + 4], 0.f), fmaxf(z[8 * c + 5], 0.f));
        v.w = pack2(fmaxf(z[8 * c + 6], 0.f), fmaxf(z[8 * c + 7], 0.f));
        *reinterpret_cast<uint4*>(sH + tc::kmajor_offset(r, 8 * c, kMlpHid)) = v;
    }
}

__device__ __forceinline__ void sync_for_mma() {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// waits for the next completion of `bar`; the result is the same in every thread
__device__ __forceinline__ bool wait_all(uint64_t* bar, uint32_t& phase) {
    bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    return ok;
}

// ------------------------------------------------------------------ inference
__global__ void __launch_bounds__(kRows) k_mlp_forward(const MlpDev w, const uint16_t* __restrict__ X,
                                                       const int32_t* __restrict__ idx, int n,
                                                       float* __restrict__ Y, int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sW1 = smem;
    uint8_t* sW2 = sW1 + kSzW1;
    uint8_t* sW3 = sW2 + kSzW2;
    uint8_t* sX = sW3 + kSzW3;
    uint8_t* sH = sX + kSzX;
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float sb[2 * kMlpHid + kMlpOut];
    int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&tslot, 128);
    if (tid == 0) tc::mbar_init(&bar, 1);
    stage_fwd_weights(w, sW1, sW2, sW3);
    for (int i = tid; i < kMlpHid; i += kRows) {
        sb[i] = w.p[kOB1 + i];
        sb[kMlpHid + i] = w.p[kOB2 + i];
    }
    if (tid < kMlpOut) sb[2 * kMlpHid + tid] = w.p[kOB3 + tid];
    sync_for_mma();
    const uint32_t tbase = tslot, lane = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    int ntiles = (n + kRows - 1) / kRows;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int row = tile * kRows + tid;
        int src = row < n ? (idx ? idx[row] : row) : -1;
        stage_x_row(X, src, sX, tid);
        sync_for_mma();
        if (tid == 0) tc::gemm_issue(tbase, sX, sW1, kMlpHid, kMlpIn, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        float z[kMlpHid];
        load_row64(tbase + lane, sb, z);
        store_relu_row(z, sH, tid);
        sync_for_mma();
        if (tid == 0) tc::gemm_issue(tbase + 64, sH, sW2, kMlpHid, kMlpHid, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        load_row64(tbase + lane + 64, sb + kMlpHid, z);
        store_relu_row(z, sH, tid);
        sync_for_mma();
        if (tid == 0) tc::gemm_issue(tbase, sH, sW3, kMlpOutPad, kMlpHid, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        float y[16];
        tc::tmem_ld16(tbase + lane, y);
        if (row < n) {
            Y[2 * (size_t)row] = y[0] + sb[2 * kMlpHid];
            Y[2 * (size_t)row + 1] = y[1] + sb[2 * kMlpHid + 1];
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait(&bar, phase ^ 1u);  // a second bounded chance for the MMAs in flight
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
}

void launch_mlp_forward(const MlpDev& w, const uint16_t* X, const int32_t* idx, int n, float* Y, int* err,
                        cudaStream_t st) {
    if (n <= 0) return;
    int ntiles = (n + kRows - 1) / kRows;
    int grid = std::min(ntiles, 152 * 4);
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    k_mlp_forward<<<grid, kRows, kFwdSmem, st>>>(w, X, idx, n, Y, err);
}

// ------------------------------------------------------------------ training
// issue the MMAs of one 128 x N x K product without committing
__device__ __forceinline__ void mmas(uint32_t d, const void* A, const void* B, int N, int K, bool acc) {
    uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
    uint32_t idesc = tc::make_idesc_bf16(N), sbo = (uint32_t)K * 16;
    for (int k = 0; k < K; k += 16) {
        uint32_t off = (uint32_t)(k >> 3) * 128;
        tc::mma_bf16(d, tc::make_sdesc(a0 + off, 128, sbo), tc::make_sdesc(b0 + off, 128, sbo), idesc, acc || k > 0);
    }
}

__global__ void __launch_bounds__(kRows, 1) k_mlp_grad(const MlpDev w, const uint16_t* __restrict__ X,
                                                       const float* __restrict__ T, const int32_t* __restrict__ idx,
                                                       int n, float scale, float* __restrict__ gpart, double* loss,
                                                       int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sW1 = smem;
    uint8_t* sW2 = sW1 + kSzW1;
    uint8_t* sW2T = sW2 + kSzW2;
    uint8_t* sW3 = sW2T + kSzW2;
    uint8_t* sW3T = sW3 + kSzW3;
    uint8_t* sX = sW3T + kSzW3;
    uint8_t* sH1 = sX + kSzX;   // H1, later dZ2^T (64 x 128)
    uint8_t* sH2 = sH1 + kSzH;  // H2, later dZ2 (128 x 64)
    uint8_t* sXT = sH2 + kSzH;  // X^T (rows 0..47), ones (row 48)
    uint8_t* sH1T = sXT + kSzT; // H1^T (rows 0..63), ones (row 64)
    uint8_t* sH2T = sH1T + kSzT;// H2^T (rows 0..63), ones (row 64); rows 0..63 later dZ1^T
    uint8_t* sdY = sH2T + kSzT; // dY (128 x 16)
    uint8_t* sdYT = sdY + kSzY; // dY^T (16 x 128)
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float sb[2 * kMlpHid + kMlpOut];
    __shared__ double sloss[kRows / 32];
    // tensor-memory columns
    constexpr uint32_t cZ1 = 0, cZ2 = 64, cY = 128, cA3 = 160, cA2 = 192, cA1 = 256;
    int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tc::tmem_alloc(&tslot, 512);
    if (tid == 0) tc::mbar_init(&bar, 1);
    stage_fwd_weights(w, sW1, sW2, sW3);
    for (int i = tid; i < kMlpHid * kMlpHid; i += kRows) {
        int u = i / kMlpHid, r = i % kMlpHid;  // W2[u][r] -> B[r][u] of dH1 = dZ2 W2
        put_bits(sW2T, tc::kmajor_offset(r, u, kMlpHid), w.w2[i]);
    }
    for (int i = tid; i < kMlpHid * kMlpOutPad; i += kRows) {
        int u = i / kMlpOutPad, o = i % kMlpOutPad;  // W3[o][u] -> B[u][o] of dH2 = dY W3
        put_bits(sW3T, tc::kmajor_offset(u, o, kMlpOutPad), o < kMlpOut ? w.w3[o * kMlpHid + u] : (uint16_t)0);
    }
    for (int i = tid; i < kRows * kRows; i += kRows) {
        int r = i / kRows, k = i % kRows;
        put_bits(sXT, tc::kmajor_offset(r, k, kRows), r == kMlpIn ? kBf16One : (uint16_t)0);
        put_bits(sH1T, tc::kmajor_offset(r, k, kRows), r == kMlpHid ? kBf16One : (uint16_t)0);
        put_bits(sH2T, tc::kmajor_offset(r, k, kRows), r == kMlpHid ? kBf16One : (uint16_t)0);
    }
    for (int i = tid; i < kRows * kMlpOutPad; i += kRows) {
        put_bits(sdY, tc::kmajor_offset(i / kMlpOutPad, i % kMlpOutPad, kMlpOutPad), 0);
        put_bits(sdYT, tc::kmajor_offset(i / kRows, i % kRows, kRows), 0);
    }
    for (int i = tid; i < kMlpHid; i += kRows) {
        sb[i] = w.p[kOB1 + i];
        sb[kMlpHid + i] = w.p[kOB2 + i];
    }
    if (tid < kMlpOut) sb[2 * kMlpHid + tid] = w.p[kOB3 + tid];
    sync_for_mma();
    const uint32_t tbase = tslot, lane = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true, first = true;
    double lsum = 0.0;
    int ntiles = (n + kRows - 1) / kRows;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int row = tile * kRows + tid;
        int src = row < n ? (idx ? idx[row] : row) : -1;
        // 1. inputs, row-wise and transposed
        stage_x_row(X, src, sX, tid);
        {
            const uint16_t* xr = X + (size_t)(src < 0 ? 0 : src) * kMlpIn;
            for (int f = 0; f < kMlpIn; f++) put_bits(sXT, tc::kmajor_offset(f, tid, kRows), src >= 0 ? xr[f] : 0);
        }
        float t0 = src >= 0 ? T[2 * (size_t)src] : 0.f, t1 = src >= 0 ? T[2 * (size_t)src + 1] : 0.f;
        sync_for_mma();
        // 2. Z1 = X W1^T
        if (tid == 0) tc::gemm_issue(tbase + cZ1, sX, sW1, kMlpHid, kMlpIn, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        float z[kMlpHid];
        uint32_t m1a = 0, m1b = 0, m2a = 0, m2b = 0;
        load_row64(tbase + lane + cZ1, sb, z);
#pragma unroll
        for (int u = 0; u < kMlpHid; u++) {
            if (z[u] > 0.f) (u < 32 ? m1a : m1b) |= 1u << (u & 31);
            put_bf16(sH1T, tc::kmajor_offset(u, tid, kRows), fmaxf(z[u], 0.f));
        }
        store_relu_row(z, sH1, tid);
        sync_for_mma();
        // 3. Z2 = H1 W2^T
        if (tid == 0) tc::gemm_issue(tbase + cZ2, sH1, sW2, kMlpHid, kMlpHid, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        load_row64(tbase + lane + cZ2, sb + kMlpHid, z);
#pragma unroll
        for (int u = 0; u < kMlpHid; u++) {
            if (z[u] > 0.f) (u < 32 ? m2a : m2b) |= 1u << (u & 31);
            put_bf16(sH2T, tc::kmajor_offset(u, tid, kRows), fmaxf(z[u], 0.f));
        }
        store_relu_row(z, sH2, tid);
        sync_for_mma();
        // 4. Y = H2 W3^T, residual, dY
        if (tid == 0) tc::gemm_issue(tbase + cY, sH2, sW3, kMlpOutPad, kMlpHid, false, &bar);
        if (!(ok = wait_all(&bar, phase))) break;
        {
            float y[16];
            tc::tmem_ld16(tbase + lane + cY, y);
            float r0 = src >= 0 ? y[0] + sb[2 * kMlpHid] - t0 : 0.f;
            float r1 = src >= 0 ? y[1] + sb[2 * kMlpHid + 1] - t1 : 0.f;
            lsum += (double)r0 * r0 + (double)r1 * r1;
            put_bf16(sdY, tc::kmajor_offset(tid, 0, kMlpOutPad), r0 * scale);
            put_bf16(sdY, tc::kmajor_offset(tid, 1, kMlpOutPad), r1 * scale);
            put_bf16(sdYT, tc::kmajor_offset(0, tid, kRows), r0 * scale);
            put_bf16(sdYT, tc::kmajor_offset(1, tid, kRows), r1 * scale);
        }
        sync_for_mma();
        // 5. gW3^T += H2^T dY (bias row 64), dH2 = dY W3
        if (tid == 0) {
            mmas(tbase + cA3, sH2T, sdYT, kMlpOutPad, kRows, !first);
            mmas(tbase + cZ2, sdY, sW3T, kMlpHid, kMlpOutPad, false);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_all(&bar, phase))) break;
        {
            float d[kMlpHid];
#pragma unroll
            for (int c = 0; c < 4; c++) tc::tmem_ld16(tbase + lane + cZ2 + 16 * c, d + 16 * c);
#pragma unroll
            for (int u = 0; u < kMlpHid; u++) {
                float g = (((u < 32 ? m2a : m2b) >> (u & 31)) & 1u) ? d[u] : 0.f;
                put_bf16(sH1, tc::kmajor_offset(u, tid, kRows), g);    // dZ2^T
                put_bf16(sH2, tc::kmajor_offset(tid, u, kMlpHid), g);  // dZ2
            }
        }
        sync_for_mma();
        // 6. gW2^T += H1^T dZ2 (bias row 64), dH1 = dZ2 W2
        if (tid == 0) {
            mmas(tbase + cA2, sH1T, sH1, kMlpHid, kRows, !first);
            mmas(tbase + cZ1, sH2, sW2T, kMlpHid, kMlpHid, false);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_all(&bar, phase))) break;
        {
            float d[kMlpHid];
#pragma unroll
            for (int c = 0; c < 4; c++) tc::tmem_ld16(tbase + lane + cZ1 + 16 * c, d + 16 * c);
#pragma unroll
            for (int u = 0; u < kMlpHid; u++) {
                float g = (((u < 32 ? m1a : m1b) >> (u & 31)) & 1u) ? d[u] : 0.f;
                put_bf16(sH2T, tc::kmajor_offset(u, tid, kRows), g);  // dZ1^T over H2^T's rows 0..63
            }
        }
        sync_for_mma();
        // 7. gW1^T += X^T dZ1 (bias row 48)
        if (tid == 0) {
            mmas(tbase + cA1, sXT, sH2T, kMlpHid, kRows, !first);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_all(&bar, phase))) break;
        first = false;
    }
    // this CTA's gradient sums into its own slot (lane r = row r of the
    // transposed gradients); the slots are added in a fixed order afterwards,
    // so training is deterministic
    float* G = gpart + (size_t)blockIdx.x * kMlpParams;
    if (ok && !first) {
        float a[kMlpHid];
#pragma unroll
        for (int c = 0; c < 4; c++) tc::tmem_ld16(tbase + lane + cA1 + 16 * c, a + 16 * c);
        if (tid < kMlpIn)
            for (int u = 0; u < kMlpHid; u++) G[kOW1 + u * kMlpIn + tid] = a[u];
        else if (tid == kMlpIn)
            for (int u = 0; u < kMlpHid; u++) G[kOB1 + u] = a[u];
#pragma unroll
        for (int c = 0; c < 4; c++) tc::tmem_ld16(tbase + lane + cA2 + 16 * c, a + 16 * c);
        if (tid < kMlpHid)
            for (int u = 0; u < kMlpHid; u++) G[kOW2 + u * kMlpHid + tid] = a[u];
        else if (tid == kMlpHid)
            for (int u = 0; u < kMlpHid; u++) G[kOB2 + u] = a[u];
        tc::tmem_ld16(tbase + lane + cA3, a);
        if (tid < kMlpHid)
            for (int o = 0; o < kMlpOut; o++) G[kOW3 + o * kMlpHid + tid] = a[o];
        else if (tid == kMlpHid)
            for (int o = 0; o < kMlpOut; o++) G[kOB3 + o] = a[o];
    } else {
        for (int k = tid; k < kMlpParams; k += kRows) G[k] = 0.f;
    }
    // loss of this CTA's samples
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) sloss[warp] = lsum;
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        tc::mbar_wait(&bar, phase ^ 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) atomicAdd(loss, 0.5 * (double)scale * (sloss[0] + sloss[1] + sloss[2] + sloss[3]));
    if (warp == 0) tc::tmem_dealloc(tbase, 512);
}

int launch_mlp_grad(const MlpDev& w, const uint16_t* X, const float* T, const int32_t* idx, int n, float scale,
                    float* gpart, double* loss, int* err, cudaStream_t st) {
    if (n <= 0) return 0;
    int ntiles = (n + kRows - 1) / kRows;
    int grid = std::min(ntiles, kGradParts);
    cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    k_mlp_grad<<<grid, kRows, kGradSmem, st>>>(w, X, T, idx, n, scale, gpart, loss, err);
    return grid;
}

// the gradient: the per-CTA slots added in slot order
__global__ void k_mlp_reduce(const float* gpart, int nparts, float* grad) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpParams) return;
    float g = 0.f;
    for (int c = 0; c < nparts; c++) g += gpart[(size_t)c * kMlpParams + k];
    grad[k] = g;
}

// Adam on the FP32 parameters (gradient: the per-CTA slots added in slot
// order); refreshes the BF16 copies
__global__ void k_mlp_adam(float* p, const float* gpart, int nparts, float* m, float* v, uint16_t* w1, uint16_t* w2,
                           uint16_t* w3, float lr, float b1, float b2, float eps, float c1, float c2) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpParams) return;
    float g = 0.f;
    for (int c = 0; c < nparts; c++) g += gpart[(size_t)c * kMlpParams + k];
    float mk = b1 * m[k] + (1.f - b1) * g;
    float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(pk));
    if (k < kOB1) w1[k] = b;
    else if (k >= kOW2 && k < kOB2) w2[k - kOW2] = b;
    else if (k >= kOW3 && k < kOB3) w3[k - kOW3] = b;
}

__global__ void k_mlp_refresh(const float* p, uint16_t* w1, uint16_t* w2, uint16_t* w3) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpOut * kMlpHid && k < kMlpOutPad * kMlpHid) w3[k] = 0;  // padding rows of W3
    if (k >= kMlpParams) return;
    uint16_t b = __bfloat16_as_ushort(__float2bfloat16_rn(p[k]));
    if (k < kOB1) w1[k] = b;
    else if (k >= kOW2 && k < kOB2) w2[k - kOW2] = b;
    else if (k >= kOW3 && k < kOB3) w3[k - kOW3] = b;
}

// ------------------------------------------------------------------ features, proposals, targets
// derivatives of the bilinear sizing interpolant at (x, y) by fixed formulas
__device__ __forceinline__ void sizing_grad_fixed(const DevGrid& g, double x, double y, double& gx, double& gy) {
    int i, j;
    double fx, fy;
    grid_locate(g, x, y, i, j, fx, fy);
    const float* r0 = g.v + (size_t)j * g.nx + i;
    const float* r1 = r0 + g.nx;
    double v00 = __ldg(r0), v10 = __ldg(r0 + 1), v01 = __ldg(r1), v11 = __ldg(r1 + 1);
    gx = fdiv(fadd(fsub(v10, v00), fmul(fy, fsub(fsub(v11, v01), fsub(v10, v00)))), g.dx);
    gy = fdiv(fadd(fsub(v01, v00), fmul(fx, fsub(fsub(v11, v10), fsub(v01, v00)))), g.dy);
}

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// One thread per slot: the 16 nearest other points of the slot's mesh by
// (squared FP64 distance, index), found ring by ring in the bucket grid until
// no unscanned bucket can hold a nearer point, then the 48 features.  In a
// batch the padding slots are skipped (their rows are left as they are).
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_features(const __grid_constant__ IterArgs<T> a, uint16_t* X, float* H,
                                                       T* px, T* py, const T* qx, const T* qy, int by_id,
                                                       float mflag) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    const MeshView& V = mesh_of<B>(a, s);
    if (B && s - V.soff >= V.n) return;
    const DevParams& P = V.P;
    T xt = a.srt.x[s], yt = a.srt.y[s];
    double xd = (double)xt, yd = (double)yt;
    int id = a.srt.id[s];
    double h = V.gh[a.cell[s]];
    // the 16 nearest so far: squared FP64 distances as their bit patterns
    // (for non-negative doubles the unsigned order of the bits is the order
    // of the values, so the insertion compares on the integer pipe), ids,
    // slots
    unsigned long long bd[16];
    int bid[16], bq[16];
    int cnt = 0;
    // once 16 are held, a candidate whose float-pair squared distance f2
    // certainly exceeds the 16th (f2 (1 - 2^-18) > bd[15], with bd[15]
    // rounded up to float in b15) is skipped without the FP64 distance: the
    // float-pair difference has a relative error below 2^-22 for |d| >=
    // 2^-20, so f2 is within 2^-20 of d^2, and such a candidate would be
    // rejected by the exact comparison anyway
    float b15 = __int_as_float(0x7f800000);
    const float4 pi4 = a.pf[s];
    int bxi, byi;
    bucket_of(P, xt, yt, bxi, byi);
    double margin = 1e-3 * (P.bsx > P.bsy ? P.bsx : P.bsy) + 4e-6 * (1.0 + fabs(xd) + fabs(yd));
    // candidate q: the float pre-test, then the exact (FP64 distance, id)
    // insertion into the 16 nearest
    auto consider = [&](int q, const float4& pq) {
        if (q == s) return;
        if (cnt == 16) {
            const float fx = ff_diff(pq.x, pq.y, pi4.x, pi4.y), fy = ff_diff(pq.z, pq.w, pi4.z, pi4.w);
            const float f2 = fx * fx + fy * fy;
            if (f2 >= 9.094947e-13f && f2 * (1.0f - 0x1p-18f) > b15) return;
        }
        double dx = fsub((double)a.srt.x[q], xd), dy = fsub((double)a.srt.y[q], yd);
        const unsigned long long d2 = (unsigned long long)__double_as_longlong(fadd(fmul(dx, dx), fmul(dy, dy)));
        int qi = a.srt.id[q];
        if (cnt == 16 && !(d2 < bd[15] || (d2 == bd[15] && qi < bid[15]))) return;
        int p = cnt < 16 ? cnt++ : 15;
        while (p > 0 && (d2 < bd[p - 1] || (d2 == bd[p - 1] && qi < bid[p - 1]))) {
            bd[p] = bd[p - 1];
            bid[p] = bid[p - 1];
            bq[p] = bq[p - 1];
            p--;
        }
        bd[p] = d2;
        bid[p] = qi;
        bq[p] = q;
        if (cnt == 16) b15 = __double2float_ru(__longlong_as_double((long long)bd[15]));
    };
    // the slots [lo, hi) four at a time, their positions loaded together
    auto scan = [&](int lo, int hi) {
        for (int q0 = lo; q0 < hi; q0 += 4) {
            float4 pq[4];
#pragma unroll
            for (int u = 0; u < 4; u++) pq[u] = q0 + u < hi ? a.pf[q0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (q0 + u < hi) consider(q0 + u, pq[u]);
        }
    };
    for (int r = 0;; r++) {
        // the ring's buckets: its top and bottom rows as one slot range each
        // (the buckets of a row are consecutive in the sorted order), the
        // two side buckets of the rows between
        for (int by = byi - r; by <= byi + r; by++) {
            if (by < 0 || by >= P.nby) continue;
            const int k0 = V.boff + by * P.nbx;
            if (r == 0 || by == byi - r || by == byi + r) {
                const int c0 = max(bxi - r, 0), c1 = min(bxi + r, P.nbx - 1);
                scan(a.bstart[k0 + c0], a.bstart[k0 + c1 + 1]);
            } else {
                if (bxi - r >= 0) scan(a.bstart[k0 + bxi - r], a.bstart[k0 + bxi - r + 1]);
                if (bxi + r < P.nbx) scan(a.bstart[k0 + bxi + r], a.bstart[k0 + bxi + r + 1]);
            }
        }
        if (bxi - r <= 0 && bxi + r >= P.nbx - 1 && byi - r <= 0 && byi + r >= P.nby - 1) break;
        if (cnt == 16) {
            double dmin = 1e300;
            if (bxi - r > 0) dmin = fmin(dmin, xd - (P.bx0 + (bxi - r) * P.bsx));
            if (bxi + r < P.nbx - 1) dmin = fmin(dmin, (P.bx0 + (bxi + r + 1) * P.bsx) - xd);
            if (byi - r > 0) dmin = fmin(dmin, yd - (P.by0 + (byi - r) * P.bsy));
            if (byi + r < P.nby - 1) dmin = fmin(dmin, (P.by0 + (byi + r + 1) * P.bsy) - yd);
            dmin -= margin;
            if (dmin > 0.0 && __longlong_as_double((long long)bd[15]) < dmin * dmin) break;
        }
    }
    size_t row = (size_t)(by_id ? id : s);
    // offsets are scaled by r_i = 1 / h_i rounded once (one division per
    // point instead of one per offset)
    const double rh = fdiv(1.0, h);
    __align__(16) uint16_t f[kMlpIn];
    for (int k = 0; k < 16; k++) {
        if (k < cnt) {
            int j = bq[k];
            f[2 * k] = bf16_bits((float)fmul(fsub((double)a.srt.x[j], xd), rh));
            f[2 * k + 1] = bf16_bits((float)fmul(fsub((double)a.srt.y[j], yd), rh));
        } else {
            f[2 * k] = f[2 * k + 1] = 0;
        }
    }
    double gx, gy;
    sizing_grad_fixed(V.siz, xd, yd, gx, gy);
    f[32] = bf16_bits((float)log(fdiv(h, P.havg)));
    f[33] = bf16_bits((float)gx);
    f[34] = bf16_bits((float)gy);
    f[35] = a.srt.cls[s] == PT_BOUNDARY ? kBf16One : 0;
    // the move in use: given by the caller, or (mflag < 0) read from the
    // slot's mesh: CVD iterations once the hybrid has switched
    float mf = mflag;
    if (mf < 0.0f) mf = (V.ctrl->method_param == 1 || (V.ctrl->method_param == 2 && V.ctrl->switched)) ? 1.0f : 0.0f;
    f[36] = bf16_bits(mf);
    f[37] = qx ? bf16_bits((float)fmul(fsub(xd, (double)qx[id]), rh)) : 0;
    f[38] = qy ? bf16_bits((float)fmul(fsub(yd, (double)qy[id]), rh)) : 0;
    for (int k = kMlpFeat; k < kMlpIn; k++) f[k] = 0;
    uint4* dst = reinterpret_cast<uint4*>(X + row * kMlpIn);
    const uint4* src = reinterpret_cast<const uint4*>(f);
#pragma unroll
    for (int c = 0; c < kMlpIn / 8; c++) dst[c] = src[c];
    if (H) H[row] = (float)h;
    if (px) {
        px[id] = xt;
        py[id] = yt;
    }
}

template <typename T>
void launch_features(const IterArgs<T>& a, uint16_t* X, float* H, T* px, T* py, const T* qx, const T* qy, int by_id,
                     float method_cvd, cudaStream_t st) {
    int g = (a.n + kThreads - 1) / kThreads;
    if (g <= 0) return;
    if (a.Vs) k_features<T, true><<<g, kThreads, 0, st>>>(a, X, H, px, py, qx, qy, by_id, method_cvd);
    else k_features<T, false><<<g, kThreads, 0, st>>>(a, X, H, px, py, qx, qy, by_id, method_cvd);
}
template void launch_features<double>(const IterArgs<double>&, uint16_t*, float*, double*, double*, const double*,
                                      const double*, int, float, cudaStream_t);
template void launch_features<float>(const IterArgs<float>&, uint16_t*, float*, float*, float*, const float*,
                                     const float*, int, float, cudaStream_t);

template <typename T, bool B>
__global__ void k_snapshot(const __grid_constant__ IterArgs<T> a, T* qx, T* qy) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    if (B && s - mesh_of<B>(a, s).soff >= mesh_of<B>(a, s).n) return;  // padding slot (its id is not a point's)
    int id = a.cur.id[s];
    qx[id] = a.cur.x[s];
    qy[id] = a.cur.y[s];
}

template <typename T>
void launch_snapshot(const IterArgs<T>& a, T* qx, T* qy, cudaStream_t st) {
    int g = (a.n + kThreads - 1) / kThreads;
    if (g <= 0) return;
    if (a.Vs) k_snapshot<T, true><<<g, kThreads, 0, st>>>(a, qx, qy);
    else k_snapshot<T, false><<<g, kThreads, 0, st>>>(a, qx, qy);
}
template void launch_snapshot<double>(const IterArgs<double>&, double*, double*, cudaStream_t);
template void launch_snapshot<float>(const IterArgs<float>&, float*, float*, cudaStream_t);

// the proposed move p + h_i Y of every slot, clamped and treated (Sec. 4.3);
// the recorded previous move is capped at one plain step (fac_pt h_i).  In a
// batch, padding slots and meshes that have terminated are left alone (the
// 32 slots of a warp belong to one mesh).
template <typename T, bool B>
__global__ void __launch_bounds__(kThreads) k_propose(const __grid_constant__ IterArgs<T> a, const float* Y, float jump) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long tcap = 0, nfail = 0;
    const MeshView& V = mesh_of<B>(a, s < a.n ? s : a.n - 1);
    if (s < a.n && (!B || (s - V.soff < V.n && !V.ctrl->terminated))) {
        T xi = a.srt.x[s], yi = a.srt.y[s];
        int ocls = a.srt.cls[s];
        T h = (T)V.gh[a.cell[s]];
        T pnx = xi + (T)Y[2 * (size_t)s] * h, pny = yi + (T)Y[2 * (size_t)s + 1] * h;
        T fx, fy;
        int ncls;
        treat_move<T>(V, xi, yi, ocls, pnx, pny, (T)jump * (T)V.P.fac_pt * h, fx, fy, ncls, tcap, nfail);
        T mx = fx - xi, my = fy - yi;
        T mv = sqrt(mx * mx + my * my), cap = (T)V.P.fac_pt * h;
        a.cur.x[s] = fx;
        a.cur.y[s] = fy;
        a.cur.id[s] = a.srt.id[s];
        a.cur.cls[s] = (uint8_t)ncls;
        a.cur.dprev[s] = mv < cap ? mv : cap;
    }
    unsigned m = __ballot_sync(0xffffffffu, nfail != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.newton_fail, (unsigned long long)__popc(m));
    m = __ballot_sync(0xffffffffu, tcap != 0);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&V.ctrl->cnt.trace_cap, (unsigned long long)__popc(m));
}

template <typename T>
void launch_propose(const IterArgs<T>& a, const float* Y, float jump, cudaStream_t st) {
    int g = (a.n + kThreads - 1) / kThreads;
    if (g <= 0) return;
    if (a.Vs) k_propose<T, true><<<g, kThreads, 0, st>>>(a, Y, jump);
    else k_propose<T, false><<<g, kThreads, 0, st>>>(a, Y, jump);
}
template void launch_propose<double>(const IterArgs<double>&, const float*, float, cudaStream_t);
template void launch_propose<float>(const IterArgs<float>&, const float*, float, cudaStream_t);

template <typename T>
__global__ void k_targets(const __grid_constant__ IterArgs<T> a, const T* px, const T* py, const float* H,
                          float* Tout) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n) return;
    int id = a.cur.id[s];
    double h = (double)H[id];
    Tout[2 * (size_t)id] = (float)(((double)a.cur.x[s] - (double)px[id]) / h);
    Tout[2 * (size_t)id + 1] = (float)(((double)a.cur.y[s] - (double)py[id]) / h);
}

template <typename T>
void launch_targets(const IterArgs<T>& a, const T* px, const T* py, const float* H, float* Tout, cudaStream_t st) {
    int g = (a.n + kThreads - 1) / kThreads;
    if (g > 0) k_targets<T><<<g, kThreads, 0, st>>>(a, px, py, H, Tout);
}
template void launch_targets<double>(const IterArgs<double>&, const double*, const double*, const float*, float*,
                                     cudaStream_t);
template void launch_targets<float>(const IterArgs<float>&, const float*, const float*, const float*, float*,
                                    cudaStream_t);
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

// ------------------------------------------------------------------ model handle
struct mlp_s {
    float *p = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    float* gpart = nullptr;  // [kGradParts][kMlpParams] per-CTA gradient slots
    uint16_t *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
    double* loss = nullptr;
    int* err = nullptr;
    int32_t* perm = nullptr;
    int64_t perm_cap = 0;
    void* stage = nullptr;  // host-input staging
    size_t stage_cap = 0;
    int64_t t = 0;          // Adam steps taken
    cudaStream_t user = nullptr, st = nullptr;
    cudaEvent_t ev = nullptr;
};

namespace trime {
MlpDev mlp_view(const mlp_s* m) { return MlpDev{m->p, m->w1, m->w2, m->w3}; }
int* mlp_err(mlp_s* m) { return m->err; }
}  // namespace trime

#define MLP_TRY(x)                                                                                    \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) return set_error(TRIME_ECUDA, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
    } while (0)

static bool dev_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int mlp_sync_in(mlp_t* m) {
    MLP_TRY(cudaEventRecord(m->ev, m->user));
    MLP_TRY(cudaStreamWaitEvent(m->st, m->ev, 0));
    return 0;
}
static int mlp_sync_out(mlp_t* m) {
    MLP_TRY(cudaEventRecord(m->ev, m->st));
    MLP_TRY(cudaStreamWaitEvent(m->user, m->ev, 0));
    return 0;
}

static int mlp_stage(mlp_t* m, size_t bytes) {
    if (bytes <= m->stage_cap) return 0;
    cudaFree(m->stage);
    m->stage = nullptr;
    m->stage_cap = 0;
    if (cudaMalloc(&m->stage, bytes) != cudaSuccess) return set_error(TRIME_ENOMEM, "cudaMalloc failed");
    m->stage_cap = bytes;
    return 0;
}

static int mlp_check_err(mlp_t* m) {
    int h = 0;
    MLP_TRY(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->st));
    MLP_TRY(cudaStreamSynchronize(m->st));
    if (h) {
        cudaMemsetAsync(m->err, 0, sizeof(int), m->st);
        return set_error(TRIME_ETIMEOUT, "tensor-core wait ran out");
    }
    return 0;
}

static int mlp_upload(mlp_t* m, const float* params) {
    MLP_TRY(cudaMemcpyAsync(m->p, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, m->st));
    k_mlp_refresh<<<(kMlpOutPad * kMlpHid > kMlpParams ? kMlpOutPad * kMlpHid : kMlpParams + 255) / 256, 256, 0,
                    m->st>>>(m->p, m->w1, m->w2, m->w3);
    MLP_TRY(cudaGetLastError());
    MLP_TRY(cudaMemsetAsync(m->m, 0, sizeof(float) * kMlpParams, m->st));
    MLP_TRY(cudaMemsetAsync(m->v, 0, sizeof(float) * kMlpParams, m->st));
    MLP_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpParams, m->st));
    MLP_TRY(cudaStreamSynchronize(m->st));
    m->t = 0;
    return 0;
}

extern "C" {

void mlp_destroy(mlp_t* m) {
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    for (void* q : {(void*)m->p, (void*)m->grad, (void*)m->gpart, (void*)m->m, (void*)m->v, (void*)m->w1, (void*)m->w2, (void*)m->w3,
                    (void*)m->loss, (void*)m->err, (void*)m->perm, m->stage})
        cudaFree(q);
    if (m->ev) cudaEventDestroy(m->ev);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
}

int mlp_create(mlp_t** out, const float* params, uint64_t seed, void* cuda_stream) {
    if (!out) return set_error(TRIME_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<float> init;
    if (!params) {
        // He initialisation for the ReLU layers, a small output layer, zero biases
        std::mt19937_64 rng(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        init.assign(kMlpParams, 0.f);
        for (int u = 0; u < kMlpHid; u++)
            for (int f = 0; f < kMlpFeat; f++) init[kOW1 + u * kMlpIn + f] = (float)(nd(rng) * std::sqrt(2.0 / kMlpFeat));
        for (int i = 0; i < kMlpHid * kMlpHid; i++) init[kOW2 + i] = (float)(nd(rng) * std::sqrt(2.0 / kMlpHid));
        for (int i = 0; i < kMlpOut * kMlpHid; i++) init[kOW3 + i] = (float)(nd(rng) * 0.1 / std::sqrt((double)kMlpHid));
        params = init.data();
    }
    for (int k = 0; k < kMlpParams; k++)
        if (!std::isfinite(params[k])) return set_error(TRIME_EINVAL, "parameters must be finite");
    mlp_t* m = new mlp_s();
    m->user = (cudaStream_t)cuda_stream;
    bool ok = cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&m->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&m->p, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->grad, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->gpart, sizeof(float) * kMlpParams * kGradParts) == cudaSuccess &&
              cudaMalloc(&m->m, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->v, sizeof(float) * kMlpParams) == cudaSuccess &&
              cudaMalloc(&m->w1, 2 * kMlpHid * kMlpIn) == cudaSuccess &&
              cudaMalloc(&m->w2, 2 * kMlpHid * kMlpHid) == cudaSuccess &&
              cudaMalloc(&m->w3, 2 * kMlpOutPad * kMlpHid) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(double)) == cudaSuccess && cudaMalloc(&m->err, sizeof(int)) == cudaSuccess &&
              cudaMemset(m->w1, 0, 2 * kMlpHid * kMlpIn) == cudaSuccess &&
              cudaMemset(m->w3, 0, 2 * kMlpOutPad * kMlpHid) == cudaSuccess &&
              cudaMemset(m->err, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        mlp_destroy(m);
        return set_error(TRIME_ENOMEM, "device allocation failed");
    }
    int rc = mlp_upload(m, params);
    if (rc) {
        mlp_destroy(m);
        return rc;
    }
    *out = m;
    return TRIME_OK;
}

int mlp_set_params(mlp_t* m, const float* params) {
    if (!m || !params) return set_error(TRIME_EINVAL, "NULL argument");
    for (int k = 0; k < kMlpParams; k++)
        if (!std::isfinite(params[k])) return set_error(TRIME_EINVAL, "parameters must be finite");
    int rc = mlp_sync_in(m);
    if (rc) return rc;
    if ((rc = mlp_upload(m, params))) return rc;
    return mlp_sync_out(m);
}

int mlp_get_params(mlp_t* m, float* params) {
    if (!m || !params) return set_error(TRIME_EINVAL, "NULL argument");
    int rc = mlp_sync_in(m);
    if (rc) return rc;
    MLP_TRY(cudaMemcpyAsync(params, m->p, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->st));
    MLP_TRY(cudaStreamSynchronize(m->st));
    return mlp_sync_out(m);
}

int mlp_forward(mlp_t* m, const uint16_t* X, int64_t n, float* Y) {
    if (!m) return set_error(TRIME_EINVAL, "model is NULL");
    if (n < 0 || n > (int64_t)1 << 30) return set_error(TRIME_EINVAL, "n out of range");
    if (n == 0) return TRIME_OK;
    if (!X || !Y) return set_error(TRIME_EINVAL, "NULL pointer");
    bool dx = dev_ptr(X), dy = dev_ptr(Y);
    int rc = mlp_sync_in(m);
    if (rc) return rc;
    size_t bx = (size_t)n * kMlpIn * 2, by = (size_t)n * 2 * sizeof(float);
    if ((rc = mlp_stage(m, (dx ? 0 : bx) + (dy ? 0 : by)))) return rc;
    const uint16_t* xs = X;
    float* ys = Y;
    if (!dx) {
        MLP_TRY(cudaMemcpyAsync(m->stage, X, bx, cudaMemcpyHostToDevice, m->st));
        xs = (const uint16_t*)m->stage;
    }
    if (!dy) ys = (float*)((char*)m->stage + (dx ? 0 : bx));
    launch_mlp_forward(mlp_view(m), xs, nullptr, (int)n, ys, m->err, m->st);
    MLP_TRY(cudaGetLastError());
    if (!dy) MLP_TRY(cudaMemcpyAsync(Y, ys, by, cudaMemcpyDeviceToHost, m->st));
    if ((rc = mlp_check_err(m))) return rc;
    return mlp_sync_out(m);
}

int mlp_loss_grad(mlp_t* m, const uint16_t* X, const float* T, int64_t n, double* loss, float* grad) {
    if (!m) return set_error(TRIME_EINVAL, "model is NULL");
    if (n <= 0 || n > (int64_t)1 << 30) return set_error(TRIME_EINVAL, "n out of range");
    if (!X || !T || !loss || !grad) return set_error(TRIME_EINVAL, "NULL pointer");
    bool dx = dev_ptr(X), dt = dev_ptr(T);
    int rc = mlp_sync_in(m);
    if (rc) return rc;
    size_t bx = (size_t)n * kMlpIn * 2, bt = (size_t)n * 2 * sizeof(float);
    if ((rc = mlp_stage(m, (dx ? 0 : bx) + (dt ? 0 : bt)))) return rc;
    const uint16_t* xs = X;
    const float* ts = T;
    if (!dx) {
        MLP_TRY(cudaMemcpyAsync(m->stage, X, bx, cudaMemcpyHostToDevice, m->st));
        xs = (const uint16_t*)m->stage;
    }
    if (!dt) {
        float* tt = (float*)((char*)m->stage + (dx ? 0 : bx));
        MLP_TRY(cudaMemcpyAsync(tt, T, bt, cudaMemcpyHostToDevice, m->st));
        ts = tt;
    }
    MLP_TRY(cudaMemsetAsync(m->loss, 0, sizeof(double), m->st));
    int parts = launch_mlp_grad(mlp_view(m), xs, ts, nullptr, (int)n, 1.0f / (float)n, m->gpart, m->loss, m->err,
                                m->st);
    k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, m->st>>>(m->gpart, parts, m->grad);
    MLP_TRY(cudaGetLastError());
    MLP_TRY(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, m->st));
    MLP_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    if ((rc = mlp_check_err(m))) return rc;
    return mlp_sync_out(m);
}

int mlp_train(mlp_t* m, const uint16_t* X, const float* T, int64_t n, int32_t epochs, int32_t batch, double lr,
              uint64_t seed, double* last_loss) {
    if (!m) return set_error(TRIME_EINVAL, "model is NULL");
    if (n <= 0 || n > (int64_t)1 << 30 || epochs < 0 || batch < 128 || !(lr > 0))
        return set_error(TRIME_EINVAL, "bad n / epochs / batch (>= 128) / lr");
    if (!X || !T || !dev_ptr(X) || !dev_ptr(T)) return set_error(TRIME_EINVAL, "X and T must be device arrays");
    int rc = mlp_sync_in(m);
    if (rc) return rc;
    if (m->perm_cap < n) {
        cudaFree(m->perm);
        m->perm = nullptr;
        m->perm_cap = 0;
        if (cudaMalloc(&m->perm, sizeof(int32_t) * (size_t)n) != cudaSuccess)
            return set_error(TRIME_ENOMEM, "cudaMalloc failed");
        m->perm_cap = n;
    }
    std::vector<int32_t> perm((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[(size_t)i] = (int32_t)i;
    std::mt19937_64 rng(seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double ep_loss = 0.0;
    for (int e = 0; e < epochs; e++) {
        for (int64_t i = n - 1; i > 0; i--) std::swap(perm[(size_t)i], perm[(size_t)(rng() % (uint64_t)(i + 1))]);
        MLP_TRY(cudaMemcpyAsync(m->perm, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, m->st));
        MLP_TRY(cudaMemsetAsync(m->loss, 0, sizeof(double), m->st));
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            int cnt = (int)std::min<int64_t>(batch, n - b0);
            int parts = launch_mlp_grad(mlp_view(m), X, T, m->perm + b0, cnt, 1.0f / (float)cnt, m->gpart, m->loss,
                                        m->err, m->st);
            m->t++;
            float c1 = (float)(1.0 - std::pow((double)b1, (double)m->t));
            float c2 = (float)(1.0 - std::pow((double)b2, (double)m->t));
            k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, m->st>>>(m->p, m->gpart, parts, m->m, m->v, m->w1, m->w2,
                                                                     m->w3, (float)lr, b1, b2, eps, c1, c2);
            nb++;
        }
        MLP_TRY(cudaGetLastError());
        double l = 0;
        MLP_TRY(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
        if ((rc = mlp_check_err(m))) return rc;  // synchronises
        ep_loss = l / (double)nb;
    }
    if (last_loss) *last_loss = ep_loss;
    return mlp_sync_out(m);
}

}  // extern "C"
