// tc.cuh -- 5th-generation tensor-core primitives (tcgen05) for sm_103a.
//
// One CTA of 128 threads (4 warps) computes D (128 x N, FP32, in tensor
// memory) += A (128 x K, BF16) * B^T (B is N x K, BF16), both operands in
// shared memory in the K-major layout without swizzling: the operand is cut
// into core matrices of 8 rows x 8 elements (16 bytes per row, 128 bytes per
// core matrix); core matrix (rb, kb) of an R x K operand starts at byte
// ((rb * K / 8) + kb) * 128, so core matrices adjacent along K are 128 bytes
// apart (the descriptor's leading byte offset) and 8-row groups are K * 16
// bytes apart (its stride byte offset).  One MMA instruction consumes K = 16
// (two core matrices along K).  Row i of D lives in tensor-memory lane i,
// column j in column base + j; warp w reads lanes 32w .. 32w + 31.
//
// Every wait is bounded: a wait that runs out sets the caller's error flag
// and the kernel still releases its tensor memory before returning.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace trime {
namespace tc {

constexpr int kTcThreads = 128;
constexpr long long kSpinLimit = 1ll << 26;  // about a second of polling

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) in the K-major core-matrix layout of an R x K operand
__host__ __device__ __forceinline__ uint32_t kmajor_offset(int r, int k, int K) {
    return (uint32_t)((((r >> 3) * (K >> 3)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading byte offset (K
// direction), stride byte offset (M/N direction), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // version
    return d;                // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 accumulator, both
// operands K-major, M = 128, N given
__host__ __device__ constexpr uint32_t make_idesc_bf16(int N) {
    return (1u << 4)                       // D format F32
           | (1u << 7)                     // A format BF16
           | (1u << 10)                    // B format BF16
           | ((uint32_t)(N >> 3) << 17)    // N / 8
           | ((uint32_t)(128 >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// waits for the phase with the given parity; false if the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kSpinLimit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// tensor-memory allocation by one whole warp; the address lands in *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes become visible to the tensor cores
__device__ __forceinline__ void fence_smem_to_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A * B^T, one instruction (K = 16); issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// arrive on the mbarrier once every MMA issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

// The whole 128 x N x K product on operands staged in shared memory.  Issued
// by thread 0; `bar` completes one phase when it is done.
__device__ __forceinline__ void gemm_issue(uint32_t d_tmem, const void* A, const void* B, int N, int K,
                                           bool accumulate, uint64_t* bar) {
    uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    uint32_t idesc = make_idesc_bf16(N);
    uint32_t sbo = (uint32_t)K * 16;  // 8 rows x K elements x 2 bytes
    for (int k = 0; k < K; k += 16) {
        uint32_t off = (uint32_t)(k >> 3) * 128;
        mma_bf16(d_tmem, make_sdesc(a0 + off, 128, sbo), make_sdesc(b0 + off, 128, sbo), idesc,
                 accumulate || k > 0);
    }
    mma_commit(bar);
}

}  // namespace tc
}  // namespace trime
