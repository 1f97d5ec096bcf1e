// BF16 GEMM on the 5th-generation tensor cores (tcgen05), FP32 accumulation
// in tensor memory (TMEM):
//   C[m][n] (+)= sum_k A[m][k] * B[n][k]      (A, B bf16 row-major, K contiguous)
// in 128 x BN output tiles and K steps of 64.  Two kernels (tc_gemm.cu):
//  * TMA-fed and warp-specialised (most shapes): 2-D tensor-map tile loads with
//    the 128-byte swizzle fill an S-stage shared-memory ring; one lane issues
//    the loads and the tcgen05.mma (K = 16 each), four warps read the two TMEM
//    accumulators with tcgen05.ld for the epilogue of one tile while the next
//    one accumulates; persistent CTAs stride over the M tiles.
//  * cp.async-fed (one or two K steps at 64- or 128-column blocks): all threads
//    copy 16-byte chunks into the K-major core-matrix layout (8 rows x 16 bytes
//    per core matrix, no swizzle), one CTA per M tile.
// Optional split-K (gridDim.z > 1) adds partial tiles atomically or stores
// each K chunk's partial tile in its own slice; otherwise the epilogue adds a
// bias, applies ReLU, and writes FP32 and/or BF16.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace gsp {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices adjacent in K), stride-dimension byte offset
// (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major,
// shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(dst_smem), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_init1(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after `budget` SM clocks.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long budget) {
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (clock64() - t0 > budget) return false;
    }
}

}  // namespace tc

// Launch C (+)= A * B^T on stream s.  A: [M][lda], B: [N][ldb] bf16 with
// lda, ldb multiples of 8 and columns K..round8(K) zero (16-byte rows);
// C: [M][ldc] float (optional), Cb: [M][ldcb] bf16 (optional).  splitk > 1
// with zstride = 0: C must be zeroed and receives atomic partial sums (no
// bias, ReLU or Cb).  splitk > 1 with zstride >= M * ldc: the partial product
// of K chunk z is stored (not added) into C + z * zstride, for a reduction in a
// fixed order by the caller (no bias, ReLU or Cb); *nsplit (optional) receives
// the number of chunks used.  bias: [N] float or null; relu: apply max(0, .)
// after the bias.  err: set to 1 if a bounded wait gave up.  Returns the
// launch error.
cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                             int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb,
                             int64_t ldcb, int M, int N, int K, const float *bias, bool relu,
                             int splitk, int *err, cudaStream_t s, int64_t zstride = 0,
                             int *nsplit = nullptr, bool dependent = false);

}  // namespace gsp
