// tcgen05 BF16 GEMM (see tc_gemm.cuh) and its C-ABI entry point.
#include <algorithm>

#include <cuda.h>

#include "gsp_internal.cuh"
#include "tc_gemm.cuh"

namespace gsp {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr long long kGemmBudget = 2000000000ll;  // ~1 s of SM clock per wait

__device__ int g_gemm_err;  // fallback error flag when the caller passes none

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The 16-byte copies of one ROWS x 64 bf16 tile of a K-contiguous matrix into
// the core-matrix layout (element (r, c) at byte (r/8)*1024 + (c/8)*128 +
// (r%8)*16 + (c%8)*2).  Thread t copies column chunk t % 8 of rows t / 8 + 16 i,
// so the 8 lanes of a row read its 128 contiguous bytes and a warp instruction
// reads 4 whole rows (coalesced).  Only the first nc8 chunks are copied (the
// ones the MMAs of this K step read); rows >= nrows and columns >= kend are
// zero-filled (kend is a multiple of 8).
template <int ROWS>
struct TileCopy {
    static_assert(ROWS % 16 == 0, "16 rows per pass of 128 threads");
    int c8, r0;
    __device__ __forceinline__ TileCopy() : c8(threadIdx.x & 7), r0(threadIdx.x >> 3) {}
    __device__ __forceinline__ void issue(uint32_t dst, const __nv_bfloat16 *__restrict__ src,
                                          int64_t ld, int row0, int nrows, int k0, int kend,
                                          int nc8) const {
        if (c8 >= nc8) return;
        const int gk = k0 + c8 * 8;
        const bool kin = gk < kend;
#pragma unroll
        for (int i = 0; i < ROWS / 16; i++) {
            const int r = r0 + 16 * i;
            const int gr = row0 + r;
            const bool in = kin && gr < nrows;
            const __nv_bfloat16 *g = in ? src + (int64_t)gr * ld + gk : src;
            cp_async16(dst + (uint32_t)((r >> 3) * 1024 + c8 * 128 + (r & 7) * 16), g,
                       in ? 16u : 0u);
        }
    }
};

// C (+)= A B^T, one 128 x BN output column block per CTA row of the grid
// (blockIdx.y), a K chunk per blockIdx.z (split-K).  The CTA's (M tile,
// 64-wide K step) pairs form one sequence that flows through a ring of S
// shared-memory stages: all 128 threads copy stage j + S - 1 (cp.async) while
// thread 0's MMAs of stage j run, and a stage is refilled only after the MMAs
// that read it have completed (one mbarrier per stage, signalled by
// tcgen05.commit).  NACC = 2: CTAs stride over the M tiles and the
// accumulator alternates between two TMEM column blocks, so the epilogue of
// tile t (tcgen05.ld by all four warps, bias, ReLU, stores or split-K
// atomics) runs while the MMAs of tile t + 1 accumulate into the other block.
// NACC = 1: one M tile per CTA (short K: many small CTAs per SM hide the
// latency instead).  Every wait is bounded; a wait that gives up sets *err,
// and the CTA waits (bounded) for its committed MMAs and its copies before it
// frees tensor memory.
template <int BN, int S, int NACC>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(
    const __nv_bfloat16 *__restrict__ A, int64_t lda, const __nv_bfloat16 *__restrict__ B,
    int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K,
    int kchunk, int64_t zstride, const float *__restrict__ bias, int relu, int *err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tcgen05 M=128 with N in 16..128");
    static_assert(S >= 1 && (NACC == 1 || NACC == 2), "ring depth and accumulators");
    static_assert(S >= 2 || NACC == 1, "a single stage serves one tile per CTA");
    constexpr int kAhead = S > 1 ? S - 1 : 1;  // entries copied ahead of the one in use
    constexpr int kWait = S > 1 ? S - 2 : 0;   // copy groups that may still be pending
    constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
    constexpr int kStageBytes = kABytes + kBBytes;
    constexpr uint32_t kCols = NACC * BN < 32 ? 32u : (uint32_t)(NACC * BN);
    constexpr uint32_t kIdesc = tc::idesc_bf16(kBM, BN);
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_stage[S];
    __shared__ __align__(8) uint64_t bar_acc[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int mtiles = (M + kBM - 1) / kBM;
    const int nks = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;  // K steps per tile
    const int ntile_mine = (int)blockIdx.x >= mtiles ? 0
                           : (NACC == 1 ? 1 : (mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1);
    const int total = ntile_mine * nks;                                   // sequence length
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), kCols);
    if (tid == 0) {
        for (int i = 0; i < S; i++) tc::mbar_init1(tc::smem_u32(&bar_stage[i]));
        for (int i = 0; i < 2; i++) tc::mbar_init1(tc::smem_u32(&bar_acc[i]));
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t sbase = tc::smem_u32(smem);
    const TileCopy<kBM> copyA;
    const TileCopy<BN> copyB;
    auto load = [&](int j) {  // copies of sequence entry j into stage j % S
        if (j < total) {
            const int lt = j / nks, ks = j - lt * nks;
            const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kBM;
            const int k0 = kbeg + ks * kBK;
            const int nc8 = 2 * ((min(kBK, kend - k0) + 15) / 16);  // chunks the MMAs read
            const uint32_t st = sbase + (uint32_t)((j % S) * kStageBytes);
            copyA.issue(st, A, lda, m0, M, k0, kend, nc8);
            copyB.issue(st + kABytes, B, ldb, n0, N, k0, kend, nc8);
        }
        cp_async_commit();  // one group per entry, empty past the end
    };
    // 16-byte float stores (8-byte bf16 stores) when every row start is aligned
    const bool vec_ok = ((ldc & 3) == 0) && (((uintptr_t)C & 15) == 0) && ((ldcb & 3) == 0) &&
                        (((uintptr_t)Cb & 7) == 0);
    auto epilogue = [&](int lt) {
        const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kBM;
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr =
            tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((NACC == 2 ? (lt & 1) : 0) * BN);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (row < M) {
                if (gridDim.z > 1 && zstride > 0) {
                    // this K chunk's partial product into its own slice of C
                    float *cz = C + (int64_t)blockIdx.z * zstride + (int64_t)row * ldc + n0 + c0;
#pragma unroll
                    for (int jj = 0; jj < 16; jj++)
                        if (n0 + c0 + jj < N) cz[jj] = v[jj];
                } else if (gridDim.z > 1) {
#pragma unroll
                    for (int jj = 0; jj < 16; jj++)
                        if (n0 + c0 + jj < N) atomicAdd(C + (int64_t)row * ldc + n0 + c0 + jj, v[jj]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; q++) {  // groups of four columns
                        const int n = n0 + c0 + 4 * q;
                        float w[4];
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            float val = v[4 * q + e];
                            if (bias && n + e < N) val += bias[n + e];
                            if (relu) val = fmaxf(val, 0.0f);
                            w[e] = val;
                        }
                        if (n + 4 <= N && vec_ok) {
                            if (C)
                                *reinterpret_cast<float4 *>(C + (int64_t)row * ldc + n) =
                                    make_float4(w[0], w[1], w[2], w[3]);
                            if (Cb) {
                                __nv_bfloat162 lo = __floats2bfloat162_rn(w[0], w[1]);
                                __nv_bfloat162 hi = __floats2bfloat162_rn(w[2], w[3]);
                                uint2 pk;
                                pk.x = *reinterpret_cast<uint32_t *>(&lo);
                                pk.y = *reinterpret_cast<uint32_t *>(&hi);
                                *reinterpret_cast<uint2 *>(Cb + (int64_t)row * ldcb + n) = pk;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                if (n + e < N) {
                                    if (C) C[(int64_t)row * ldc + n + e] = w[e];
                                    if (Cb) Cb[(int64_t)row * ldcb + n + e] = __float2bfloat16_rn(w[e]);
                                }
                            }
                        }
                    }
                }
            }
        }
    };
    bool ok = true;
    int committed = 0;  // stage mbarrier phases committed by thread 0 (MMAs issued)
    for (int j = 0; j < kAhead; j++) load(j);
    for (int j = 0; j < total && ok; j++) {
        const int lt = j / nks, ks = j - lt * nks;
        cp_async_wait<kWait>();   // this thread's copies of entry j have landed
        tc::fence_proxy_async();  // ... and are visible to the tensor cores
        tc::fence_before();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            const int k0 = kbeg + ks * kBK;
            const int nmma = (min(kBK, kend - k0) + 15) / 16;  // K = 16 per MMA
            const uint32_t st = sbase + (uint32_t)((j % S) * kStageBytes);
            const uint32_t acc = tmem + (uint32_t)((NACC == 2 ? (lt & 1) : 0) * BN);
            for (int kk = 0; kk < nmma; kk++) {
                // two core matrices along K (256 bytes) per MMA
                const uint64_t ad = tc::smem_desc(st + kk * 256, 128, 1024);
                const uint64_t bd = tc::smem_desc(st + kABytes + kk * 256, 128, 1024);
                tc::mma_bf16(acc, ad, bd, kIdesc, (ks > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(tc::smem_u32(&bar_stage[j % S]));
            if (ks == nks - 1) tc::mma_commit(tc::smem_u32(&bar_acc[lt & 1]));
        }
        committed = j + 1;
        // entry j + kAhead goes into the stage of entry j + kAhead - S, once that
        // entry's MMAs are done (nothing to refill near the end of the sequence)
        const int nxt = j + kAhead, jp = nxt - S;
        if (jp >= 0 && nxt < total) {
            const bool done = tc::mbar_wait_bounded(tc::smem_u32(&bar_stage[jp % S]),
                                                    (uint32_t)((jp / S) & 1), kGemmBudget);
            if (!__all_sync(0xffffffffu, done)) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        load(nxt);
        // the previous tile's epilogue, while this tile's MMAs run
        if (NACC == 2 && ks == 0 && lt > 0) {
            const bool done = tc::mbar_wait_bounded(tc::smem_u32(&bar_acc[(lt - 1) & 1]),
                                                    (uint32_t)(((lt - 1) >> 1) & 1), kGemmBudget);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
            tc::fence_after();
            epilogue(lt - 1);
        }
    }
    if (ok && ntile_mine > 0 && nks > 0) {
        const int lt = ntile_mine - 1;
        const bool done = tc::mbar_wait_bounded(tc::smem_u32(&bar_acc[lt & 1]),
                                                (uint32_t)((lt >> 1) & 1), kGemmBudget);
        if (__syncthreads_and(done)) {
            tc::fence_after();
            epilogue(lt);
        } else {
            ok = false;
        }
    }
    cp_async_wait<0>();  // no copy in flight into shared memory when the CTA ends
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // never release tensor memory under MMAs still in flight (bounded): the
        // last committed stage barrier completes after every earlier MMA
        if (committed > 0) {
            const int jl = committed - 1;
            (void)tc::mbar_wait_bounded(tc::smem_u32(&bar_stage[jl % S]),
                                        (uint32_t)((jl / S) & 1), kGemmBudget);
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// ------------------------------------------------ TMA-fed, warp-specialised GEMM
// Long K (three or more 64-wide steps per CTA): 2-D TMA tile loads with the
// 128-byte swizzle feed an S-stage shared-memory ring (full / empty mbarriers
// per stage); warp 4's lane 0 issues the loads and the tcgen05.mma (K = 16
// each), committing each stage to its empty barrier and each finished M tile
// to an accumulator barrier; warps 0-3 (TMEM lanes 0-127) run the epilogue of
// a tile while the MMAs of the next one accumulate into the other of two TMEM
// accumulators, and release it on a second barrier.  The K-loop costs the
// other 127 threads nothing.  Every wait is bounded; a wait that gives up sets
// *err, and the issuing lane first waits (bounded) for the loads it issued.

__device__ __forceinline__ void mbar_init_n(uint32_t bar, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive1(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// 2-D tile of a tensor map into shared memory, coordinates {k, row} in
// elements, completion counted on bar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *tm, int k, int row,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(k), "r"(row), "r"(bar)
        : "memory");
}
// Shared-memory descriptor of a K-major tile written by TMA with the 128-byte
// swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte
// offset), descriptor version 1, swizzle mode 2 (128 bytes); the leading byte
// offset is not used by swizzled K-major layouts.  A K = 16 slice of the atom
// starts 32 bytes further.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// The epilogue of one 128 x BN tile for this thread's row (TMEM lane): bias,
// ReLU and FP32 / bf16 stores; with split-K, the partial sums as atomics
// (zstride 0) or into the K chunk's own slice of C.
template <int BN>
__device__ __forceinline__ void store_tile(uint32_t lane_addr, int row, int n0, int M, int N,
                                           float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb,
                                           const float *__restrict__ bias, int relu, bool split,
                                           int64_t zstride, bool vec_ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
        if (row >= M) continue;
        if (split && zstride > 0) {
            float *cz = C + (int64_t)blockIdx.z * zstride + (int64_t)row * ldc + n0 + c0;
#pragma unroll
            for (int jj = 0; jj < 16; jj++)
                if (n0 + c0 + jj < N) cz[jj] = v[jj];
        } else if (split) {
#pragma unroll
            for (int jj = 0; jj < 16; jj++)
                if (n0 + c0 + jj < N) atomicAdd(C + (int64_t)row * ldc + n0 + c0 + jj, v[jj]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int n = n0 + c0 + 4 * q;
                float w[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    float val = v[4 * q + e];
                    if (bias && n + e < N) val += bias[n + e];
                    if (relu) val = fmaxf(val, 0.0f);
                    w[e] = val;
                }
                if (n + 4 <= N && vec_ok) {
                    if (C)
                        *reinterpret_cast<float4 *>(C + (int64_t)row * ldc + n) =
                            make_float4(w[0], w[1], w[2], w[3]);
                    if (Cb) {
                        __nv_bfloat162 lo = __floats2bfloat162_rn(w[0], w[1]);
                        __nv_bfloat162 hi = __floats2bfloat162_rn(w[2], w[3]);
                        uint2 pk;
                        pk.x = *reinterpret_cast<uint32_t *>(&lo);
                        pk.y = *reinterpret_cast<uint32_t *>(&hi);
                        *reinterpret_cast<uint2 *>(Cb + (int64_t)row * ldcb + n) = pk;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        if (n + e < N) {
                            if (C) C[(int64_t)row * ldc + n + e] = w[e];
                            if (Cb) Cb[(int64_t)row * ldcb + n + e] = __float2bfloat16_rn(w[e]);
                        }
                    }
                }
            }
        }
    }
}

template <int BN, int S>
__global__ void __launch_bounds__(160) gemm_tma_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float *C,
    int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K, int kchunk,
    int64_t zstride, const float *__restrict__ bias, int relu, int *err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tcgen05 M=128 with N in 16..128");
    constexpr int kABytes = kBM * 128, kBBytes = BN * 128;  // 64 bf16 of K per row
    constexpr int kStageBytes = kABytes + kBBytes;          // a multiple of 1024
    constexpr uint32_t kCols = 2 * BN < 32 ? 32u : (uint32_t)(2 * BN);
    constexpr uint32_t kIdesc = tc::idesc_bf16(kBM, BN);
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (tc::smem_u32(smem_raw) + 1023u) & ~1023u;  // swizzle atoms: 1024 B
    const int n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int mtiles = (M + kBM - 1) / kBM;
    const int nks = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;
    const int ntile_mine =
        (int)blockIdx.x >= mtiles ? 0 : (mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
    const int total = ntile_mine * nks;
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), kCols);
    if (tid == 0) {
        for (int i = 0; i < S; i++) {
            mbar_init_n(tc::smem_u32(&full[i]), 1);
            mbar_init_n(tc::smem_u32(&empty[i]), 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init_n(tc::smem_u32(&accf[i]), 1);
            mbar_init_n(tc::smem_u32(&acce[i]), 4);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    wait_prior_grid();  // the operands may come from the kernel launched just before
    const uint32_t tmem = tmem_base;
    bool ok = true;
    if (warp == 4) {
        if (lane == 0 && total > 0) {
            auto stage_addr = [&](int j) { return sbase + (uint32_t)((j % S) * kStageBytes); };
            auto issue = [&](int j) {  // the loads of sequence entry j into stage j % S
                const int lt = j / nks, ks = j - lt * nks;
                const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kBM;
                const uint32_t st = stage_addr(j), fb = tc::smem_u32(&full[j % S]);
                mbar_expect_tx(fb, (uint32_t)kStageBytes);
                tma_load_2d(st, &tmA, kbeg + ks * kBK, m0, fb);
                tma_load_2d(st + kABytes, &tmB, kbeg + ks * kBK, n0, fb);
            };
            int issued = 0, consumed = 0;  // entries whose loads were issued / waited for
            for (; issued < min(S, total); issued++) issue(issued);
            for (int j = 0; j < total; j++) {
                const int lt = j / nks, ks = j - lt * nks;
                // accumulator lt & 1 is free once the epilogue of tile lt - 2 released it
                if (ks == 0 && lt >= 2 &&
                    !tc::mbar_wait_bounded(tc::smem_u32(&acce[lt & 1]),
                                           (uint32_t)(((lt >> 1) - 1) & 1), kGemmBudget)) {
                    ok = false;
                    break;
                }
                if (!tc::mbar_wait_bounded(tc::smem_u32(&full[j % S]), (uint32_t)((j / S) & 1),
                                           kGemmBudget)) {
                    ok = false;
                    break;
                }
                consumed = j + 1;
                tc::fence_after();
                const int k0 = kbeg + ks * kBK;
                const int nmma = (min(kBK, kend - k0) + 15) / 16;  // K = 16 per MMA
                const uint32_t st = stage_addr(j);
                const uint32_t acc = tmem + (uint32_t)((lt & 1) * BN);
                for (int kk = 0; kk < nmma; kk++)
                    tc::mma_bf16(acc, smem_desc_sw128(st + kk * 32),
                                 smem_desc_sw128(st + kABytes + kk * 32), kIdesc,
                                 (ks > 0 || kk > 0) ? 1u : 0u);
                tc::mma_commit(tc::smem_u32(&empty[j % S]));
                if (ks == nks - 1) tc::mma_commit(tc::smem_u32(&accf[lt & 1]));
                // entry j - 1 + S into the stage of entry j - 1, once its MMAs are done
                if (j >= 1 && issued < total) {
                    if (!tc::mbar_wait_bounded(tc::smem_u32(&empty[(j - 1) % S]),
                                               (uint32_t)(((j - 1) / S) & 1), kGemmBudget)) {
                        ok = false;
                        break;
                    }
                    issue(issued++);
                }
            }
            if (!ok) {
                atomicExch(err, 1);
                for (int j = consumed; j < issued; j++)  // loads issued but not waited for
                    (void)tc::mbar_wait_bounded(tc::smem_u32(&full[j % S]),
                                                (uint32_t)((j / S) & 1), kGemmBudget);
            }
            // every committed MMA done before tensor memory is released
            if (consumed > 0)
                (void)tc::mbar_wait_bounded(tc::smem_u32(&empty[(consumed - 1) % S]),
                                            (uint32_t)(((consumed - 1) / S) & 1), kGemmBudget);
        }
        __syncwarp();
    } else {
        const bool vec_ok = ((ldc & 3) == 0) && (((uintptr_t)C & 15) == 0) && ((ldcb & 3) == 0) &&
                            (((uintptr_t)Cb & 7) == 0);
        for (int lt = 0; lt < ntile_mine; lt++) {
            bool done = true;
            if (lane == 0)
                done = tc::mbar_wait_bounded(tc::smem_u32(&accf[lt & 1]), (uint32_t)((lt >> 1) & 1),
                                             kGemmBudget);
            if (!__shfl_sync(0xffffffffu, done, 0)) {
                ok = false;
                break;
            }
            tc::fence_after();
            const int m0 = ((int)blockIdx.x + lt * (int)gridDim.x) * kBM;
            const uint32_t lane_addr =
                tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((lt & 1) * BN);
            store_tile<BN>(lane_addr, m0 + warp * 32 + lane, n0, M, N, C, ldc, Cb, ldcb, bias, relu,
                           gridDim.z > 1, zstride, vec_ok);
            tc::fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(tc::smem_u32(&acce[lt & 1]));
        }
        if (!ok && lane == 0) atomicExch(err, 1);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of a row-major bf16 matrix [rows][ld] whose first k columns hold
// data: boxes of 64 columns x box_rows rows, 128-byte swizzle, zero fill
// outside [0, k) x [0, rows).
cudaError_t make_tmap(CUtensorMap *tm, const __nv_bfloat16 *base, int64_t rows, int64_t k,
                      int64_t ld, int box_rows) {
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                          cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                              const_cast<__nv_bfloat16 *>(base), gdim, gstride, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr int kTmaStages = 4;

template <int BN>
constexpr int tma_smem() {
    return kTmaStages * (kBM + BN) * kBK * 2 + 1024;  // + alignment slack for the 1024-B atoms
}

template <int BN>
cudaError_t launch_tma(dim3 grid, bool dependent, cudaStream_t s, const CUtensorMap &tmA,
                       const CUtensorMap &tmB,
                       float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K,
                       int kchunk, int64_t zstride, const float *bias, int relu, int *err) {
    constexpr int smem = tma_smem<BN>();
    cudaError_t e =
        ensure_kernel_smem(reinterpret_cast<const void *>(gemm_tma_kernel<BN, kTmaStages>), smem);
    if (e != cudaSuccess) return e;
    if (dependent)
        return launch_dependent(gemm_tma_kernel<BN, kTmaStages>, grid, dim3(160), (size_t)smem, s, tmA,
                                tmB, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, relu, err);
    gemm_tma_kernel<BN, kTmaStages><<<grid, 160, smem, s>>>(tmA, tmB, C, ldc, Cb, ldcb, M, N, K,
                                                            kchunk, zstride, bias, relu, err);
    return cudaSuccess;
}

// Launch one instantiation; its dynamic shared-memory limit (above the 48 KB
// default) is raised once per device.
template <int BN, int S, int NACC>
cudaError_t launch_bn(dim3 grid, cudaStream_t s, const __nv_bfloat16 *A, int64_t lda,
                      const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc,
                      __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K, int kchunk,
                      int64_t zstride, const float *bias, int relu, int *err) {
    constexpr int smem = S * (kBM + BN) * kBK * 2;
    cudaError_t e =
        ensure_kernel_smem(reinterpret_cast<const void *>(gemm_bf16_kernel<BN, S, NACC>), smem);
    if (e != cudaSuccess) return e;
    gemm_bf16_kernel<BN, S, NACC><<<grid, 128, smem, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N,
                                                          K, kchunk, zstride, bias, relu, err);
    return cudaSuccess;
}

// Short K (one or two 64-wide steps per tile) at 64- and 128-column blocks:
// the cp.async kernel with one CTA per M tile, one accumulator and one or two
// stages (small CTAs, many per SM, hide the latency).  Everything else: the
// TMA-fed warp-specialised kernel, a 4-stage ring, two accumulators, and
// persistent CTAs striding over the M tiles.
template <int BN>
cudaError_t launch_n(int ksteps, int mtiles, int ntiles, int splitk, int nsm, bool dependent,
                     cudaStream_t s,
                     const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                     float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K,
                     int kchunk, int64_t zstride, const float *bias, int relu, int *err) {
    // short K (one or two 64-wide steps) with wide column blocks: the cp.async
    // kernel, one CTA per M tile, many per SM; the persistent TMA kernel's 4
    // epilogue warps per SM (one CTA of 132 KB) cannot keep up with 128-column
    // output tiles there (72.6 vs 52.0 us for 262144 x 128 x 64), while at 16-
    // and 32-column blocks it is the faster one (36.5 vs 51.5 us at 16)
    if (ksteps <= 2 && BN >= 64) {
        dim3 grid((unsigned)mtiles, (unsigned)ntiles, (unsigned)splitk);
        if (ksteps == 1)
            return launch_bn<BN, 1, 1>(grid, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk,
                                       zstride, bias, relu, err);
        return launch_bn<BN, 2, 1>(grid, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk,
                                   zstride, bias, relu, err);
    }
    // longer K: the TMA-fed warp-specialised kernel, persistent CTAs over the M tiles
    constexpr int smem = tma_smem<BN>();
    const int per_sm = std::max(1, (227 * 1024) / (smem + 1024));
    const int64_t want = ((int64_t)nsm * per_sm + (int64_t)ntiles * splitk - 1) /
                         ((int64_t)ntiles * splitk);
    const int mgrid = (int)std::max<int64_t>(1, std::min<int64_t>(mtiles, want));
    dim3 grid((unsigned)mgrid, (unsigned)ntiles, (unsigned)splitk);
    CUtensorMap tmA, tmB;
    cudaError_t e = make_tmap(&tmA, A, M, K, lda, kBM);
    if (e == cudaSuccess) e = make_tmap(&tmB, B, N, K, ldb, BN);
    if (e != cudaSuccess) return e;
    return launch_tma<BN>(grid, dependent, s, tmA, tmB, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, relu,
                          err);
}

}  // namespace

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                             int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb,
                             int64_t ldcb, int M, int N, int K, const float *bias, bool relu,
                             int splitk, int *err, cudaStream_t s, int64_t zstride, int *nsplit,
                             bool dependent) {
    if (M <= 0 || N <= 0 || K <= 0 || (K & 7) || (lda & 7) || (ldb & 7) || lda < K || ldb < K ||
        (((uintptr_t)A | (uintptr_t)B) & 15) || (!C && !Cb) || (splitk > 1 && !C) ||
        zstride < 0 || (zstride > 0 && (!C || Cb || bias || relu || zstride < (int64_t)M * ldc)))
        return cudaErrorInvalidValue;
    if (!err) {
        cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
        if (e != cudaSuccess) return e;
    }
    const int ksteps = (K + kBK - 1) / kBK;
    splitk = std::max(1, std::min(splitk, ksteps));
    const int kchunk = ((ksteps + splitk - 1) / splitk) * kBK;
    splitk = (K + kchunk - 1) / kchunk;
    if (nsplit) *nsplit = splitk;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        (void)cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    (void)cudaGetLastError();
    // the widest column block (at most 128) that covers N; narrower while the grid
    // would leave more than half of the SMs without a CTA (few M tiles: the A
    // tiles are then read by several CTAs, from L2)
    const int mtiles = (M + kBM - 1) / kBM;
    int BN = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : 128;
    while (BN > 16 && (int64_t)mtiles * ((N + BN - 1) / BN) * splitk < nsm / 2) BN /= 2;
    const int ntiles = (N + BN - 1) / BN;
    const int csteps = kchunk / kBK;  // K steps of one CTA's chunk
    const int r = relu ? 1 : 0;
    cudaError_t e;
    switch (BN) {
        case 16: e = launch_n<16>(csteps, mtiles, ntiles, splitk, nsm, dependent, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        case 32: e = launch_n<32>(csteps, mtiles, ntiles, splitk, nsm, dependent, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        case 64: e = launch_n<64>(csteps, mtiles, ntiles, splitk, nsm, dependent, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        default: e = launch_n<128>(csteps, mtiles, ntiles, splitk, nsm, dependent, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gsp

extern "C" gsp_status gsp_gemm_bf16(const void *d_A, int64_t lda, const void *d_B, int64_t ldb,
                                    float *d_C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                                    const float *d_bias, int32_t relu, int32_t splitk,
                                    int32_t *d_err, void *stream) {
    if (!d_A || !d_B || !d_C || ldc < N) return GSP_ERR_INVALID_ARG;
    if ((((uintptr_t)d_A | (uintptr_t)d_B) & 15) || (lda & 7) || (ldb & 7) || (K & 7))
        return GSP_ERR_ALIGN;
    cudaError_t e = gsp::launch_gemm_bf16(
        (const __nv_bfloat16 *)d_A, lda, (const __nv_bfloat16 *)d_B, ldb, d_C, ldc, nullptr, 0, M,
        N, K, d_bias, relu != 0, splitk, d_err, (cudaStream_t)stream, 0, nullptr);
    if (e != cudaSuccess) {
        gsp::record_error(e, "gemm launch");
        return e == cudaErrorInvalidValue ? GSP_ERR_INVALID_ARG : GSP_ERR_CUDA;
    }
    return GSP_OK;
}
