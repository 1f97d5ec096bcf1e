// tcgen05 BF16 GEMM (see tc_gemm.cuh) and its C-ABI entry point.
#include <algorithm>

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

// Launch one instantiation; its dynamic shared-memory limit (above the 48 KB
// default) is raised once per instantiation.
template <int BN, int S, int NACC>
cudaError_t launch_bn(dim3 grid, cudaStream_t s, const __nv_bfloat16 *A, int64_t lda,
                      const __nv_bfloat16 *B, int64_t ldb, float *C, int64_t ldc,
                      __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K, int kchunk,
                      int64_t zstride, const float *bias, int relu, int *err) {
    constexpr int smem = S * (kBM + BN) * kBK * 2;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(gemm_bf16_kernel<BN, S, NACC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    gemm_bf16_kernel<BN, S, NACC><<<grid, 128, smem, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N,
                                                          K, kchunk, zstride, bias, relu, err);
    return cudaSuccess;
}

// Short K (one or two 64-wide steps per tile): one CTA per M tile, one
// accumulator, and one or two stages (small CTAs, many per SM, hide the
// latency).  Longer K: a 4-stage ring, two accumulators, and persistent CTAs
// striding over the M tiles.
template <int BN>
cudaError_t launch_n(int ksteps, int mtiles, int ntiles, int splitk, int nsm, cudaStream_t s,
                     const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B, int64_t ldb,
                     float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K,
                     int kchunk, int64_t zstride, const float *bias, int relu, int *err) {
    if (ksteps <= 2) {
        dim3 grid((unsigned)mtiles, (unsigned)ntiles, (unsigned)splitk);
        if (ksteps == 1)
            return launch_bn<BN, 1, 1>(grid, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk,
                                       zstride, bias, relu, err);
        return launch_bn<BN, 2, 1>(grid, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk,
                                   zstride, bias, relu, err);
    }
    constexpr int smem = 4 * (kBM + BN) * kBK * 2;
    const int per_sm = std::max(1, (227 * 1024) / (smem + 1024));
    const int64_t want = ((int64_t)nsm * per_sm + (int64_t)ntiles * splitk - 1) /
                         ((int64_t)ntiles * splitk);
    const int mgrid = (int)std::max<int64_t>(1, std::min<int64_t>(mtiles, want));
    dim3 grid((unsigned)mgrid, (unsigned)ntiles, (unsigned)splitk);
    return launch_bn<BN, 4, 2>(grid, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride,
                               bias, relu, err);
}

}  // namespace

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                             int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb,
                             int64_t ldcb, int M, int N, int K, const float *bias, bool relu,
                             int splitk, int *err, cudaStream_t s, int64_t zstride, int *nsplit) {
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
        case 16: e = launch_n<16>(csteps, mtiles, ntiles, splitk, nsm, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        case 32: e = launch_n<32>(csteps, mtiles, ntiles, splitk, nsm, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        case 64: e = launch_n<64>(csteps, mtiles, ntiles, splitk, nsm, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
        default: e = launch_n<128>(csteps, mtiles, ntiles, splitk, nsm, s, A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, kchunk, zstride, bias, r, err); break;
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
