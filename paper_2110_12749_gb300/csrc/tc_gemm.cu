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

// Copy the first nc8 8-column chunks of one 128 x 64 (or BN x 64) bf16 tile of a
// K-contiguous matrix into the core-matrix layout: element (r, c) at byte
// (r/8)*1024 + (c/8)*128 + (r%8)*16 + (c%8)*2.  Consecutive threads take
// consecutive rows of one chunk, so each quarter warp writes 128 contiguous
// bytes.  Rows >= nrows and columns >= kend read as zero (kend is a multiple
// of 8).
template <int ROWS>
__device__ __forceinline__ void stage_tile(uint8_t *dst, const __nv_bfloat16 *__restrict__ src,
                                           int64_t ld, int row0, int nrows, int k0, int kend,
                                           int nc8) {
    for (int idx = threadIdx.x; idx < ROWS * nc8; idx += 128) {
        const int r = idx % ROWS, c8 = idx / ROWS;
        const int gr = row0 + r, gk = k0 + c8 * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < nrows && gk < kend)
            v = __ldg(reinterpret_cast<const uint4 *>(src + (int64_t)gr * ld + gk));
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * 1024 + c8 * 128 + (r & 7) * 16) = v;
    }
}

template <int BN>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(
    const __nv_bfloat16 *__restrict__ A, int64_t lda, const __nv_bfloat16 *__restrict__ B,
    int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb, int64_t ldcb, int M, int N, int K,
    int kchunk, const float *__restrict__ bias, int relu, int *err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 M=128 needs N in 16..256");
    __shared__ __align__(1024) uint8_t sA[kBM * kBK * 2];
    __shared__ __align__(1024) uint8_t sB[BN * kBK * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    constexpr uint32_t kCols = BN < 32 ? 32u : (uint32_t)BN;
    constexpr uint32_t kIdesc = tc::idesc_bf16(kBM, BN);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int mtiles = (M + kBM - 1) / kBM;
    const uint32_t bar = tc::smem_u32(&mbar);
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), kCols);
    if (tid == 0) tc::mbar_init1(bar);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t aaddr = tc::smem_u32(sA), baddr = tc::smem_u32(sB);
    uint32_t phase = 0;
    bool ok = true;
    bool pending = false;  // MMAs committed and not yet waited for
    // CTAs stride over the M tiles; tensor memory and the barrier are reused
    for (int mt = blockIdx.x; mt < mtiles && ok; mt += gridDim.x) {
        const int m0 = mt * kBM;
        for (int k0 = kbeg; k0 < kend; k0 += kBK) {
            const int nk = min(kBK, kend - k0);       // a multiple of 8
            const int nmma = (nk + 15) / 16;          // K = 16 per MMA
            // stage the 16-byte chunks the MMAs read (2 per MMA; zeros past kend)
            stage_tile<kBM>(sA, A, lda, m0, M, k0, kend, 2 * nmma);
            stage_tile<BN>(sB, B, ldb, n0, N, k0, kend, 2 * nmma);
            tc::fence_proxy_async();  // generic-proxy smem writes -> tensor-core reads
            tc::fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after();
                for (int kk = 0; kk < nmma; kk++) {
                    // two core matrices along K (256 bytes) per MMA
                    const uint64_t ad = tc::smem_desc(aaddr + kk * 256, 128, 1024);
                    const uint64_t bd = tc::smem_desc(baddr + kk * 256, 128, 1024);
                    tc::mma_bf16(tmem, ad, bd, kIdesc, (k0 > kbeg || kk > 0) ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            pending = true;
            const bool done = tc::mbar_wait_bounded(bar, phase, kGemmBudget);
            phase ^= 1u;
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
            pending = false;
            tc::fence_after();
        }
        if (!ok || kbeg >= kend) break;
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int n = n0 + c0 + j;
                    if (n >= N) break;
                    float val = v[j];
                    if (gridDim.z > 1) {
                        atomicAdd(C + (int64_t)row * ldc + n, val);
                    } else {
                        if (bias) val += bias[n];
                        if (relu) val = fmaxf(val, 0.0f);
                        if (C) C[(int64_t)row * ldc + n] = val;
                        if (Cb) Cb[(int64_t)row * ldcb + n] = __float2bfloat16_rn(val);
                    }
                }
            }
        }
        // every lane's tensor-memory reads are complete before the next tile's MMAs
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // never release tensor memory under MMAs still in flight (bounded)
        if (pending) (void)tc::mbar_wait_bounded(bar, phase ^ 1u, kGemmBudget);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace

cudaError_t launch_gemm_bf16(const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                             int64_t ldb, float *C, int64_t ldc, __nv_bfloat16 *Cb,
                             int64_t ldcb, int M, int N, int K, const float *bias, bool relu,
                             int splitk, int *err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || (K & 7) || (lda & 7) || (ldb & 7) || lda < K || ldb < K ||
        (((uintptr_t)A | (uintptr_t)B) & 15) || (!C && !Cb) || (splitk > 1 && !C))
        return cudaErrorInvalidValue;
    if (!err) {
        cudaError_t e = cudaGetSymbolAddress((void **)&err, g_gemm_err);
        if (e != cudaSuccess) return e;
    }
    const int ksteps = (K + kBK - 1) / kBK;
    splitk = std::max(1, std::min(splitk, ksteps));
    const int kchunk = ((ksteps + splitk - 1) / splitk) * kBK;
    splitk = (K + kchunk - 1) / kchunk;
    const int BN = N <= 16 ? 16 : N <= 32 ? 32 : N <= 64 ? 64 : 128;
    // one CTA per M tile: with one synchronous stage -> MMA -> epilogue chain
    // per tile, many short CTAs overlap better than fewer CTAs striding over
    // the tiles (measured); the kernel still strides if the grid is capped
    const int mtiles = (M + kBM - 1) / kBM, ntiles = (N + BN - 1) / BN;
    const int mgrid = std::max(1, std::min(mtiles, 1 << 30));
    dim3 grid((unsigned)mgrid, (unsigned)ntiles, (unsigned)splitk);
    const int r = relu ? 1 : 0;
    switch (BN) {
        case 16:
            gemm_bf16_kernel<16><<<grid, 128, 0, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K,
                                                      kchunk, bias, r, err);
            break;
        case 32:
            gemm_bf16_kernel<32><<<grid, 128, 0, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K,
                                                      kchunk, bias, r, err);
            break;
        case 64:
            gemm_bf16_kernel<64><<<grid, 128, 0, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K,
                                                      kchunk, bias, r, err);
            break;
        default:
            gemm_bf16_kernel<128><<<grid, 128, 0, s>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K,
                                                       kchunk, bias, r, err);
            break;
    }
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
        N, K, d_bias, relu != 0, splitk, d_err, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        gsp::record_error(e, "gemm launch");
        return e == cudaErrorInvalidValue ? GSP_ERR_INVALID_ARG : GSP_ERR_CUDA;
    }
    return GSP_OK;
}
