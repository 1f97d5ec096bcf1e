// Ingest transpose: time-major 8-bit samples [N][C] (the order of PSRFITS
// files and of Alg. 2's numpts x numchan input matrix, Sec. 2.3) into the
// channel-major [C][N] layout the dedispersion kernels read.  HBM-bound: one
// read and one write per byte.  A CTA moves a 64 x 64 byte tile through shared
// memory, with 16-byte global accesses when pointers and strides allow
// (ingest_transpose16_kernel), else 4-byte or byte accesses.
#include "gsp_internal.cuh"

namespace {

constexpr int kTile = 64;

__global__ void __launch_bounds__(256) ingest_transpose_kernel(const uint8_t *__restrict__ in,
                                                               int64_t in_stride, int64_t N, int C,
                                                               uint8_t *__restrict__ out,
                                                               int64_t out_stride, bool words) {
    __shared__ uint8_t tile[kTile][kTile + 4];
    const int64_t t0 = (int64_t)blockIdx.x * kTile;   // time
    const int c0 = blockIdx.y * kTile;                // channel
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
    // load: rows are times, 4 channels per thread
    for (int r = ty; r < kTile; r += 16) {
        const int64_t t = t0 + r;
        const int c = c0 + 4 * tx;
        uint32_t v = 0;
        if (t < N) {
            const uint8_t *src = in + t * in_stride + c;
            if (words && c + 3 < C) {
                v = __ldg(reinterpret_cast<const uint32_t *>(src));
            } else {
                for (int k = 0; k < 4; k++)
                    if (c + k < C) v |= (uint32_t)__ldg(src + k) << (8 * k);
            }
        }
        tile[r][4 * tx + 0] = (uint8_t)v;
        tile[r][4 * tx + 1] = (uint8_t)(v >> 8);
        tile[r][4 * tx + 2] = (uint8_t)(v >> 16);
        tile[r][4 * tx + 3] = (uint8_t)(v >> 24);
    }
    __syncthreads();
    // store: rows are channels, 4 times per thread
    for (int r = ty; r < kTile; r += 16) {
        const int c = c0 + r;
        if (c >= C) continue;
        const int64_t t = t0 + 4 * tx;
        const uint32_t v = (uint32_t)tile[4 * tx + 0][r] | ((uint32_t)tile[4 * tx + 1][r] << 8) |
                           ((uint32_t)tile[4 * tx + 2][r] << 16) |
                           ((uint32_t)tile[4 * tx + 3][r] << 24);
        uint8_t *dst = out + (int64_t)c * out_stride + t;
        if (words && t + 3 < N) {
            *reinterpret_cast<uint32_t *>(dst) = v;
        } else {
            for (int k = 0; k < 4; k++)
                if (t + k < N) dst[k] = (uint8_t)(v >> (8 * k));
        }
    }
}

// The same with 16-byte global accesses (pointers and strides 16-byte
// aligned) on 256 (time) x 64 (channel) tiles: thread (r, q) loads bytes
// [16q, 16q + 16) of time rows r, r + 64, r + 128, r + 192 into 4-byte words of a
// padded tile (17 words per row); thread (c, q) then gathers byte c of the
// 16-sample groups q, q + 4, q + 8, q + 12 into 16-byte stores of channel row c.
// Four loads and four stores per thread keep more bytes in flight.  Edge
// tiles fall back to byte accesses.
constexpr int kTileT16 = 256;

__global__ void __launch_bounds__(256) ingest_transpose16_kernel(const uint8_t *__restrict__ in,
                                                                 int64_t in_stride, int64_t N,
                                                                 int C, uint8_t *__restrict__ out,
                                                                 int64_t out_stride) {
    __shared__ uint32_t tile[kTileT16][17];
    const int64_t t0 = (int64_t)blockIdx.x * kTileT16;
    const int c0 = blockIdx.y * kTile;
    const int q = threadIdx.x & 3;
#pragma unroll
    for (int i = 0; i < kTileT16 / 64; i++) {
        const int r = (threadIdx.x >> 2) + 64 * i;
        const int64_t t = t0 + r;
        const int c = c0 + 16 * q;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < N) {
            const uint8_t *src = in + t * in_stride + c;
            if (c + 15 < C) {
                v = __ldg(reinterpret_cast<const uint4 *>(src));
            } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                for (int k = 0; k < 16; k++)
                    if (c + k < C) w[k >> 2] |= (uint32_t)__ldg(src + k) << (8 * (k & 3));
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tile[r][4 * q + 0] = v.x;
        tile[r][4 * q + 1] = v.y;
        tile[r][4 * q + 2] = v.z;
        tile[r][4 * q + 3] = v.w;
    }
    __syncthreads();
    const int cl = threadIdx.x >> 2;   // channel inside the tile
    const int c = c0 + cl;
    if (c >= C) return;
    const uint32_t sh = 8u * (uint32_t)(cl & 3);
#pragma unroll
    for (int j = 0; j < kTileT16 / 64; j++) {
        const int grp = q + 4 * j;       // 16-sample group inside the tile
        const int64_t t = t0 + 16 * grp;
        uint32_t w[4];
#pragma unroll
        for (int g = 0; g < 4; g++) {
            uint32_t b[4];
#pragma unroll
            for (int k = 0; k < 4; k++) b[k] = (tile[16 * grp + 4 * g + k][cl >> 2] >> sh) & 0xffu;
            w[g] = b[0] | (b[1] << 8) | (b[2] << 16) | (b[3] << 24);
        }
        uint8_t *dst = out + (int64_t)c * out_stride + t;
        if (t + 15 < N) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            for (int k = 0; k < 16; k++)
                if (t + k < N) dst[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
        }
    }
}

}  // namespace

extern "C" gsp_status gsp_ingest_transpose(const uint8_t *d_in, int64_t n_samp, int32_t nchan,
                                           int64_t in_stride, uint8_t *d_out, int64_t out_stride,
                                           void *stream) {
    if (!d_in || !d_out || n_samp < 0 || nchan <= 0 || in_stride < nchan || out_stride < n_samp)
        return GSP_ERR_INVALID_ARG;
    if (n_samp == 0) return GSP_OK;
    const int64_t tiles_t = (n_samp + kTile - 1) / kTile;
    const int tiles_c = (nchan + kTile - 1) / kTile;
    if (tiles_c > 65535 || tiles_t > 0x7fffffffll) return GSP_ERR_INVALID_ARG;
    const bool words = ((((uintptr_t)d_in | (uintptr_t)d_out) & 3) == 0) && (in_stride % 4 == 0) &&
                       (out_stride % 4 == 0);
    dim3 grid((unsigned)tiles_t, (unsigned)tiles_c);
    const bool v16 = ((((uintptr_t)d_in | (uintptr_t)d_out) & 15) == 0) && (in_stride % 16 == 0) &&
                     (out_stride % 16 == 0);
    if (v16) {
        dim3 grid16((unsigned)((n_samp + kTileT16 - 1) / kTileT16), (unsigned)tiles_c);
        ingest_transpose16_kernel<<<grid16, 256, 0, (cudaStream_t)stream>>>(
            d_in, in_stride, n_samp, nchan, d_out, out_stride);
    }
    else
        ingest_transpose_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_in, in_stride, n_samp,
                                                                        nchan, d_out, out_stride,
                                                                        words);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gsp::record_error(e, "ingest transpose launch");
        return GSP_ERR_CUDA;
    }
    return GSP_OK;
}
