// Candidate ranker: a small CNN over 64 x 64 DM-time snippets of the
// single-pulse candidates, trained and run on the GPU (the project's own
// design for the candidate-ranking step the paper motivates, Sec. 1-2: it
// ranks the plain threshold output, never replaces it).
//
// Network: three conv 3x3 (pad 1) + bias + ReLU + 2x2 max-pool layers
// (1 -> 8 -> 16 -> 32 channels, 64x64 -> 8x8), fc 2048 -> 96 + ReLU, fc 96 -> 2.
// Activations are NHWC.  Every convolution of a training pass is an im2col
// GEMM on the tcgen05 tensor cores (tc_gemm.cu), BF16 operands and FP32
// accumulation in tensor memory, bias and ReLU fused into the epilogue.  An
// inference pass fuses each conv layer with its bias, ReLU and pool at the
// same rounding points: layer 0 (one input channel, K = 9) on the CUDA cores,
// layers 1 and 2 as implicit GEMMs on the tensor cores that gather their taps
// straight from the activations.  fc 2048 -> 96 and the
// back-propagated products of both fc layers and the convolutions are GEMMs
// too (weight gradients with split-K over the batch pixels).  The 96 -> 2
// layer, the loss, pooling, im2col / col2im, bias gradients and Adam are
// elementwise kernels in FP32.  Every operand of a product is rounded to
// bf16 (nearest even), at the same points as the CPU oracle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dd_tiled.cuh"
#include "gsp_internal.cuh"
#include "tc_gemm.cuh"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kS = 64;          // snippet side
constexpr int kFc = 2048;       // 32 x 8 x 8 features
constexpr int kHid = 96;        // hidden units of fc1 (202,786 parameters in all)
constexpr int kFc1Split = 8;    // most K chunks of fc1 (K = 2048: 32 steps of 64)
constexpr int kLayers = 3;
// per conv layer: input channels, output channels, input side
__host__ __device__ constexpr int cin_of(int l) { return l == 0 ? 1 : (l == 1 ? 8 : 16); }
__host__ __device__ constexpr int cout_of(int l) { return l == 0 ? 8 : (l == 1 ? 16 : 32); }
__host__ __device__ constexpr int side_of(int l) { return l == 0 ? 64 : (l == 1 ? 32 : 16); }

__host__ __device__ constexpr int round8(int v) { return (v + 7) & ~7; }
__host__ __device__ constexpr int kdim(int l) { return 9 * cin_of(l); }         // im2col K
__host__ __device__ constexpr int kpad(int l) { return round8(kdim(l)); }

// Parameter offsets in the flat FP32 vector (order w1 b1 w2 b2 w3 b3 w4 b4 w5 b5,
// each in the oracle's layout: conv w[co][ci][ky][kx], fc w[out][in]).
struct Offsets {
    int64_t w[5], b[5], total;
};
constexpr int kWsize[5] = {8 * 1 * 9, 16 * 8 * 9, 32 * 16 * 9, kHid * kFc, 2 * kHid};
constexpr int kBsize[5] = {8, 16, 32, kHid, 2};
Offsets offsets() {
    Offsets o{};
    int64_t p = 0;
    for (int i = 0; i < 5; i++) {
        o.w[i] = p;
        p += kWsize[i];
        o.b[i] = p;
        p += kBsize[i];
    }
    o.total = p;
    return o;
}

// ------------------------------------------------------------- elementwise

// im2col of an NHWC activation (layer 0: the FP32 snippets, rounded to bf16
// here): col[(b, y, x)][(ky * 3 + kx) * CIN + ci] = a[b][y + ky - 1][x + kx - 1][ci],
// zero outside the image and in the padding columns K..Kp.  One thread per
// pixel writes its whole row of Kp values in 16-byte pieces (consecutive
// threads write consecutive rows); channel taps are read 16 bytes at a time
// when CIN is a multiple of 8.
template <typename T, int CIN>
__global__ void __launch_bounds__(256) im2col_kernel(const T *__restrict__ a, int B, int H,
                                                     bf16 *__restrict__ col) {
    constexpr int K = 9 * CIN, KP = (K + 7) & ~7;
    const int64_t npix = (int64_t)B * H * H;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = p / (H * H);
        const int rem = (int)(p - b * H * H);
        const int y = rem / H, x = rem - (rem / H) * H;
        __align__(16) bf16 row[KP];
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
            const bool in = yy >= 0 && yy < H && xx >= 0 && xx < H;
            const T *src = a + ((b * H + yy) * H + xx) * CIN;
            if constexpr (CIN % 8 == 0 && sizeof(T) == 2) {
#pragma unroll
                for (int c8 = 0; c8 < CIN / 8; c8++) {
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (in) v = __ldg(reinterpret_cast<const uint4 *>(src) + c8);
                    *reinterpret_cast<uint4 *>(&row[tap * CIN + c8 * 8]) = v;
                }
            } else {
#pragma unroll
                for (int ci = 0; ci < CIN; ci++)
                    row[tap * CIN + ci] = __float2bfloat16_rn(in ? (float)src[ci] : 0.0f);
            }
        }
#pragma unroll
        for (int k = K; k < KP; k++) row[k] = __float2bfloat16_rn(0.0f);
        uint4 *dst = reinterpret_cast<uint4 *>(col + p * KP);
#pragma unroll
        for (int q = 0; q < KP / 8; q++) dst[q] = *reinterpret_cast<const uint4 *>(&row[q * 8]);
    }
}

// fma(a, b.x, c.x), fma(a, b.y, c.y) as one packed instruction (two IEEE
// single-precision FMAs, the same results as two fmaf): half the issue slots
__device__ __forceinline__ float2 fma_pair(float a, float2 b, float2 c) {
    uint64_t av, bv, cv, d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cv) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(av), "l"(bv), "l"(cv));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
    return r;
}

// Layer 0 of an inference pass: conv 3x3 (1 -> 8, pad 1) + bias + ReLU + 2x2
// max-pool straight from the FP32 snippets, on the CUDA cores: with one input
// channel the product has K = 9, too short for the tensor pipe to pay for its
// staging.  The rounding points are those of the im2col + GEMM + pool path:
// inputs and weights in bf16, the nine products and the bias summed in FP32
// (in the same order), the pooled maximum rounded to bf16.  One thread per pair
// of horizontally adjacent pooled pixels reads its 4 x 6 input patch; per
// channel it loads the nine weights once and computes the pair's 2 x 4 conv
// outputs, then writes the two pixels' 8 bf16 results as two 16-byte stores
// (NHWC, as pool_kernel<8>).  Channels 2p and 2p + 1 share each packed FMA.
__global__ void __launch_bounds__(256) conv0_pool_kernel(const float *__restrict__ x, int B,
                                                         const bf16 *__restrict__ W0,
                                                         const float *__restrict__ b0,
                                                         bf16 *__restrict__ a0) {
    constexpr int C = 8, KP = kpad(0), H = kS, H2 = kS / 2, HP = H2 / 2;
    __shared__ float2 sw[C / 2][9];  // channels 2p and 2p + 1 side by side
    __shared__ float2 sb[C / 2];
    for (int i = threadIdx.x; i < C * 9; i += blockDim.x) {
        const float w = __bfloat162float(W0[(i / 9) * KP + i % 9]);
        if ((i / 9) & 1) sw[i / 18][i % 9].y = w;
        else sw[i / 18][i % 9].x = w;
    }
    for (int i = threadIdx.x; i < C; i += blockDim.x) {
        if (i & 1) sb[i / 2].y = b0[i];
        else sb[i / 2].x = b0[i];
    }
    __syncthreads();
    const int64_t total = (int64_t)B * H2 * HP;  // pixel pairs
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = q / (H2 * HP);
        const int rem = (int)(q - b * H2 * HP);
        const int y2 = rem / HP, x2 = 2 * (rem - (rem / HP) * HP);  // first pooled column
        const float *img = x + b * H * H;
        float v[4][6];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int yy = 2 * y2 - 1 + r;
#pragma unroll
            for (int c = 0; c < 6; c++) {
                const int xx = 2 * x2 - 1 + c;
                const bool in = yy >= 0 && yy < H && xx >= 0 && xx < H;
                v[r][c] = in ? __bfloat162float(__float2bfloat16_rn(__ldg(img + yy * H + xx)))
                             : 0.0f;
            }
        }
        __align__(16) bf16 out[2][C];
#pragma unroll
        for (int cp = 0; cp < C / 2; cp++) {  // channels 2 cp and 2 cp + 1 together
            float2 w[9];
#pragma unroll
            for (int k = 0; k < 9; k++) w[k] = sw[cp][k];
            const float2 bias = sb[cp];
#pragma unroll
            for (int px = 0; px < 2; px++) {
                float m0 = 0.0f, m1 = 0.0f;  // ReLU outputs are >= 0
#pragma unroll
                for (int dy = 0; dy < 2; dy++)
#pragma unroll
                    for (int dx = 0; dx < 2; dx++) {
                        float2 z = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int ky = 0; ky < 3; ky++)
#pragma unroll
                            for (int kx = 0; kx < 3; kx++)
                                z = fma_pair(v[dy + ky][2 * px + dx + kx], w[ky * 3 + kx], z);
                        m0 = fmaxf(m0, z.x + bias.x);
                        m1 = fmaxf(m1, z.y + bias.y);
                    }
                out[px][2 * cp] = __float2bfloat16_rn(m0);
                out[px][2 * cp + 1] = __float2bfloat16_rn(m1);
            }
        }
        const int64_t pix = (b * H2 + y2) * H2 + x2;
        *reinterpret_cast<uint4 *>(a0 + pix * C) = *reinterpret_cast<const uint4 *>(out[0]);
        *reinterpret_cast<uint4 *>(a0 + (pix + 1) * C) = *reinterpret_cast<const uint4 *>(out[1]);
    }
}

// 2x2 max-pool of the ReLU'd pre-activations z (FP32 NHWC [B][H][H][C]):
// out bf16 [B][H/2][H/2][C], idx = argmax in (0,0), (0,1), (1,0), (1,1) order
// (first maximum wins).  One thread per pooled pixel, all C channels (float4
// loads).
template <int C>
__global__ void __launch_bounds__(256) pool_kernel(const float *__restrict__ z, int B, int H,
                                                   bf16 *__restrict__ out,
                                                   uint8_t *__restrict__ idx) {
    const int H2 = H / 2;
    const int64_t total = (int64_t)B * H2 * H2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = q / (H2 * H2);
        const int rem = (int)(q - b * H2 * H2);
        const int y = rem / H2, x = rem - (rem / H2) * H2;
        const float *p0 = z + ((b * H + 2 * y) * H + 2 * x) * C;
        const float *src[4] = {p0, p0 + C, p0 + (int64_t)H * C, p0 + (int64_t)H * C + C};
#pragma unroll
        for (int c4 = 0; c4 < C / 4; c4++) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; k++) v[k] = __ldg(reinterpret_cast<const float4 *>(src[k]) + c4);
            float m[4] = {v[0].x, v[0].y, v[0].z, v[0].w};
            uint32_t kk[4] = {0, 0, 0, 0};
#pragma unroll
            for (int k = 1; k < 4; k++) {
                const float w[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (w[e] > m[e]) {
                        m[e] = w[e];
                        kk[e] = (uint32_t)k;
                    }
            }
            const int64_t o = q * C + c4 * 4;
#pragma unroll
            for (int e = 0; e < 4; e++) out[o + e] = __float2bfloat16_rn(m[e]);
            *reinterpret_cast<uint32_t *>(idx + o) = kk[0] | (kk[1] << 8) | (kk[2] << 16) | (kk[3] << 24);
        }
    }
}

// Back through the pool and the ReLU: g[b][y][x][c] = ga[b][y/2][x/2][c] if (y, x)
// is the window's argmax and z > 0, else 0.  Writes bf16 g as [P][C] and as
// its transpose [C][P] (P = B*H*H pixels, ldT >= P), and adds FP32 per-channel
// sums into db.
__global__ void pool_back_kernel(const float *__restrict__ ga, const uint8_t *__restrict__ idx,
                                 const float *__restrict__ z, int B, int H, int C,
                                 bf16 *__restrict__ g, bf16 *__restrict__ gT, int64_t ldT,
                                 float *__restrict__ db) {
    extern __shared__ float sdb[];
    for (int c = threadIdx.x; c < C; c += blockDim.x) sdb[c] = 0.0f;
    __syncthreads();
    const int H2 = H / 2;
    const int64_t P = (int64_t)B * H * H;
    const int64_t total = P * C;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int64_t p = i / C;
        const int x = (int)(p % H), y = (int)((p / H) % H);
        const int64_t b = p / ((int64_t)H * H);
        const int64_t q = ((b * H2 + y / 2) * H2 + x / 2) * C + c;
        const int k = (y & 1) * 2 + (x & 1);
        float v = 0.0f;
        if (idx[q] == k && z[i] > 0.0f) v = ga[q];
        g[i] = __float2bfloat16_rn(v);
        gT[(int64_t)c * ldT + p] = __float2bfloat16_rn(v);
        if (v != 0.0f) atomicAdd(&sdb[c], v);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x)
        if (sdb[c] != 0.0f) atomicAdd(&db[c], sdb[c]);
}

// col2im (gather form): ga[b][y][x][ci] = sum over taps (ky, kx) of
// dcol[(b, y - ky + 1, x - kx + 1)][(ky * 3 + kx) * Cin + ci].
__global__ void col2im_kernel(const float *__restrict__ dcol, int B, int H, int Cin, int Kp,
                              float *__restrict__ ga) {
    const int64_t total = (int64_t)B * H * H * Cin;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const int64_t p = i / Cin;
        const int x = (int)(p % H), y = (int)((p / H) % H);
        const int64_t b = p / ((int64_t)H * H);
        float s = 0.0f;
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int yy = y - tap / 3 + 1, xx = x - tap % 3 + 1;
            if (yy >= 0 && yy < H && xx >= 0 && xx < H)
                s += dcol[((b * H + yy) * H + xx) * Kp + tap * Cin + ci];
        }
        ga[i] = s;
    }
}

// bf16 transpose: out[c][r] = in[r][c] for r < R, c < Cc (32 x 32 tiles).
__global__ void transpose_kernel(const bf16 *__restrict__ in, int64_t ldi, int64_t R, int Cc,
                                 bf16 *__restrict__ out, int64_t ldo) {
    __shared__ bf16 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int c = c0 + threadIdx.x;
        t[k][threadIdx.x] = (r < R && c < Cc) ? in[r * ldi + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (c < Cc && r < R) out[(int64_t)c * ldo + r] = t[threadIdx.x][k];
    }
}

// fc 96 -> 2 (CUDA cores): z5[b][o] = sum_k a4[b][k] * bf16(w5[o][k]) + b5[o].
__global__ void fc2_kernel(const bf16 *__restrict__ a4, const float *__restrict__ w5,
                           const float *__restrict__ b5, int B, float *__restrict__ z5) {
    gsp::wait_prior_grid();  // a4 comes from the kernel launched just before
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * 2) return;
    const int b = i / 2, o = i % 2;
    float s = 0.0f;
    for (int k = 0; k < kHid; k++)
        s = fmaf((float)a4[b * kHid + k], __bfloat162float(__float2bfloat16_rn(w5[o * kHid + k])), s);
    z5[i] = s + b5[o];
}

// Mean softmax cross-entropy and its gradient g5 = (softmax - onehot) / B, one
// block; loss_out (optional) receives the mean loss.
__global__ void loss_kernel(const float *__restrict__ z5, const int32_t *__restrict__ y, int B,
                            float *__restrict__ g5, float *__restrict__ loss_out) {
    __shared__ float red[256];
    float acc = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float z0 = z5[2 * b], z1 = z5[2 * b + 1];
        const float m = fmaxf(z0, z1);
        const float e0 = expf(z0 - m), e1 = expf(z1 - m);
        const float s = e0 + e1;
        const int lab = y[b] ? 1 : 0;
        acc += -logf((lab ? e1 : e0) / s);
        g5[2 * b] = (e0 / s - (lab == 0 ? 1.0f : 0.0f)) / (float)B;
        g5[2 * b + 1] = (e1 / s - (lab == 1 ? 1.0f : 0.0f)) / (float)B;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss_out) *loss_out = red[0] / (float)B;
}

// Back through fc 96 -> 2 and the ReLU of fc1 (CUDA cores):
//   dw5[o][k] = sum_b bf16(g5[b][o]) * a4[b][k],  db5[o] = sum_b g5[b][o]   (block 0)
//   g4[b][k]  = (sum_o bf16(g5[b][o]) * bf16(w5[o][k])) * [z4[b][k] > 0]
// g4 is written as bf16 [B][96] and transposed [96][ldT]; db4 += FP32 sums.
__global__ void fc2_back_kernel(const float *__restrict__ g5, const bf16 *__restrict__ a4,
                                const float *__restrict__ w5, const float *__restrict__ z4,
                                int B, float *__restrict__ dw5, float *__restrict__ db5,
                                bf16 *__restrict__ g4, bf16 *__restrict__ g4T, int64_t ldT,
                                float *__restrict__ db4) {
    const int k = threadIdx.x;  // kHid threads: one hidden unit each
    if (blockIdx.x == 0) {
        float s0 = 0.0f, s1 = 0.0f, t0 = 0.0f, t1 = 0.0f;
        for (int b = 0; b < B; b++) {
            const float a = (float)a4[b * kHid + k];
            s0 = fmaf(__bfloat162float(__float2bfloat16_rn(g5[2 * b])), a, s0);
            s1 = fmaf(__bfloat162float(__float2bfloat16_rn(g5[2 * b + 1])), a, s1);
            t0 += g5[2 * b];
            t1 += g5[2 * b + 1];
        }
        dw5[k] = s0;
        dw5[kHid + k] = s1;
        if (k == 0) {
            db5[0] = t0;
            db5[1] = t1;
        }
    }
    const float w0 = __bfloat162float(__float2bfloat16_rn(w5[k]));
    const float w1 = __bfloat162float(__float2bfloat16_rn(w5[kHid + k]));
    float dsum = 0.0f;
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const float ga = __bfloat162float(__float2bfloat16_rn(g5[2 * b])) * w0 +
                         __bfloat162float(__float2bfloat16_rn(g5[2 * b + 1])) * w1;
        const float v = z4[b * kHid + k] > 0.0f ? ga : 0.0f;
        g4[b * kHid + k] = __float2bfloat16_rn(v);
        g4T[(int64_t)k * ldT + b] = __float2bfloat16_rn(v);
        dsum += v;
    }
    atomicAdd(&db4[k], dsum);
}

// Adam on the flat FP32 parameter vector (step number t >= 1).
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 GEMM copies of the conv weights: W[co][(ky*3+kx)*Cin + ci] (padded to
// Kp) and its transpose WT[k][co] (ld Cout8), from w[co][ci][ky][kx]; and the
// fc1 weight W4 [96][2048] with its transpose W4T [2048][96].
__global__ void pack_kernel(const float *__restrict__ params, int64_t w1, int64_t w2, int64_t w3,
                            int64_t w4, bf16 *__restrict__ W0, bf16 *__restrict__ W0T,
                            bf16 *__restrict__ W1, bf16 *__restrict__ W1T, bf16 *__restrict__ W2,
                            bf16 *__restrict__ W2T, bf16 *__restrict__ W4,
                            bf16 *__restrict__ W4T) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < (int64_t)kHid * kFc) {
        const bf16 v = __float2bfloat16_rn(params[w4 + i]);
        W4[i] = v;
        W4T[(i % kFc) * kHid + i / kFc] = v;
    }
    const int64_t woff[3] = {w1, w2, w3};
    bf16 *Wd[3] = {W0, W1, W2};
    bf16 *WTd[3] = {W0T, W1T, W2T};
#pragma unroll
    for (int l = 0; l < kLayers; l++) {
        const int Cin = cin_of(l), Cout = cout_of(l), Kp = kpad(l);
        if (i < (int64_t)Cout * Kp) {
            const int co = (int)(i / Kp), k = (int)(i % Kp);
            float v = 0.0f;
            if (k < 9 * Cin) {
                const int tap = k / Cin, ci = k % Cin;
                v = params[woff[l] + ((int64_t)co * Cin + ci) * 9 + tap];
            }
            const bf16 b = __float2bfloat16_rn(v);
            Wd[l][i] = b;
            WTd[l][(int64_t)k * round8(Cout) + co] = b;
        }
    }
}

// Back to the oracle's conv weight-gradient layout: dw[co][ci][ky][kx] =
// dW[co][(ky*3+kx)*Cin + ci].
__global__ void unpack_conv_grad_kernel(const float *__restrict__ dW, int Cin, int Cout, int Kp,
                                        float *__restrict__ dw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Cout * Cin * 9) return;
    const int tap = i % 9, ci = (i / 9) % Cin, co = i / (9 * Cin);
    dw[i] = dW[(int64_t)co * Kp + tap * Cin + ci];
}

}  // namespace

namespace {

// fc1's epilogue after a split-K product: z4 = ReLU(sum over the S partial
// products, in chunk order, + bias) and a4 = bf16(z4).  One thread per output.
__global__ void fc1_finish_kernel(const float *__restrict__ part, int S, int64_t zstride, int B,
                                  const float *__restrict__ bias, float *__restrict__ z4,
                                  bf16 *__restrict__ a4) {
    gsp::wait_prior_grid();  // part comes from the kernel launched just before
    const int64_t total = (int64_t)B * kHid;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = part[i];
        for (int z = 1; z < S; z++) acc += part[(int64_t)z * zstride + i];
        const float v = fmaxf(acc + bias[i % kHid], 0.0f);
        z4[i] = v;
        a4[i] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------- fused conv layers for inference

namespace tc = gsp::tc;
namespace ptx = gsp::ptx;

constexpr long long kConvBudget = 2000000000ll;  // ~1 s of SM clock per wait

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

// Layers 1 and 2 of an inference pass: conv 3x3 (CIN -> COUT, pad 1) as an
// implicit GEMM on the tcgen05 tensor cores, + bias + ReLU + 2x2 max-pool in
// the epilogue, from the bf16 NHWC activation act [B][SIDE][SIDE][CIN] to the
// pooled bf16 NHWC output out [B][SIDE/2][SIDE/2][COUT].  The products and
// their rounding points are those of the im2col + GEMM + pool path (the same
// K order and K = 16 steps, FP32 accumulation in tensor memory, bias after
// the accumulation, the pooled maximum rounded to bf16).
//
// Persistent CTAs of 4 warps stride over 128-pixel M tiles (a tile is 128 /
// SIDE whole image rows, so every 2x2 pooling window lies inside it).  Each
// thread gathers the 9 taps of its pixel straight from act with 16-byte
// cp.async copies (zero-filled outside the image) into the K-major
// core-matrix layout; the weights are staged once per CTA.  One A buffer and
// one accumulator per CTA, so that many CTAs fit an SM.  Per tile: wait for
// the gather, MMAs, wait for them; then the next tile's gather runs under
// this tile's epilogue, which pools mostly in registers:
//  * SIDE 16: a tile is 8 image rows, warp w holding rows 2w and 2w + 1
//    (lane l: row 2w + l / 16, column l % 16), so each pooling window lies in
//    one warp: two shuffles (partners l ^ 1 and l ^ 16).
//  * SIDE 32: a tile is 4 image rows, warp w holding row w: a shuffle pools
//    column pairs (l ^ 1), and warps 1 and 3 hand their row maxima to warps 0
//    and 2 through a 2 KB shared buffer.
// Every wait is bounded; on a timeout the kernel sets *err, waits (bounded)
// for its MMAs in flight and releases its tensor memory.
template <int CIN, int COUT, int SIDE>
__global__ void __launch_bounds__(128) conv_pool_solo_tc_kernel(const bf16 *__restrict__ act,
                                                                int B, const bf16 *__restrict__ W,
                                                                const float *__restrict__ bias,
                                                                bf16 *__restrict__ out, int *err) {
    constexpr int PW = SIDE / 2;
    static_assert(CIN % 8 == 0 && COUT % 16 == 0 && COUT <= 32, "shapes of layers 1 and 2");
    static_assert(SIDE == 16 || SIDE == 32, "16 x 16 or 32 x 32 images");
    constexpr int K = 9 * CIN;
    constexpr int NK16 = (K + 15) / 16;
    constexpr int KC = K / 8;
    constexpr int KCS = NK16 * 2;
    constexpr uint32_t SBO = KCS * 128;
    constexpr int A_BYTES = 128 * KCS * 16;
    constexpr uint32_t kCols = COUT < 32 ? 32u : (uint32_t)COUT;
    constexpr uint32_t kIdesc = tc::idesc_bf16(128, COUT);
    constexpr int KP = (K + 7) & ~7;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem, *sB = smem + A_BYTES;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sB + COUT * KCS * 16);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    __shared__ float sbias[COUT];
    __shared__ __align__(16) float sx[SIDE == 32 ? 2 : 1][16][16];  // SIDE 32: odd rows' maxima

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (int64_t)B * SIDE * SIDE / 128;
    const int64_t my = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kCols);
    if (tid == 0) tc::mbar_init1(tc::smem_u32(bar));
    for (int i = tid; i < COUT; i += 128) sbias[i] = bias[i];
    for (int idx = tid; idx < COUT * KCS; idx += 128) {
        const int n = idx % COUT, q = idx / COUT;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (q < KC) v = __ldg(reinterpret_cast<const uint4 *>(W + (int64_t)n * KP) + q);
        *reinterpret_cast<uint4 *>(sB + (n >> 3) * SBO + q * 128 + (n & 7) * 16) = v;
    }
    for (int idx = tid; idx < 128 * (KCS - KC); idx += 128) {
        const int r = idx & 127, q = KC + (idx >> 7);
        *reinterpret_cast<uint4 *>(sA + (r >> 3) * SBO + q * 128 + (r & 7) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    gsp::wait_prior_grid();  // act comes from the kernel launched just before
    const uint32_t a_addr = tc::smem_u32(sA), b_addr = tc::smem_u32(sB);
    const uint32_t bar0 = tc::smem_u32(bar);

    auto gather = [&](int64_t tile) {
        const int64_t p = tile * 128 + tid;
        const int rem = (int)(p & (SIDE * SIDE - 1));
        const int y = rem / SIDE, x = rem % SIDE;
        const bf16 *base = act + p * CIN;
        const uint32_t dst = a_addr + (tid >> 3) * SBO + (tid & 7) * 16;
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const bool in = (unsigned)(y + dy) < (unsigned)SIDE && (unsigned)(x + dx) < (unsigned)SIDE;
            const bf16 *src = in ? base + (dy * SIDE + dx) * CIN : act;
#pragma unroll
            for (int j = 0; j < CIN / 8; j++)
                cp_async16(dst + (tap * (CIN / 8) + j) * 128, src + (in ? j * 8 : 0), in ? 16u : 0u);
        }
    };
    // bias + ReLU, 2x2 max, bf16 stores by the lane of each window's first pixel
    auto epilogue = [&](int64_t tile) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        const int64_t m0 = tile * 128;
        const int64_t b = m0 / (SIDE * SIDE);
        const int y0 = (int)(m0 - b * SIDE * SIDE) / SIDE;  // the tile's first image row
        const int py = SIDE == 16 ? y0 / 2 + warp : y0 / 2 + (warp >> 1);  // pooled row
        const int px = SIDE == 16 ? (lane & 15) >> 1 : lane >> 1;
        bf16 *dst = out + ((b * PW + py) * PW + px) * COUT;
        const bool writer = SIDE == 16 ? (lane & 17) == 0 : ((lane & 1) == 0 && (warp & 1) == 0);
#pragma unroll
        for (int c0 = 0; c0 < COUT; c0 += 16) {
            float v[16];
            tc::tmem_ld16(taddr + (uint32_t)c0, v);
            float z[16];
#pragma unroll
            for (int c = 0; c < 16; c++) {
                z[c] = fmaxf(v[c] + sbias[c0 + c], 0.0f);
                z[c] = fmaxf(z[c], __shfl_xor_sync(0xffffffffu, z[c], 1));
                if (SIDE == 16) z[c] = fmaxf(z[c], __shfl_xor_sync(0xffffffffu, z[c], 16));
            }
            if (SIDE == 32) {
                // the odd row of each row pair hands its column-pair maxima over
                if ((warp & 1) && (lane & 1) == 0) {
#pragma unroll
                    for (int c = 0; c < 16; c += 4)
                        *reinterpret_cast<float4 *>(&sx[warp >> 1][lane >> 1][c]) =
                            make_float4(z[c], z[c + 1], z[c + 2], z[c + 3]);
                }
                __syncthreads();
                if (writer) {
#pragma unroll
                    for (int c = 0; c < 16; c += 4) {
                        const float4 q = *reinterpret_cast<const float4 *>(&sx[warp >> 1][lane >> 1][c]);
                        z[c] = fmaxf(z[c], q.x);
                        z[c + 1] = fmaxf(z[c + 1], q.y);
                        z[c + 2] = fmaxf(z[c + 2], q.z);
                        z[c + 3] = fmaxf(z[c + 3], q.w);
                    }
                }
                __syncthreads();  // sx is rewritten by the next column block or tile
            }
            if (writer) {
                __align__(16) bf16 o[16];
#pragma unroll
                for (int c = 0; c < 16; c++) o[c] = __float2bfloat16_rn(z[c]);
                *reinterpret_cast<uint4 *>(dst + c0) = *reinterpret_cast<const uint4 *>(o);
                *reinterpret_cast<uint4 *>(dst + c0 + 8) = *reinterpret_cast<const uint4 *>(o + 8);
            }
        }
    };

    uint32_t ph = 0u;
    bool pend = false, ok = true;
    if (my > 0) {
        gather(blockIdx.x);
        cp_async_commit();
    }
    for (int64_t k = 0; k < my; k++) {
        const int64_t tile = blockIdx.x + k * gridDim.x;
        cp_async_wait<0>();
        tc::fence_proxy_async();  // this thread's copies -> tensor-core reads
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < NK16; kk++) {
                const uint64_t ad = tc::smem_desc(a_addr + kk * 256, 128, SBO);
                const uint64_t bd = tc::smem_desc(b_addr + kk * 256, 128, SBO);
                tc::mma_bf16(tmem, ad, bd, kIdesc, kk > 0 ? 1u : 0u);
            }
            tc::mma_commit(bar0);
        }
        pend = true;
        const bool done = tc::mbar_wait_bounded(bar0, ph, kConvBudget);
        if (!__syncthreads_and(done)) {
            ok = false;
            break;
        }
        ph ^= 1u;
        pend = false;
        tc::fence_after();
        if (k + 1 < my) {  // the MMAs are done with A: refill it under the epilogue
            gather(tile + gridDim.x);
            cp_async_commit();
        }
        epilogue(tile);
    }
    cp_async_wait<0>();
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        if (pend) (void)tc::mbar_wait_bounded(bar0, ph, kConvBudget);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

template <int CIN, int COUT>
constexpr int conv_pool_solo_smem() {
    return 128 * ((9 * CIN + 15) / 16) * 2 * 16 + COUT * ((9 * CIN + 15) / 16) * 2 * 16 + 8 + 16;
}

}  // namespace

struct gsp_ranker_s {
    int max_batch = 0;
    Offsets off{};
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    int64_t step = 0;
    // packed bf16 weights
    bf16 *W[kLayers] = {}, *WT[kLayers] = {}, *W4 = nullptr, *W4T = nullptr;
    // activations
    bf16 *col[kLayers] = {}, *colT[kLayers] = {}, *a[kLayers] = {};
    float *z[kLayers] = {};
    uint8_t *idx[kLayers] = {};
    float *z4 = nullptr, *z5 = nullptr, *g5 = nullptr, *ga3 = nullptr, *loss = nullptr;
    bf16 *a4 = nullptr, *g4 = nullptr, *g4T = nullptr, *a3T = nullptr;
    // backward scratch
    bf16 *gz[kLayers] = {}, *gzT[kLayers] = {};
    float *ga[kLayers] = {};    // gradient w.r.t. the pooled output of layer l
    float *dcol = nullptr, *dW = nullptr;
    float *fc1_part = nullptr;  // [kFc1Split][max_batch][kHid] partial products of fc1
    int *err = nullptr;
    std::vector<void *> allocs;
    int32_t launches = 0;
    int32_t last_n = 0;      // snippets of the last pass
    int last_pass = 0;       // 0 none, 1 inference (gsp_ranker_forward), 2 training step
};

namespace {

template <typename T>
bool ralloc(gsp_ranker_s *r, T **p, size_t n) {
    if (cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    r->allocs.push_back(*p);
    return true;
}

void free_ranker(gsp_ranker_s *r) {
    if (!r) return;
    for (void *p : r->allocs) cudaFree(p);
    delete r;
}

int blocks_for(int64_t n, int threads = 256) {
    return (int)std::min<int64_t>((n + threads - 1) / threads, 152 * 16);
}

#define RK_LAUNCH(...)                                \
    do {                                              \
        __VA_ARGS__;                                  \
        cudaError_t e_ = cudaGetLastError();          \
        if (e_ != cudaSuccess) return e_;             \
        r->launches++;                                \
    } while (0)

cudaError_t pack(gsp_ranker_s *r, cudaStream_t s) {
    RK_LAUNCH((pack_kernel<<<blocks_for((int64_t)kHid * kFc), 256, 0, s>>>(
        r->params, r->off.w[0], r->off.w[1], r->off.w[2], r->off.w[3], r->W[0], r->WT[0], r->W[1],
        r->WT[1], r->W[2], r->WT[2], r->W4, r->W4T)));
    return cudaSuccess;
}

cudaError_t gemm(gsp_ranker_s *r, const bf16 *A, int64_t lda, const bf16 *B, int64_t ldb, float *C,
                 int64_t ldc, bf16 *Cb, int64_t ldcb, int M, int N, int K, const float *bias,
                 bool relu, int splitk, cudaStream_t s) {
    cudaError_t e = gsp::launch_gemm_bf16(A, lda, B, ldb, C, ldc, Cb, ldcb, M, N, K, bias, relu,
                                          splitk, r->err, s);
    if (e == cudaSuccess) r->launches++;
    return e;
}

// CTAs per SM of a fused conv kernel from its resources: shared memory (stages +
// static + the per-CTA reservation), registers, threads, and at most 512
// tensor-memory columns per SM (cols per CTA).  The runtime's occupancy query
// answers one CTA per SM for these kernels whatever their shared memory, while
// several do run side by side (four CTAs per SM run layer 1 2.3x faster than
// one), so the count is computed here.  Also raises the kernel's dynamic
// shared-memory limit on the current device and asks for the largest
// shared-memory carveout (every launch calls that too: attributes are per device).
template <typename Kern>
cudaError_t conv_ctas_per_sm(Kern kern, int smem, int cols, int *out) {
    cudaError_t e = gsp::ensure_kernel_smem(reinterpret_cast<const void *>(kern), smem, true);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    int dev = 0, smem_sm = 0, resv = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int by_smem = smem_sm / (smem + (int)fa.sharedSizeBytes + resv);
    const int by_regs = 65536 / (128 * std::max(fa.numRegs, 1));
    const int by_tmem = 512 / std::max(32, cols);
    *out = std::max(1, std::min(std::min(by_smem, by_regs), std::min(by_tmem, 16)));
    return cudaSuccess;
}

template <int CIN, int COUT, int SIDE>
cudaError_t launch_conv_pool_solo(gsp_ranker_s *r, const bf16 *act, int n, const bf16 *W,
                                  const float *bias, bf16 *out, cudaStream_t s, bool dependent) {
    constexpr int smem = conv_pool_solo_smem<CIN, COUT>();
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = conv_ctas_per_sm(conv_pool_solo_tc_kernel<CIN, COUT, SIDE>, smem, COUT,
                                         &blocks_per_sm);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = gsp::ensure_kernel_smem(
            reinterpret_cast<const void *>(conv_pool_solo_tc_kernel<CIN, COUT, SIDE>), smem, true);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (int64_t)n * SIDE * SIDE / 128;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sms * blocks_per_sm));
    if (dependent) {
        e = gsp::launch_dependent(conv_pool_solo_tc_kernel<CIN, COUT, SIDE>, dim3(grid), dim3(128),
                                  (size_t)smem, s, act, n, W, bias, out, r->err);
        if (e != cudaSuccess) return e;
        r->launches++;
        return cudaSuccess;
    }
    RK_LAUNCH((conv_pool_solo_tc_kernel<CIN, COUT, SIDE><<<grid, 128, smem, s>>>(act, n, W, bias, out,
                                                                               r->err)));
    return cudaSuccess;
}

// Forward pass of n snippets (FP32 [n][64][64]); logits into r->z5.  A
// training pass keeps what the backward pass needs (im2col matrices,
// pre-activations, pool argmaxes); an inference pass runs each conv layer as
// one fused conv + bias + ReLU + pool kernel.
cudaError_t forward(gsp_ranker_s *r, const float *x, int n, bool train, cudaStream_t s) {
    for (int l = 0; l < kLayers; l++) {
        const int H = side_of(l), Cin = cin_of(l), Cout = cout_of(l), Kp = kpad(l);
        const int64_t P = (int64_t)n * H * H;
        (void)Cin;
        if (!train) {
            cudaError_t e = cudaSuccess;
            if (l == 0)
                RK_LAUNCH((conv0_pool_kernel<<<blocks_for(P / 8), 256, 0, s>>>(
                    x, n, r->W[0], r->params + r->off.b[0], r->a[0])));
            else if (l == 1)
                e = launch_conv_pool_solo<8, 16, 32>(r, r->a[0], n, r->W[1], r->params + r->off.b[1],
                                                     r->a[1], s, true);
            else
                e = launch_conv_pool_solo<16, 32, 16>(r, r->a[1], n, r->W[2], r->params + r->off.b[2],
                                                      r->a[2], s, true);
            if (e != cudaSuccess) return e;
            continue;
        }
        if (l == 0)
            RK_LAUNCH((im2col_kernel<float, 1><<<blocks_for(P), 256, 0, s>>>(x, n, H, r->col[0])));
        else if (l == 1)
            RK_LAUNCH((im2col_kernel<bf16, 8><<<blocks_for(P), 256, 0, s>>>(r->a[0], n, H, r->col[1])));
        else
            RK_LAUNCH((im2col_kernel<bf16, 16><<<blocks_for(P), 256, 0, s>>>(r->a[1], n, H, r->col[2])));
        cudaError_t e = gemm(r, r->col[l], Kp, r->W[l], Kp, r->z[l], Cout, nullptr, 0, (int)P, Cout,
                             Kp, r->params + r->off.b[l], true, 1, s);
        if (e != cudaSuccess) return e;
        if (l == 0)
            RK_LAUNCH((pool_kernel<8><<<blocks_for(P / 4), 256, 0, s>>>(r->z[0], n, H, r->a[0], r->idx[0])));
        else if (l == 1)
            RK_LAUNCH((pool_kernel<16><<<blocks_for(P / 4), 256, 0, s>>>(r->z[1], n, H, r->a[1], r->idx[1])));
        else
            RK_LAUNCH((pool_kernel<32><<<blocks_for(P / 4), 256, 0, s>>>(r->z[2], n, H, r->a[2], r->idx[2])));
    }
    // fc1 (K = 2048) as a deterministic split-K product: enough K chunks for a
    // CTA per SM even at one column block, at least four 64-wide steps each;
    // the chunks' partial products are summed in order by fc1_finish_kernel
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        (void)cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int mt = (n + 127) / 128;
    const int want = std::max(1, std::min(kFc1Split, std::min(kFc / (4 * 64), nsm / mt)));
    const int64_t zs = (int64_t)r->max_batch * kHid;
    int used = 1;
    // in an inference pass each kernel after the first is launched as a
    // programmatic dependent of the one before (its blocks are scheduled while
    // that kernel drains and wait for its output in wait_prior_grid)
    cudaError_t e = gsp::launch_gemm_bf16(r->a[2], kFc, r->W4, kFc, r->fc1_part, kHid, nullptr, 0, n,
                                          kHid, kFc, nullptr, false, want, r->err, s, zs, &used,
                                          !train);
    if (e != cudaSuccess) return e;
    r->launches++;
    if (!train) {
        e = gsp::launch_dependent(fc1_finish_kernel, dim3(blocks_for((int64_t)n * kHid)), dim3(256),
                                  0, s, (const float *)r->fc1_part, used, zs, n,
                                  (const float *)(r->params + r->off.b[3]), r->z4, r->a4);
        if (e == cudaSuccess)
            e = gsp::launch_dependent(fc2_kernel, dim3((2 * n + 127) / 128), dim3(128), 0, s,
                                      (const bf16 *)r->a4, (const float *)(r->params + r->off.w[4]),
                                      (const float *)(r->params + r->off.b[4]), n, r->z5);
        if (e != cudaSuccess) return e;
        r->launches += 2;
        return cudaSuccess;
    }
    RK_LAUNCH((fc1_finish_kernel<<<blocks_for((int64_t)n * kHid), 256, 0, s>>>(
        r->fc1_part, used, zs, n, r->params + r->off.b[3], r->z4, r->a4)));
    RK_LAUNCH((fc2_kernel<<<(2 * n + 127) / 128, 128, 0, s>>>(r->a4, r->params + r->off.w[4],
                                                              r->params + r->off.b[4], n, r->z5)));
    return cudaSuccess;
}

// Loss, gradients (into r->grads, the oracle's layout) and one Adam step.
cudaError_t backward(gsp_ranker_s *r, const int32_t *labels, int n, float lr, cudaStream_t s) {
    const int n8 = round8(n);
    cudaError_t e = cudaMemsetAsync(r->grads, 0, (size_t)r->off.total * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->g4T, 0, (size_t)kHid * n8 * sizeof(bf16), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->a3T, 0, (size_t)kFc * n8 * sizeof(bf16), s);
    if (e != cudaSuccess) return e;
    RK_LAUNCH((loss_kernel<<<1, 256, 0, s>>>(r->z5, labels, n, r->g5, r->loss)));
    RK_LAUNCH((fc2_back_kernel<<<std::min(n, 152), kHid, 0, s>>>(
        r->g5, r->a4, r->params + r->off.w[4], r->z4, n, r->grads + r->off.w[4],
        r->grads + r->off.b[4], r->g4, r->g4T, n8, r->grads + r->off.b[3])));
    {
        dim3 grid((unsigned)((n + 31) / 32), (unsigned)(kFc / 32));
        RK_LAUNCH((transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(r->a[2], kFc, n, kFc, r->a3T, n8)));
    }
    e = gemm(r, r->g4T, n8, r->a3T, n8, r->grads + r->off.w[3], kFc, nullptr, 0, kHid, kFc, n8,
             nullptr, false, 1, s);
    if (e == cudaSuccess)
        e = gemm(r, r->g4, kHid, r->W4T, kHid, r->ga[2], kFc, nullptr, 0, n, kFc, kHid, nullptr,
                 false, 1, s);
    if (e != cudaSuccess) return e;
    for (int l = kLayers - 1; l >= 0; l--) {
        const int H = side_of(l), Cin = cin_of(l), Cout = cout_of(l), Kp = kpad(l);
        const int64_t P = (int64_t)n * H * H;  // a multiple of 256
        RK_LAUNCH((pool_back_kernel<<<blocks_for(P * Cout), 256, Cout * sizeof(float), s>>>(
            r->ga[l], r->idx[l], r->z[l], n, H, Cout, r->gz[l], r->gzT[l], P,
            r->grads + r->off.b[l])));
        {
            dim3 grid((unsigned)((P + 31) / 32), (unsigned)((Kp + 31) / 32));
            RK_LAUNCH((transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(r->col[l], Kp, P, Kp,
                                                                      r->colT[l], P)));
        }
        e = cudaMemsetAsync(r->dW, 0, (size_t)Cout * Kp * sizeof(float), s);
        if (e != cudaSuccess) return e;
        const int ksteps = (int)(P / 64);
        const int splitk = std::max(1, std::min(ksteps, 4 * 152 / std::max(1, (Kp + 127) / 128)));
        e = gemm(r, r->gzT[l], P, r->colT[l], P, r->dW, Kp, nullptr, 0, Cout, Kp, (int)P, nullptr,
                 false, splitk, s);
        if (e != cudaSuccess) return e;
        RK_LAUNCH((unpack_conv_grad_kernel<<<(Cout * Cin * 9 + 255) / 256, 256, 0, s>>>(
            r->dW, Cin, Cout, Kp, r->grads + r->off.w[l])));
        if (l > 0) {
            e = gemm(r, r->gz[l], Cout, r->WT[l], round8(Cout), r->dcol, Kp, nullptr, 0, (int)P, Kp,
                     Cout, nullptr, false, 1, s);
            if (e != cudaSuccess) return e;
            RK_LAUNCH((col2im_kernel<<<blocks_for(P * Cin), 256, 0, s>>>(r->dcol, n, H, Cin, Kp,
                                                                          r->ga[l - 1])));
        }
    }
    r->step++;
    const double c1 = 1.0 - std::pow(0.9, (double)r->step);
    const double c2 = 1.0 - std::pow(0.999, (double)r->step);
    RK_LAUNCH((adam_kernel<<<blocks_for(r->off.total), 256, 0, s>>>(
        r->params, r->grads, r->m, r->v, r->off.total, lr, 0.9f, 0.999f, 1e-8f, (float)c1,
        (float)c2)));
    return pack(r, s);
}

gsp_status status_of(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GSP_OK;
    gsp::record_error(e, what);
    return e == cudaErrorInvalidValue ? GSP_ERR_INVALID_ARG : GSP_ERR_CUDA;
}

// Snippet of candidate blockIdx.x: out[i][j] = sum over the samples s of time
// bin j (f = max(1, w / 4) samples, bins centred on t + w / 2) of the
// normalised series of row dm - 32 + i, ((D - m) - (c0 + beta j)) / sigma_ref
// (0 in bad blocks, rows with sigma_ref = 0, outside the rows or past Ls),
// divided by sqrt(f).  A bin is summed as exact integer runs inside one search
// block, with the block's trend applied in closed form.
//
// A row of the snippet reads 64 f consecutive samples of D.  The CTA streams
// them through a shared-memory ring of two halves with 1-D bulk copies (one
// per row, 16-byte aligned span [t_al, t_end) around the row's 64 f samples,
// completion counted on the half's mbarrier): thread 0 fills half (b & 1) with
// the S rows of batch b while the warps sum batch b - 1 from the other half,
// S = the rows of this candidate's span that fit a half.  The warps share the
// batch's 2 S half-rows of 32 bins; lane l sums one bin (f is odd except for
// f = 2, so the lanes' strided reads hit distinct banks).  A candidate whose span
// leaves [0, stride) of its rows, or a series that is not 16-byte aligned,
// reads D directly instead (same sums).  Every wait is bounded; a wait that
// gives up sets *err, waits (bounded) for the copies it issued and leaves.
// Bytes per half of the ring: a sweep of 8 to 48 KB halves (and of 128- and
// 256-thread CTAs) over a searched beam's 130k candidates put 24 KB halves and
// 256 threads first, at 4.6 TB/s of snippet reads (three CTAs per SM).
constexpr int kSnipHalf = 24 * 1024;
constexpr long long kSnipBudget = 2000000000ll;

// One run's term of a bin, ((sd - n m) - (n c0 + beta sj)) / sigma_ref, from
// dev = sd - n m (exact; sd the run's sum) and sj = the sum of its in-block
// sample indices, rounded step by step (no contraction into FMAs), so that
// both snippet paths give the same float.
__device__ __forceinline__ float run_term(float dev, int n, int64_t sj, const gsp::BlockParam &q,
                                          float inv) {
    const float t = __fadd_rn(__fmul_rn((float)n, q.c0), __fmul_rn(q.beta, (float)sj));
    return __fmul_rn(__fsub_rn(dev, t), inv);
}

// Positions inside a candidate's rows are int32 offsets from T0 = b0 * B, the
// start of the first search block its bins touch (b0 = max(tlo, 0) / B); a
// block index bi is then relative to b0.  bsh = log2(B) when B is a power of
// two, else -1.
__device__ __forceinline__ int rel_block(int r, int B, int bsh) {
    return bsh >= 0 ? (r >> bsh) : r / B;
}

// Bin [r0, r1) of one row (relative positions, clipped to the searched
// span); src[off + r] is the sample at relative position r and brow[bi] the
// parameters of relative block bi.  At most two runs (f <= B), each summed
// exactly in Acc: int32 (wrapping, exact) when f times the largest D stays
// below 2^31, else int64.
template <typename Acc>
__device__ __forceinline__ float snippet_bin(const int32_t *src, int off, int r0, int r1, int B,
                                             int bsh, const gsp::BlockParam *brow, float inv) {
    float v = 0.0f;
    int s0 = r0;
    while (s0 < r1) {
        const int bi = rel_block(s0, B, bsh), bs = bi * B;
        const int e = min(r1, bs + B);
        const int n = e - s0;
        const gsp::BlockParam q = brow[bi];
        if (q.good) {
            const int32_t *p = src + off + s0;
            Acc sd = 0;  // exact
#pragma unroll 4
            for (int k = 0; k < n; k++) sd += p[k];
            const int64_t sj = (int64_t)n * (s0 - bs) + (int64_t)n * (n - 1) / 2;
            const float dev =
                sizeof(Acc) == 4
                    ? (float)(int32_t)((uint32_t)sd - (uint32_t)n * (uint32_t)q.m)
                    : (float)((int64_t)sd - (int64_t)n * q.m);
            v = __fadd_rn(v, run_term(dev, n, sj, q, inv));
        }
        s0 = e;
    }
    return v;
}

template <int HALF>
__global__ void __launch_bounds__(256) snippet_kernel(
    const int32_t *__restrict__ D, int64_t stride, int ndm, int64_t Ls, int B,
    const gsp::BlockParam *__restrict__ bp, int64_t nb_max, const float *__restrict__ sinv,
    const gsp_cand *__restrict__ cands, const int32_t *__restrict__ order, int64_t dmax,
    float *__restrict__ out, int *err) {
    extern __shared__ __align__(128) int32_t ring[];  // 2 * HALF bytes
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_inv[kS];
    const int64_t ck = order ? order[blockIdx.x] : blockIdx.x;  // this CTA's candidate
    const gsp_cand c = cands[ck];
    const int f = max(1, c.width / 4);
    const int64_t tlo = c.t + c.width / 2 - (int64_t)(kS / 2) * f;  // first sample of bin 0
    const float rs = 1.0f / sqrtf((float)f);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = (int)(blockDim.x >> 5);
    float *o = out + ck * kS * kS;
    // the 16-byte aligned span of every row: samples [t_al, t_end)
    const int64_t t_al = tlo >= 0 ? (tlo & ~(int64_t)3) : -((-tlo + 3) & ~(int64_t)3);
    const int64_t t_end = (tlo + (int64_t)kS * f + 3) & ~(int64_t)3;
    const int64_t rowb64 = (t_end - t_al) * 4;
    const bool bulk = ((reinterpret_cast<uintptr_t>(D) & 15u) == 0) && (stride % 4 == 0) &&
                      t_al >= 0 && t_end <= stride && rowb64 <= HALF;
    const uint32_t rowb = bulk ? (uint32_t)rowb64 : 0u;
    const int S = bulk ? min(kS, (int)(HALF / rowb)) : kS;  // rows per batch
    const int nbatch = (kS + S - 1) / S;
    const int64_t b0 = max(tlo, (int64_t)0) / B;           // first search block of the span
    const int64_t T0 = b0 * B;
    const int alo = (int)(tlo - T0);                       // bin 0 relative to T0
    const int lrel = (int)min(Ls - T0, (int64_t)1 << 30);  // end of the searched span
    const int bsh = (B & (B - 1)) == 0 ? __ffs(B) - 1 : -1;
    const bool narrow = (int64_t)f * dmax < 2147483648ll;  // int32 run sums are exact
    for (int i = tid; i < kS; i += blockDim.x) {
        const int r = c.dm_idx - kS / 2 + i;
        s_inv[i] = (r >= 0 && r < ndm) ? sinv[r] : 0.0f;
    }
    const uint32_t ring0 = ptx::smem_addr(ring);
    const uint32_t bar0 = ptx::smem_addr(&bar[0]);
    if (tid == 0) {
        ptx::mbar_init(bar0, 1);
        ptx::mbar_init(bar0 + 8, 1);
        ptx::fence_barrier_init();
    }
    __syncthreads();
    // thread 0: the copies of batch b into half b & 1 (rows with sigma_ref = 0
    // are not copied); returns the bytes expected on the half's barrier
    auto issue = [&](int b) {
        const int r0 = b * S, n = min(S, kS - r0);
        uint32_t bytes = 0;
        for (int k = 0; k < n; k++) bytes += s_inv[r0 + k] != 0.0f ? rowb : 0u;
        const uint32_t hb = bar0 + 8u * (uint32_t)(b & 1);
        ptx::mbar_arrive_expect_tx(hb, bytes);
        for (int k = 0; k < n; k++) {
            if (s_inv[r0 + k] == 0.0f) continue;
            const int r = c.dm_idx - kS / 2 + r0 + k;
            ptx::bulk_g2s(ring0 + (uint32_t)(b & 1) * HALF + (uint32_t)k * rowb,
                          D + (int64_t)r * stride + t_al, rowb, hb);
        }
    };
    if (bulk && tid == 0) {
        issue(0);
        if (nbatch > 1) issue(1);
    }
    bool ok = true;
    int waited = 0;  // batches whose copies are known to have landed
    for (int b = 0; b < nbatch; b++) {
        const int r0 = b * S, n = min(S, kS - r0);
        if (bulk) {
            const bool done = ptx::mbar_wait(bar0 + 8u * (uint32_t)(b & 1), (uint32_t)((b >> 1) & 1),
                                             kSnipBudget);
            if (!__syncthreads_and(done)) {
                ok = false;
                break;
            }
            waited = b + 1;
        }
        const int32_t *half = ring + (size_t)(b & 1) * (HALF / 4);
        // 2 n half-rows of 32 bins over the warps: warp task wt is row wt / 2,
        // bins 32 (wt % 2) + lane
        for (int wt = warp; wt < 2 * n; wt += nwarps) {
            const int k = wt >> 1, i = r0 + k, j = 32 * (wt & 1) + lane;
            const float inv = s_inv[i];
            float v = 0.0f;
            if (inv != 0.0f) {  // warp-uniform
                const int r = c.dm_idx - kS / 2 + i;
                const gsp::BlockParam *brow = bp + (int64_t)r * nb_max + b0;
                // the ring row holds samples t_al.. (T0 - t_al <= 3); D's row from T0
                const int32_t *src = bulk ? half + (size_t)k * (rowb / 4) : D + (int64_t)r * stride + T0;
                const int off = bulk ? (int)(T0 - t_al) : 0;
                const int r0 = max(alo + j * f, 0), r1 = min(alo + (j + 1) * f, lrel);
                v = narrow ? snippet_bin<int32_t>(src, off, r0, r1, B, bsh, brow, inv)
                           : snippet_bin<int64_t>(src, off, r0, r1, B, bsh, brow, inv);
            }
            o[i * kS + j] = v * rs;
        }
        if (bulk && b + 2 < nbatch) {
            __syncthreads();  // every warp is done with half b & 1
            if (tid == 0) issue(b + 2);
        }
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // the copies of the (at most two) batches issued but not waited for
        for (int b = waited; b < min(nbatch, waited + 2); b++)
            (void)ptx::mbar_wait(bar0 + 8u * (uint32_t)(b & 1), (uint32_t)((b >> 1) & 1), kSnipBudget);
    }
}

// 1 / sigma_ref of every row in FP32 (0 where sigma_ref = 0), once per
// snippet call: FP64 division is slow on this GPU, so the snippet CTAs read
// these instead of dividing per row.
__global__ void inv_sigma_kernel(const double *__restrict__ sref, int ndm, float *__restrict__ sinv) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < ndm; r += gridDim.x * blockDim.x)
        sinv[r] = sref[r] > 0.0 ? (float)(1.0 / sref[r]) : 0.0f;
}

// The order in which the snippet CTAs take the candidates: by time bucket
// (t >> shift), a counting sort.  Candidates close in time share the samples
// of their rows' windows, so CTAs that run together then find them in L2
// whatever the caller's order (gsp_candidates sorts by DM first).  Each CTA
// still writes its own candidate's snippet, so the output does not depend on
// the order within a bucket (which the atomics leave open).
__global__ void time_bucket_count_kernel(const gsp_cand *__restrict__ cands, int n, int shift,
                                         int nbk, uint32_t *__restrict__ hist) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t bk = min(max(cands[k].t >> shift, (int64_t)0), (int64_t)nbk - 1);
        atomicAdd(hist + bk, 1u);
    }
}

// hist[0 .. nbk) -> exclusive prefix (one CTA of 1024 threads; nbk <= 1024)
__global__ void __launch_bounds__(1024) time_bucket_scan_kernel(uint32_t *__restrict__ hist,
                                                                int nbk) {
    __shared__ uint32_t wsum[32];
    const int i = threadIdx.x, lane = i & 31, warp = i >> 5;
    const uint32_t v = i < nbk ? hist[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; w++) off += wsum[w];
    if (i < nbk) hist[i] = off + x - v;
}

__global__ void time_bucket_scatter_kernel(const gsp_cand *__restrict__ cands, int n, int shift,
                                           int nbk, uint32_t *__restrict__ next,
                                           int32_t *__restrict__ order) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t bk = min(max(cands[k].t >> shift, (int64_t)0), (int64_t)nbk - 1);
        order[atomicAdd(next + bk, 1u)] = k;
    }
}

// Block-local inclusive prefix sums of a series, for snippets of wide bins:
// P[r][b B + k] = sum of D[r][b B .. b B + k] (mod 2^32) for every search block
// b < nb of every row.  A run of samples inside one block then sums to the
// difference of two entries, exact whenever the run's true sum lies within
// int32 (at most f samples of at most nchan * 255 each).  One CTA per (row,
// block) job, grid-stride; each warp scans 128 consecutive samples of a
// 1024-sample chunk with shuffles, the warps' totals are combined through
// shared memory, and a carry runs across the chunks of a block.
__global__ void __launch_bounds__(256) block_prefix_kernel(const int32_t *__restrict__ D,
                                                           int64_t stride, int ndm, int64_t nb,
                                                           int B, int32_t *__restrict__ P,
                                                           int64_t pstride) {
    __shared__ uint32_t wsum[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t job = blockIdx.x; job < (int64_t)ndm * nb; job += gridDim.x) {
        const int64_t r = job / nb, b = job - r * nb;
        const int32_t *src = D + r * stride + b * B;
        int32_t *dst = P + r * pstride + b * B;
        uint32_t carry = 0;  // sum of the block's samples before this chunk
        for (int c0 = 0; c0 < B; c0 += 1024) {
            uint32_t v[4], run = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int idx = c0 + warp * 128 + k * 32 + lane;
                uint32_t x = idx < B ? (uint32_t)__ldg(src + idx) : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                v[k] = x + run;
                run += __shfl_sync(0xffffffffu, x, 31);
            }
            if (lane == 0) wsum[warp] = run;
            __syncthreads();
            uint32_t off = carry, tot = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                off += w < warp ? wsum[w] : 0u;
                tot += wsum[w];
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int idx = c0 + warp * 128 + k * 32 + lane;
                if (idx < B) dst[idx] = (int32_t)(v[k] + off);
            }
            carry += tot;
            __syncthreads();  // wsum is rewritten by the next chunk
        }
    }
}

// Bin [r0, r1) of one row (relative positions as in snippet_bin) from the
// block-local prefix sums, pc[r] the entry at relative position r: at most two
// runs (f <= B), the second one starting a block; the three prefix entries are
// loaded before any is used.  Run sums are differences mod 2^32, exact since
// they lie within int32; the same run_term arithmetic as snippet_bin, so the
// same float.
__device__ __forceinline__ float snippet_bin_prefix(const int32_t *__restrict__ pc, int r0, int r1,
                                                    int B, int bsh, const gsp::BlockParam *brow,
                                                    float inv) {
    if (r0 >= r1) return 0.0f;
    const int bi = rel_block(r0, B, bsh), bs = bi * B, be = bs + B;
    const bool split = r1 > be;
    const int e1 = split ? be : r1;
    const uint32_t p_lo = r0 > bs ? (uint32_t)__ldg(pc + r0 - 1) : 0u;
    const uint32_t p_hi = (uint32_t)__ldg(pc + e1 - 1);
    const uint32_t p_2 = split ? (uint32_t)__ldg(pc + r1 - 1) : 0u;
    float v = 0.0f;
    {
        const int n = e1 - r0;
        const gsp::BlockParam q = brow[bi];
        if (q.good) {
            const float dev = (float)(int32_t)(p_hi - p_lo - (uint32_t)n * (uint32_t)q.m);
            const int64_t sj = (int64_t)n * (r0 - bs) + (int64_t)n * (n - 1) / 2;
            v = __fadd_rn(v, run_term(dev, n, sj, q, inv));
        }
    }
    if (split) {  // [be, r1) at the start of block bi + 1
        const int n = r1 - be;
        const gsp::BlockParam q = brow[bi + 1];
        if (q.good) {
            const float dev = (float)(int32_t)(p_2 - (uint32_t)n * (uint32_t)q.m);
            const int64_t sj = (int64_t)n * (n - 1) / 2;
            v = __fadd_rn(v, run_term(dev, n, sj, q, inv));
        }
    }
    return v;
}

// Snippets from the block-local prefix sums P of the series D (see
// snippet_kernel for the definition): two to three 4-byte loads per bin instead
// of f.  CTA per candidate; warp w builds rows w, w + 8, ..., lane l bins l and
// l + 32.  A candidate whose bins could span more than two blocks (f > B) or
// whose run sums could leave int32 sums its bins from D directly.
__global__ void __launch_bounds__(256) snippet_prefix_kernel(
    const int32_t *__restrict__ P, int64_t pstride, const int32_t *__restrict__ D, int64_t stride,
    int ndm, int64_t Ls, int B, const gsp::BlockParam *__restrict__ bp, int64_t nb_max,
    const float *__restrict__ sinv, const gsp_cand *__restrict__ cands,
    const int32_t *__restrict__ order, int64_t dmax, float *__restrict__ out) {
    const int64_t ck = order ? order[blockIdx.x] : blockIdx.x;  // this CTA's candidate
    const gsp_cand c = cands[ck];
    const int f = max(1, c.width / 4);
    const bool via_prefix = f <= B && (int64_t)f * dmax < 2147483648ll;
    const int64_t tlo = c.t + c.width / 2 - (int64_t)(kS / 2) * f;  // first sample of bin 0
    const int64_t b0 = max(tlo, (int64_t)0) / B, T0 = b0 * B;
    const int alo = (int)(tlo - T0);
    const int lrel = (int)min(Ls - T0, (int64_t)1 << 30);
    const int bsh = (B & (B - 1)) == 0 ? __ffs(B) - 1 : -1;
    const float rs = 1.0f / sqrtf((float)f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = (int)(blockDim.x >> 5);
    float *o = out + ck * kS * kS;
    const int ra0 = max(alo + lane * f, 0), ra1 = min(alo + (lane + 1) * f, lrel);
    const int rb0 = max(alo + (32 + lane) * f, 0), rb1 = min(alo + (33 + lane) * f, lrel);
    for (int i = warp; i < kS; i += nwarps) {
        const int r = c.dm_idx - kS / 2 + i;
        const float inv = (r >= 0 && r < ndm) ? sinv[r] : 0.0f;
        float v0 = 0.0f, v1 = 0.0f;
        if (inv != 0.0f) {  // warp-uniform
            const gsp::BlockParam *brow = bp + (int64_t)r * nb_max + b0;
            if (via_prefix) {
                const int32_t *pc = P + (int64_t)r * pstride + T0;
                v0 = snippet_bin_prefix(pc, ra0, ra1, B, bsh, brow, inv);
                v1 = snippet_bin_prefix(pc, rb0, rb1, B, bsh, brow, inv);
            } else {
                const int32_t *dc = D + (int64_t)r * stride + T0;
                v0 = snippet_bin<int64_t>(dc, 0, ra0, ra1, B, bsh, brow, inv);
                v1 = snippet_bin<int64_t>(dc, 0, rb0, rb1, B, bsh, brow, inv);
            }
        }
        o[i * kS + lane] = v0 * rs;
        o[i * kS + 32 + lane] = v1 * rs;
    }
}

}  // namespace

extern "C" {

gsp_status gsp_ranker_snippets(gsp_plan_t p, const int32_t *d_D, int64_t stride,
                               const gsp_cand *d_cands, int32_t n, float *d_out, void *stream) {
    if (!p || !d_D || !d_cands || !d_out || n < 0) return GSP_ERR_INVALID_ARG;
    if (!p->have_search) return GSP_ERR_STATE;
    if (n == 0) return GSP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int B = p->desc.block_len;
    const int64_t Ls = p->last_nb * B;
    const int64_t dmax = (int64_t)p->desc.nchan * 255;
    // prefix sums pay off once the candidates' direct reads (64 x 64 f samples
    // each; f is taken as 4 here, the narrowest bins that fill a 16-byte
    // chunk) exceed building them (one read and one write of the series)
    const bool big = (int64_t)n * kS * kS * 4 >= 2 * (int64_t)p->desc.ndm * Ls;
    const bool use_prefix = Ls > 0 && (p->snippet_path == 2 || (p->snippet_path == 0 && big));
    // CTAs take the candidates in time order (buckets of 2^shift samples, at
    // most 1024 buckets over the series)
    int shift = 12;
    while (shift < 40 && (std::max<int64_t>(Ls, 1) >> shift) >= 1024) shift++;
    const int nbk = (int)std::min<int64_t>(1024, (std::max<int64_t>(Ls, 1) >> shift) + 1);
    if ((size_t)n > p->d_order_elems) {
        cudaFree(p->d_order);
        p->d_order = nullptr;
        p->d_order_elems = 0;
        if (cudaMalloc((void **)&p->d_order, (size_t)n * sizeof(int32_t)) != cudaSuccess) {
            (void)cudaGetLastError();
            return GSP_ERR_OOM;
        }
        p->d_order_elems = (size_t)n;
    }
    if (!p->d_order_hist &&
        cudaMalloc((void **)&p->d_order_hist, 1024 * sizeof(uint32_t)) != cudaSuccess) {
        (void)cudaGetLastError();
        p->d_order_hist = nullptr;
        return GSP_ERR_OOM;
    }
    if (!p->d_sinv &&
        cudaMalloc((void **)&p->d_sinv, (size_t)p->desc.ndm * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        p->d_sinv = nullptr;
        return GSP_ERR_OOM;
    }
    {
        const int g = (int)std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)p->num_sms * 4);
        cudaError_t e = cudaMemsetAsync(p->d_order_hist, 0, (size_t)nbk * sizeof(uint32_t), s);
        if (e == cudaSuccess) {
            time_bucket_count_kernel<<<g, 256, 0, s>>>(d_cands, n, shift, nbk, p->d_order_hist);
            time_bucket_scan_kernel<<<1, 1024, 0, s>>>(p->d_order_hist, nbk);
            time_bucket_scatter_kernel<<<g, 256, 0, s>>>(d_cands, n, shift, nbk, p->d_order_hist,
                                                         p->d_order);
            inv_sigma_kernel<<<(p->desc.ndm + 255) / 256, 256, 0, s>>>(p->d_sref, p->desc.ndm,
                                                                     p->d_sinv);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return status_of(e, "snippet order launch");
    }
    if (use_prefix) {
        const int64_t pstride = (Ls + 3) & ~(int64_t)3;
        const size_t need = (size_t)p->desc.ndm * (size_t)pstride;
        if (need > p->d_prefix_elems) {
            cudaFree(p->d_prefix);
            p->d_prefix = nullptr;
            p->d_prefix_elems = 0;
            p->prefix_seq = 0;
            if (cudaMalloc((void **)&p->d_prefix, need * sizeof(int32_t)) != cudaSuccess) {
                (void)cudaGetLastError();
                return GSP_ERR_OOM;
            }
            p->d_prefix_elems = need;
        }
        if (p->prefix_seq != p->search_seq || p->prefix_src != d_D || p->prefix_src_stride != stride ||
            p->prefix_stride != pstride) {
            const int64_t jobs = (int64_t)p->desc.ndm * p->last_nb;
            const int grid = (int)std::min<int64_t>(jobs, (int64_t)p->num_sms * 8);
            block_prefix_kernel<<<grid, 256, 0, s>>>(d_D, stride, p->desc.ndm, p->last_nb, B,
                                                      p->d_prefix, pstride);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return status_of(e, "prefix launch");
            p->prefix_seq = p->search_seq;
            p->prefix_src = d_D;
            p->prefix_src_stride = stride;
            p->prefix_stride = pstride;
        }
        snippet_prefix_kernel<<<n, 256, 0, s>>>(p->d_prefix, pstride, d_D, stride, p->desc.ndm, Ls,
                                                B, p->d_bparam, p->nb_max, p->d_sinv, d_cands,
                                                p->d_order, dmax, d_out);
        return status_of(cudaGetLastError(), "snippet launch");
    }
    {
        cudaError_t e = gsp::ensure_kernel_smem(
            reinterpret_cast<const void *>(snippet_kernel<kSnipHalf>), 2 * kSnipHalf, true);
        if (e != cudaSuccess) return status_of(e, "snippet attributes");
    }
    snippet_kernel<kSnipHalf><<<n, 256, 2 * kSnipHalf, s>>>(
        d_D, stride, p->desc.ndm, Ls, B, p->d_bparam, p->nb_max, p->d_sinv, d_cands, p->d_order,
        dmax, d_out, p->d_err);
    return status_of(cudaGetLastError(), "snippet launch");
}

int64_t gsp_ranker_num_params(void) { return offsets().total; }

gsp_status gsp_ranker_create(gsp_ranker_t *out, int32_t max_batch, uint64_t seed) {
    if (!out || max_batch < 1 || max_batch > 4096) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    gsp_ranker_s *r = new (std::nothrow) gsp_ranker_s();
    if (!r) return GSP_ERR_OOM;
    r->max_batch = max_batch;
    r->off = offsets();
    const int Bm = max_batch, B8 = round8(Bm);
    const int64_t T = r->off.total;
    bool ok = ralloc(r, &r->params, T) && ralloc(r, &r->grads, T) && ralloc(r, &r->m, T) &&
              ralloc(r, &r->v, T) && ralloc(r, &r->W4, (size_t)kHid * kFc) &&
              ralloc(r, &r->W4T, (size_t)kHid * kFc) && ralloc(r, &r->z4, (size_t)Bm * kHid) &&
              ralloc(r, &r->a4, (size_t)Bm * kHid) && ralloc(r, &r->z5, (size_t)Bm * 2) &&
              ralloc(r, &r->g5, (size_t)Bm * 2) && ralloc(r, &r->g4, (size_t)Bm * kHid) &&
              ralloc(r, &r->g4T, (size_t)kHid * B8) && ralloc(r, &r->a3T, (size_t)kFc * B8) &&
              ralloc(r, &r->loss, 1) && ralloc(r, &r->err, 1);
    size_t dcol = 0, dw = 0;
    for (int l = 0; ok && l < kLayers; l++) {
        const int H = side_of(l), Cout = cout_of(l), Kp = kpad(l);
        const int64_t P = (int64_t)Bm * H * H;
        ok = ralloc(r, &r->W[l], (size_t)Cout * Kp) && ralloc(r, &r->WT[l], (size_t)Kp * round8(Cout)) &&
             ralloc(r, &r->col[l], (size_t)P * Kp) && ralloc(r, &r->colT[l], (size_t)P * Kp) &&
             ralloc(r, &r->z[l], (size_t)P * Cout) && ralloc(r, &r->a[l], (size_t)P / 4 * Cout) &&
             ralloc(r, &r->idx[l], (size_t)P / 4 * Cout) && ralloc(r, &r->gz[l], (size_t)P * Cout) &&
             ralloc(r, &r->gzT[l], (size_t)P * Cout) && ralloc(r, &r->ga[l], (size_t)P / 4 * Cout);
        if (l > 0) dcol = std::max(dcol, (size_t)P * Kp);
        dw = std::max(dw, (size_t)Cout * Kp);
    }
    ok = ok && ralloc(r, &r->dcol, dcol) && ralloc(r, &r->dW, dw) &&
         ralloc(r, &r->fc1_part, (size_t)kFc1Split * Bm * kHid);
    if (!ok) {
        free_ranker(r);
        return GSP_ERR_OOM;
    }
    // He-uniform weights, zero biases, from a 64-bit LCG (host)
    std::vector<float> h((size_t)T, 0.0f);
    uint64_t st = seed * 6364136223846793005ull + 1442695040888963407ull;
    for (int i = 0; i < 5; i++) {
        const int fan_in = i < 3 ? 9 * cin_of(i) : (i == 3 ? kFc : kHid);
        const double lim = std::sqrt(6.0 / fan_in);
        for (int64_t j = 0; j < kWsize[i]; j++) {
            st = st * 6364136223846793005ull + 1442695040888963407ull;
            const double u = (double)(st >> 11) * (1.0 / 9007199254740992.0);
            h[(size_t)(r->off.w[i] + j)] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    cudaError_t e = cudaMemcpy(r->params, h.data(), (size_t)T * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->m, 0, (size_t)T * 4);
    if (e == cudaSuccess) e = cudaMemset(r->v, 0, (size_t)T * 4);
    if (e == cudaSuccess) e = cudaMemset(r->err, 0, sizeof(int));
    if (e == cudaSuccess) e = pack(r, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        gsp::record_error(e, "ranker init");
        free_ranker(r);
        return GSP_ERR_CUDA;
    }
    *out = r;
    return GSP_OK;
}

gsp_status gsp_ranker_destroy(gsp_ranker_t r) {
    if (!r) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    free_ranker(r);
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

gsp_status gsp_ranker_set_params(gsp_ranker_t r, const float *host_params) {
    if (!r || !host_params) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpy(r->params, host_params, (size_t)r->off.total * 4,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(r->m, 0, (size_t)r->off.total * 4);
    if (e == cudaSuccess) e = cudaMemset(r->v, 0, (size_t)r->off.total * 4);
    if (e == cudaSuccess) e = pack(r, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    r->step = 0;
    return status_of(e, "ranker set params");
}

gsp_status gsp_ranker_get_params(gsp_ranker_t r, float *host_params, float *host_grads) {
    if (!r) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && host_params)
        e = cudaMemcpy(host_params, r->params, (size_t)r->off.total * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_grads)
        e = cudaMemcpy(host_grads, r->grads, (size_t)r->off.total * 4, cudaMemcpyDeviceToHost);
    return status_of(e, "ranker get params");
}

gsp_status gsp_ranker_forward(gsp_ranker_t r, const float *d_x, int32_t n, float *d_logits,
                              void *stream) {
    if (!r || !d_x || n < 1 || n > r->max_batch) return GSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    r->launches = 0;
    cudaError_t e = forward(r, d_x, n, false, s);
    r->last_n = n;
    r->last_pass = 1;
    if (e == cudaSuccess && d_logits)
        e = cudaMemcpyAsync(d_logits, r->z5, (size_t)n * 2 * 4, cudaMemcpyDeviceToDevice, s);
    return status_of(e, "ranker forward");
}

gsp_status gsp_ranker_train_step(gsp_ranker_t r, const float *d_x, const int32_t *d_labels,
                                 int32_t n, float lr, float *d_loss, void *stream) {
    if (!r || !d_x || !d_labels || n < 1 || n > r->max_batch || !(lr >= 0.0f))
        return GSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    r->launches = 0;
    cudaError_t e = forward(r, d_x, n, true, s);
    if (e == cudaSuccess) e = backward(r, d_labels, n, lr, s);
    r->last_n = n;
    r->last_pass = 2;
    if (e == cudaSuccess && d_loss)
        e = cudaMemcpyAsync(d_loss, r->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    return status_of(e, "ranker train step");
}

gsp_status gsp_ranker_finish(gsp_ranker_t r, void *stream) {
    if (!r) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, r->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_of(e, "ranker finish");
    if (flag) {
        cudaMemset(r->err, 0, sizeof(int));
        return GSP_ERR_TIMEOUT;
    }
    return GSP_OK;
}

int32_t gsp_ranker_launches(gsp_ranker_t r) { return r ? r->launches : -1; }

gsp_status gsp_ranker_tensor(gsp_ranker_t r, const char *name, void *host_out, int64_t cap_bytes,
                             int64_t *bytes) {
    if (!r || !name || !bytes || cap_bytes < 0) return GSP_ERR_INVALID_ARG;
    if (r->last_pass == 0) return GSP_ERR_STATE;
    const int64_t n = r->last_n;
    const void *src = nullptr;
    int64_t size = 0;
    bool train_only = false;
    const std::string nm(name);
    for (int l = 0; l < kLayers && !src; l++) {
        const int64_t H = side_of(l), H2 = H / 2, C = cout_of(l);
        const std::string d = std::to_string(l);
        if (nm == "a" + d) { src = r->a[l]; size = n * H2 * H2 * C * 2; }
        else if (nm == "z" + d) { src = r->z[l]; size = n * H * H * C * 4; train_only = true; }
        else if (nm == "idx" + d) { src = r->idx[l]; size = n * H2 * H2 * C; train_only = true; }
        else if (nm == "ga" + d) { src = r->ga[l]; size = n * H2 * H2 * C * 4; train_only = true; }
        else if (nm == "gz" + d) { src = r->gz[l]; size = n * H * H * C * 2; train_only = true; }
    }
    if (!src) {
        if (nm == "z4") { src = r->z4; size = n * kHid * 4; }
        else if (nm == "a4") { src = r->a4; size = n * kHid * 2; }
        else if (nm == "z5") { src = r->z5; size = n * 2 * 4; }
        else if (nm == "g5") { src = r->g5; size = n * 2 * 4; train_only = true; }
        else if (nm == "g4") { src = r->g4; size = n * kHid * 2; train_only = true; }
        else return GSP_ERR_INVALID_ARG;
    }
    if (train_only && r->last_pass != 2) return GSP_ERR_STATE;
    *bytes = size;
    if (!host_out || cap_bytes < size) return GSP_ERR_CAPACITY;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host_out, src, (size_t)size, cudaMemcpyDeviceToHost);
    return status_of(e, "ranker tensor");
}

}  // extern "C"
