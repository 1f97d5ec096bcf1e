// Single-pulse search of dedispersed series (the step after dedispersion in
// the pipeline of Sec. 2.1-2.2; the paper names it, the steps are these):
//   1. blocks [bB, (b+1)B) of each DM row; least-squares line per block from
//      exact integer sums, residual RMS sigma_b (block_stats_kernel);
//   2. sigma_ref = lower median of sigma_b per row, bad-block flags
//      (row_sigma_kernel);
//   3. boxcar S/N over the widths, best width per sample, threshold and the
//      per-window maximum, appended to the candidate buffer (boxcar_kernel).
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "gsp_internal.cuh"

namespace gsp {

namespace {

constexpr int kStatThreads = 256;
constexpr int kBoxThreads = 256;
constexpr int kChunk = 1024;  // samples per boxcar sub-chunk

struct WidthTable {
    int w[kMaxWidths];
    float tri[kMaxWidths];  // w (w - 1) / 2
    int n;
    int wmax;
};

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Closed form of the block's least-squares line from exact integer sums
// S0 = sum D_j, S1 = sum j D_j, S2 = sum D_j^2 (j = 0..B-1), in exact 128-bit
// integers U = B S2 - S0^2, V = 2 S1 - (B-1) S0 and
// N = U (B^2 - 1) - 3 V^2 = B^2 (B^2 - 1) * sigma_b^2, so that
// sigma_b = sqrt(N / (B^2 (B^2 - 1))) (population RMS of the residual from
// the line) and beta = 6 V / (B (B^2 - 1)).
__device__ __forceinline__ void finish_block(long long s0, long long s1, long long s2, int B,
                                             int64_t idx, double *__restrict__ sigma_b,
                                             BlockParam *__restrict__ bparam) {
    const __int128 Bi = B;
    const __int128 bb1 = Bi * Bi - 1;
    double sig = 0.0, beta = 0.0;
    if (B > 1) {
        const __int128 U = Bi * (__int128)s2 - (__int128)s0 * (__int128)s0;
        const __int128 V = 2 * (__int128)s1 - (Bi - 1) * (__int128)s0;
        const __int128 N = U * bb1 - 3 * V * V;
        const double den = (double)B * (double)B * (double)bb1;
        sig = N > 0 ? sqrt((double)N / den) : 0.0;
        beta = 6.0 * (double)V / ((double)B * (double)bb1);
    }
    const double mean = (double)s0 / (double)B;
    const long long m = (long long)floor(mean + 0.5);
    const double jbar = 0.5 * (double)(B - 1);
    const double c0 = (double)(s0 - m * (long long)B) / (double)B - beta * jbar;
    sigma_b[idx] = sig;
    BlockParam bp;
    bp.m = (int32_t)m;
    bp.c0 = (float)c0;
    bp.beta = (float)beta;
    bp.good = 1;
    bparam[idx] = bp;
}

// Step 1.  One CTA per (block, row).  Exact int64 sums S0 = sum D_j,
// S1 = sum j D_j, S2 = sum D_j^2 over j = 0..B-1, then in exact 128-bit
// integers U = B S2 - S0^2, V = 2 S1 - (B-1) S0 and
// N = U (B^2 - 1) - 3 V^2 = B^2 (B^2 - 1) * sigma_b^2, so that
// sigma_b = sqrt(N / (B^2 (B^2 - 1))) (population RMS of the residual from
// the least-squares line) and beta = 6 V / (B (B^2 - 1)).
__global__ void __launch_bounds__(kStatThreads) block_stats_kernel(
    const int32_t *__restrict__ D, int64_t stride, int B, int64_t nb_max,
    double *__restrict__ sigma_b, BlockParam *__restrict__ bparam) {
    const int b = blockIdx.x;
    const int row = blockIdx.y;
    const int32_t *d = D + (int64_t)row * stride + (int64_t)b * B;
    long long s0 = 0, s1 = 0, s2 = 0;
    for (int j = threadIdx.x; j < B; j += kStatThreads) {
        const long long v = d[j];
        s0 += v;
        s1 += (long long)j * v;
        s2 += v * v;
    }
    s0 = warp_sum_ll(s0);
    s1 = warp_sum_ll(s1);
    s2 = warp_sum_ll(s2);
    __shared__ long long red[3][kStatThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s0;
        red[1][wid] = s1;
        red[2][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    s0 = s1 = s2 = 0;
    for (int i = 0; i < kStatThreads / 32; i++) {
        s0 += red[0][i];
        s1 += red[1][i];
        s2 += red[2][i];
    }
    finish_block(s0, s1, s2, B, (int64_t)row * nb_max + b, sigma_b, bparam);
}

// Step 1 when the dedispersion kernel has already accumulated the exact block
// sums (bsum[row][b] = {S0, S1, S2}): one thread per (row, block).
__global__ void __launch_bounds__(256) block_params_kernel(
    const unsigned long long *__restrict__ bsum, int64_t nb, int B, int64_t nb_max, int ndm,
    double *__restrict__ sigma_b, BlockParam *__restrict__ bparam) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb * ndm) return;
    const int row = (int)(g / nb);
    const int64_t b = g - (int64_t)row * nb;
    const unsigned long long *q = bsum + ((int64_t)row * nb_max + b) * 3;
    finish_block((long long)q[0], (long long)q[1], (long long)q[2], B, (int64_t)row * nb_max + b,
                 sigma_b, bparam);
}

// Step 2.  One CTA per row: lower median of the nb block sigmas (bitonic sort
// in shared memory, or rank counting when nb exceeds the shared buffer), bad
// flags, and the per-width S/N scale 1 / (sigma_ref sqrt(w)).
constexpr int kSortMax = 4096;  // 32 KB of doubles, within the default limit

__global__ void __launch_bounds__(512) row_sigma_kernel(
    const double *__restrict__ sigma_b, int64_t nb, int64_t nb_max, double bad_lo,
    double bad_hi, WidthTable wt, double *__restrict__ sref_out, float *__restrict__ scale_out,
    uint8_t *__restrict__ bad_out, BlockParam *__restrict__ bparam) {
    extern __shared__ double sbuf[];
    __shared__ double s_ref;
    const int row = blockIdx.x;
    const double *sg = sigma_b + (int64_t)row * nb_max;
    const int64_t k = (nb - 1) / 2;
    if (nb <= kSortMax) {
        int n2 = 1;
        while (n2 < nb) n2 <<= 1;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) sbuf[i] = i < nb ? sg[i] : DBL_MAX;
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                    const int jx = i ^ stride;
                    if (jx > i) {
                        const bool up = (i & size) == 0;
                        const double a = sbuf[i], c = sbuf[jx];
                        if ((a > c) == up) {
                            sbuf[i] = c;
                            sbuf[jx] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) s_ref = sbuf[k];
    } else {
        // rank of element i: #(smaller) + #(equal with lower index)
        for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
            const double v = sg[i];
            int64_t r = 0;
            for (int64_t q = 0; q < nb; q++) {
                const double u = sg[q];
                r += (u < v) || (u == v && q < i);
            }
            if (r == k) s_ref = v;
        }
    }
    __syncthreads();
    const double sref = s_ref;
    if (threadIdx.x == 0) sref_out[row] = sref;
    if (threadIdx.x < wt.n)
        scale_out[(int64_t)row * wt.n + threadIdx.x] =
            sref > 0.0 ? (float)(1.0 / (sref * sqrt((double)wt.w[threadIdx.x]))) : 0.0f;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
        const double v = sg[b];
        const bool bad = !(sref > 0.0) || v < bad_lo * sref || v > bad_hi * sref;
        bad_out[(int64_t)row * nb_max + b] = bad ? 1 : 0;
        bparam[(int64_t)row * nb_max + b].good = bad ? 0 : 1;
    }
}

struct Best {
    float snr;
    int64_t t;
    int w;
};

__device__ __forceinline__ bool better(const Best &a, const Best &b) {
    // larger S/N wins; equal S/N: smaller t
    return a.snr > b.snr || (a.snr == b.snr && a.t < b.t);
}

// Step 3.  One CTA per (candidate window, row).  The window's samples are
// processed in sub-chunks of kChunk: exact uint32 prefix sums of the integer
// series y = D - m_b (0 in bad blocks) give every boxcar's integer sum
// Y(t, w); the fitted-line part Cr(t, w) = sum (c0_b + beta_b j) over the
// same samples is evaluated in closed form per block segment; then
// S/N = (Y - Cr) / (sigma_ref sqrt(w)).
// The default width set {1,2,3,4,6,9,14,20,30,45,70,100,150} as compile-time
// constants (immediate shared-memory offsets in the specialised kernel).
__host__ __device__ constexpr int default_width(int i) {
    return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 3 : i == 3 ? 4 : i == 4 ? 6 : i == 5 ? 9
         : i == 6 ? 14 : i == 7 ? 20 : i == 8 ? 30 : i == 9 ? 45 : i == 10 ? 70
         : i == 11 ? 100 : 150;
}
constexpr int kNumDefaultWidths = 13;

template <bool kWriteSnr, bool kDefaultW = false>
__global__ void __launch_bounds__(kBoxThreads) boxcar_kernel(
    const int32_t *__restrict__ D, int64_t stride, int64_t Ls, int B, int64_t nb_max,
    int64_t t_offset, int64_t win_len, int64_t k0, int64_t nwin, int wpc, WidthTable wt,
    const BlockParam *__restrict__ bparam, const float *__restrict__ scale, float threshold,
    float *__restrict__ snr_out, gsp_cand *__restrict__ cands,
    unsigned long long *__restrict__ ncand, int64_t max_cands,
    gsp_cand *__restrict__ slots = nullptr) {
    extern __shared__ uint32_t sP[];  // prefix sums, kChunk + wmax entries
    __shared__ uint32_t warp_tot[kBoxThreads / 32];
    __shared__ Best wbest[kBoxThreads / 32];
    __shared__ float s_scale[kMaxWidths];
    const int row = blockIdx.y;
    const int32_t *d = D + (int64_t)row * stride;
    const BlockParam *bp = bparam + (int64_t)row * nb_max;
    const int nb = (int)(Ls / B);
    if (threadIdx.x < wt.n) s_scale[threadIdx.x] = scale[(int64_t)row * wt.n + threadIdx.x];
    __syncthreads();
    const bool live = s_scale[0] != 0.0f;
    float sc[kNumDefaultWidths];
#pragma unroll
    for (int iw = 0; iw < kNumDefaultWidths; iw++) sc[iw] = kDefaultW ? s_scale[iw] : 0.0f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // samples per thread in the prefix phase: a sub-chunk plus the widest boxcar
    // minus one (150 for the default widths, at most 1024)
    constexpr int kPer = (kChunk + (kDefaultW ? 150 : 1024) + kBoxThreads - 1) / kBoxThreads;
    // this CTA's windows wi in [wfirst, wlast) of the row (CTAs of a few windows
    // each: a CTA per window spent most of its time being launched)
    const int64_t wfirst = (int64_t)blockIdx.x * wpc;
    const int64_t wlast = min(wfirst + (int64_t)wpc, nwin);
    for (int64_t wi = wfirst; wi < wlast; wi++) {
    const int64_t win = k0 + wi;
    int64_t ws = win * win_len - t_offset, we = ws + win_len;
    if (ws < 0) ws = 0;
    if (we > Ls) we = Ls;
    Best run{-FLT_MAX, 0, 0};
    bool have = false;

    for (int64_t s = ws; s < we; s += kChunk) {
        const int64_t e = min(s + (int64_t)kChunk, we);
        const int64_t pe = min(e + (int64_t)wt.wmax - 1, Ls);  // prefix covers [s, pe)
        const int len = (int)(pe - s);
        const int64_t b_s = s / B;                 // block of the sub-chunk's first sample
        const int j_s = (int)(s - b_s * B);        // its index inside that block
        // integer series y = D - m_b (0 in bad blocks), per-thread consecutive segment
        const int per = (len + kBoxThreads - 1) / kBoxThreads;
        const int i0 = threadIdx.x * per;
        uint32_t y[kPer];
        uint32_t loc = 0;
        {
            const int rel = j_s + i0;
            int b = (int)b_s + rel / B;
            int j = rel - (b - (int)b_s) * B;
            BlockParam q = bp[min(b, nb - 1)];
#pragma unroll
            for (int r = 0; r < kPer; r++) {
                y[r] = 0;
                if (r < per && i0 + r < len) {
                    if (j == B) {
                        b++;
                        j = 0;
                        q = bp[b];
                    }
                    y[r] = q.good ? (uint32_t)(d[s + i0 + r] - q.m) : 0u;
                    loc += y[r];
                    j++;
                }
            }
        }
        // block exclusive scan of the per-thread totals
        uint32_t incl = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        uint32_t run_p = incl - loc;
        for (int q = 0; q < wid; q++) run_p += warp_tot[q];
#pragma unroll
        for (int r = 0; r < kPer; r++) {
            if (r < per && i0 + r < len) {
                sP[i0 + r] = run_p;
                run_p += y[r];
            }
        }
        if (threadIdx.x == kBoxThreads - 1) sP[len] = run_p;  // running total at pe
        __syncthreads();

        Best mine{-FLT_MAX, INT64_MAX, 0};
        // this thread's first sample, as block offset bo from b_s and index j1 in
        // that block; both advance by kBoxThreads samples per iteration (no division)
        int bo = (j_s + (int)threadIdx.x) / B;
        int j1 = j_s + (int)threadIdx.x - bo * B;
        // samples i <= fit150 (fitw) have every default (every) boxcar inside the series
        const int fit150 = (int)max((int64_t)-1, min((int64_t)kChunk, Ls - 150 - s));
        const int fitw = (int)max((int64_t)-1, min((int64_t)kChunk, Ls - (int64_t)wt.wmax - s));
        for (int i = threadIdx.x; i < (int)(e - s); i += kBoxThreads, j1 += kBoxThreads) {
            while (j1 >= B) {
                j1 -= B;
                bo++;
            }
            const int64_t t = s + i;
            const int b = (int)b_s + bo;
            const BlockParam q = bp[b];
            const int rem = B - j1;                 // samples left in block b
            const float g = q.good ? q.c0 + q.beta * (float)j1 : 0.0f;
            const float beta1 = q.good ? q.beta : 0.0f;
            const uint32_t p0 = sP[i];
            float bsnr = -FLT_MAX;
            int bw = 0;
            if (kDefaultW && !kWriteSnr && i <= fit150 && 150 <= rem) {
                // default widths inside block b: the maximum S/N first (one max per
                // width); the width that reaches it is recovered only when it
                // passes the threshold (rare)
                float v[kNumDefaultWidths];
#pragma unroll
                for (int iw = 0; iw < kNumDefaultWidths; iw++) {
                    const int w = default_width(iw);
                    const int32_t Y = (int32_t)(sP[i + w] - p0);
                    const float cr = (float)w * g + beta1 * (0.5f * (float)w * (float)(w - 1));
                    v[iw] = ((float)Y - cr) * sc[iw];
                    bsnr = fmaxf(bsnr, v[iw]);
                }
                if (bsnr >= threshold) {
                    // first width reaching the maximum (ties: the smaller width)
#pragma unroll
                    for (int iw = kNumDefaultWidths - 1; iw >= 0; iw--)
                        if (v[iw] == bsnr) bw = default_width(iw);
                }
            } else if (kDefaultW && !kWriteSnr && i <= fit150) {
                // default widths near the end of block b: boxcars longer than the
                // samples left run into block b + 1 and take its line there
                const BlockParam q2 = bp[b + 1];
                const float c02 = q2.good ? q2.c0 : 0.0f;
                const float beta2 = q2.good ? q2.beta : 0.0f;
#pragma unroll
                for (int iw = 0; iw < kNumDefaultWidths; iw++) {
                    const int w = default_width(iw);
                    const int32_t Y = (int32_t)(sP[i + w] - p0);
                    float cr;
                    if (w <= rem) {
                        cr = (float)w * g + beta1 * (0.5f * (float)w * (float)(w - 1));
                    } else {
                        const int n1 = rem, n2 = w - rem;
                        cr = (float)n1 * g + beta1 * (0.5f * (float)n1 * (float)(n1 - 1)) +
                             (float)n2 * c02 + beta2 * (0.5f * (float)n2 * (float)(n2 - 1));
                    }
                    const float v = ((float)Y - cr) * sc[iw];
                    if (v > bsnr) {
                        bsnr = v;
                        bw = w;
                    }
                }
            } else if (kDefaultW && i <= fit150 && 150 <= rem) {
                // default widths, every boxcar inside block b
#pragma unroll
                for (int iw = 0; iw < kNumDefaultWidths; iw++) {
                    const int w = default_width(iw);
                    const int32_t Y = (int32_t)(sP[i + w] - p0);
                    const float cr = (float)w * g + beta1 * (0.5f * (float)w * (float)(w - 1));
                    const float v = ((float)Y - cr) * sc[iw];
                    if (kWriteSnr) snr_out[((int64_t)row * kNumDefaultWidths + iw) * Ls + t] = v;
                    if (v > bsnr) {
                        bsnr = v;
                        bw = w;
                    }
                }
            } else if (!kDefaultW && i <= fitw && wt.wmax <= rem) {
                // every boxcar inside block b: no bounds or straddle checks
#pragma unroll
                for (int iw = 0; iw < kMaxWidths; iw++) {
                    if (iw < wt.n) {
                        const int w = wt.w[iw];
                        const int32_t Y = (int32_t)(sP[i + w] - p0);
                        const float cr = (float)w * g + beta1 * wt.tri[iw];
                        const float v = ((float)Y - cr) * s_scale[iw];
                        if (kWriteSnr) snr_out[((int64_t)row * wt.n + iw) * Ls + t] = v;
                        if (v > bsnr) {
                            bsnr = v;
                            bw = w;
                        }
                    }
                }
            } else {
                BlockParam q2 = q;
                if (b + 1 < nb) q2 = bp[b + 1];
                const float c02 = q2.good ? q2.c0 : 0.0f;
                const float beta2 = q2.good ? q2.beta : 0.0f;
                for (int iw = 0; iw < wt.n; iw++) {
                    const int w = wt.w[iw];
                    float v;
                    if (t + w > Ls) {
                        v = __int_as_float(0x7fc00000);  // NaN: boxcar runs past the last block
                    } else {
                        const int32_t Y = (int32_t)(sP[i + w] - p0);
                        float cr;
                        if (w <= rem) {
                            cr = (float)w * g + beta1 * wt.tri[iw];
                        } else {
                            const int n1 = rem, n2 = w - rem;
                            cr = (float)n1 * g + beta1 * (0.5f * (float)n1 * (float)(n1 - 1)) +
                                 (float)n2 * c02 + beta2 * (0.5f * (float)n2 * (float)(n2 - 1));
                        }
                        v = ((float)Y - cr) * s_scale[iw];
                        if (v > bsnr) {
                            bsnr = v;
                            bw = w;
                        }
                    }
                    if (kWriteSnr) snr_out[((int64_t)row * wt.n + iw) * Ls + t] = v;
                }
            }
            if (live && bw > 0 && bsnr >= threshold) {
                const Best c{bsnr, t, bw};
                if (better(c, mine)) mine = c;
            }
        }
        // block argmax (S/N desc, t asc), skipped when no sample of the sub-chunk
        // reached the threshold (most of them)
        if (!__syncthreads_or(mine.w > 0)) continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            Best other;
            other.snr = __shfl_xor_sync(0xffffffffu, mine.snr, o);
            other.t = __shfl_xor_sync(0xffffffffu, mine.t, o);
            other.w = __shfl_xor_sync(0xffffffffu, mine.w, o);
            if (better(other, mine)) mine = other;
        }
        if (lane == 0) wbest[wid] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            Best bb = wbest[0];
            for (int q = 1; q < kBoxThreads / 32; q++)
                if (better(wbest[q], bb)) bb = wbest[q];
            if (bb.w > 0 && (!have || bb.snr > run.snr)) {
                run = bb;
                have = true;
            }
        }
        __syncthreads();
    }
    if (slots != nullptr) {
        // one slot per (row, window), in (row, window) order; width 0 = empty
        if (threadIdx.x == 0) {
            gsp_cand c;
            c.dm_idx = row;
            c.width = have ? run.w : 0;
            c.t = run.t;
            c.snr = run.snr;
            c.beam = 0;
            slots[(int64_t)row * nwin + wi] = c;
        }
    } else if (threadIdx.x == 0 && have) {
        const unsigned long long idx = atomicAdd(ncand, 1ull);
        if ((int64_t)idx < max_cands) {
            gsp_cand c;
            c.dm_idx = row;
            c.width = run.w;
            c.t = run.t;
            c.snr = run.snr;
            c.beam = 0;
            cands[idx] = c;
        }
    }
    }  // windows
}

// Stream compaction of the (row, window) slots into a dense candidate list in
// (row, t) order: per chunk of kCompact slots count the non-empty ones, scan
// the chunk counts, then scatter.  Records beyond max_cands are dropped; the
// total is written to *ncand.
constexpr int kCompact = 1024;

__global__ void __launch_bounds__(kCompact) slot_count_kernel(const gsp_cand *__restrict__ slots,
                                                              int64_t nslots,
                                                              unsigned int *__restrict__ counts) {
    const int64_t i = (int64_t)blockIdx.x * kCompact + threadIdx.x;
    const int f = (i < nslots && slots[i].width > 0) ? 1 : 0;
    const int c = __syncthreads_count(f);
    if (threadIdx.x == 0) counts[blockIdx.x] = (unsigned int)c;
}

__global__ void __launch_bounds__(kCompact) slot_scan_kernel(unsigned int *__restrict__ counts,
                                                             int64_t nchunks,
                                                             unsigned long long *__restrict__ ncand) {
    // exclusive scan of counts in place (one CTA, tiles of kCompact)
    __shared__ unsigned long long warp_tot[kCompact / 32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nchunks; base += kCompact) {
        const int64_t i = base + threadIdx.x;
        const unsigned long long v = i < nchunks ? counts[i] : 0ull;
        unsigned long long incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        unsigned long long pre = carry;
        for (int q = 0; q < wid; q++) pre += warp_tot[q];
        const unsigned long long excl = pre + incl - v;
        __syncthreads();
        if (i < nchunks) counts[i] = (unsigned int)excl;  // fits: total <= nslots < 2^32
        if (threadIdx.x == kCompact - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *ncand = carry;
}

__global__ void __launch_bounds__(kCompact) slot_scatter_kernel(
    const gsp_cand *__restrict__ slots, int64_t nslots, const unsigned int *__restrict__ offsets,
    gsp_cand *__restrict__ cands, int64_t max_cands) {
    __shared__ unsigned int warp_tot[kCompact / 32];
    const int64_t i = (int64_t)blockIdx.x * kCompact + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    gsp_cand c;
    c.width = 0;
    if (i < nslots) c = slots[i];
    const unsigned int f = c.width > 0 ? 1u : 0u;
    const unsigned int bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_tot[wid] = __popc(bal);
    __syncthreads();
    unsigned int pre = offsets[blockIdx.x];
    for (int q = 0; q < wid; q++) pre += warp_tot[q];
    pre += __popc(bal & ((1u << lane) - 1u));
    if (f && (int64_t)pre < max_cands) cands[pre] = c;
}

}  // namespace

cudaError_t launch_search(gsp_plan_s *p, const int32_t *D, int64_t n_out, int64_t stride,
                          int64_t t_offset, float *snr_out, const unsigned long long *bsum,
                          cudaStream_t s, int32_t *nlaunch) {
    const int B = p->desc.block_len;
    const int64_t nb = n_out / B;
    const int64_t Ls = nb * B;
    const int ndm = p->desc.ndm;
    cudaError_t e = cudaMemsetAsync(p->d_ncand, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (nb == 0) return cudaSuccess;
    WidthTable wt{};
    wt.n = (int)p->widths.size();
    wt.wmax = 0;
    for (int i = 0; i < wt.n; i++) {
        wt.w[i] = p->widths[i];
        wt.tri[i] = 0.5f * (float)p->widths[i] * (float)(p->widths[i] - 1);
        wt.wmax = max(wt.wmax, p->widths[i]);
    }
    if (bsum) {
        const int64_t n = nb * ndm;
        block_params_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            bsum, nb, B, p->nb_max, ndm, p->d_sigma_b, p->d_bparam);
    } else {
        block_stats_kernel<<<dim3((unsigned)nb, (unsigned)ndm), kStatThreads, 0, s>>>(
            D, stride, B, p->nb_max, p->d_sigma_b, p->d_bparam);
    }
    *nlaunch += 1;
    int n2 = 1;
    while (n2 < nb) n2 <<= 1;
    const size_t sm_sort = nb <= kSortMax ? (size_t)n2 * sizeof(double) : 0;
    row_sigma_kernel<<<ndm, 512, sm_sort, s>>>(p->d_sigma_b, nb, p->nb_max, (double)p->desc.bad_lo,
                                               (double)p->desc.bad_hi, wt, p->d_sref, p->d_scale,
                                               p->d_bad, p->d_bparam);
    *nlaunch += 1;
    const int64_t L = p->desc.window_len;
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int64_t k0 = fdiv(t_offset, L);
    const int64_t k1 = fdiv(t_offset + Ls - 1, L);
    const size_t sm_box = (size_t)(kChunk + wt.wmax + 1) * sizeof(uint32_t);
    // windows per CTA: up to 8 while there are still 16 CTAs per SM
    const int64_t nwin = k1 - k0 + 1;
    const int wpc = (int)std::max<int64_t>(
        1, std::min<int64_t>(8, nwin * ndm / (16 * (int64_t)std::max(p->num_sms, 1))));
    dim3 grid((unsigned)((nwin + wpc - 1) / wpc), (unsigned)ndm);
    bool dflt = wt.n == kNumDefaultWidths;
    for (int i = 0; dflt && i < wt.n; i++) dflt = wt.w[i] == default_width(i);
    if (snr_out && dflt)
        boxcar_kernel<true, true><<<grid, kBoxThreads, sm_box, s>>>(
            D, stride, Ls, B, p->nb_max, t_offset, L, k0, nwin, wpc, wt, p->d_bparam, p->d_scale,
            p->desc.threshold, snr_out, p->d_cands, p->d_ncand, p->desc.max_cands, p->d_slots);
    else if (snr_out)
        boxcar_kernel<true><<<grid, kBoxThreads, sm_box, s>>>(
            D, stride, Ls, B, p->nb_max, t_offset, L, k0, nwin, wpc, wt, p->d_bparam, p->d_scale,
            p->desc.threshold, snr_out, p->d_cands, p->d_ncand, p->desc.max_cands, p->d_slots);
    else if (dflt)
        boxcar_kernel<false, true><<<grid, kBoxThreads, sm_box, s>>>(
            D, stride, Ls, B, p->nb_max, t_offset, L, k0, nwin, wpc, wt, p->d_bparam, p->d_scale,
            p->desc.threshold, snr_out, p->d_cands, p->d_ncand, p->desc.max_cands, p->d_slots);
    else
        boxcar_kernel<false><<<grid, kBoxThreads, sm_box, s>>>(
            D, stride, Ls, B, p->nb_max, t_offset, L, k0, nwin, wpc, wt, p->d_bparam, p->d_scale,
            p->desc.threshold, snr_out, p->d_cands, p->d_ncand, p->desc.max_cands, p->d_slots);
    *nlaunch += 1;
    // dense candidate list in (row, t) order
    const int64_t nslots = nwin * ndm;
    const int64_t nchunks = (nslots + kCompact - 1) / kCompact;
    slot_count_kernel<<<(unsigned)nchunks, kCompact, 0, s>>>(p->d_slots, nslots, p->d_chunk);
    slot_scan_kernel<<<1, kCompact, 0, s>>>(p->d_chunk, nchunks, p->d_ncand);
    slot_scatter_kernel<<<(unsigned)nchunks, kCompact, 0, s>>>(p->d_slots, nslots, p->d_chunk,
                                                              p->d_cands, p->desc.max_cands);
    *nlaunch += 3;
    return cudaGetLastError();
}

cudaError_t launch_search_explicit(const SearchScratch &sc, const SearchConfig &cfg,
                                   const int32_t *D, int64_t n_out, int64_t stride,
                                   int64_t t_offset, gsp_cand *cands,
                                   unsigned long long *ncand, int64_t max_cands, cudaStream_t s) {
    const int B = cfg.block_len;
    const int64_t nb = n_out / B;
    const int64_t Ls = nb * B;
    if (nb == 0) return cudaSuccess;
    WidthTable wt{};
    wt.n = cfg.nwidths;
    wt.wmax = 0;
    for (int i = 0; i < wt.n; i++) {
        wt.w[i] = cfg.widths[i];
        wt.tri[i] = 0.5f * (float)cfg.widths[i] * (float)(cfg.widths[i] - 1);
        wt.wmax = max(wt.wmax, cfg.widths[i]);
    }
    block_stats_kernel<<<dim3((unsigned)nb, (unsigned)cfg.ndm), kStatThreads, 0, s>>>(
        D, stride, B, sc.nb_stride, sc.sigma_b, sc.bparam);
    int n2 = 1;
    while (n2 < nb) n2 <<= 1;
    const size_t sm_sort = nb <= kSortMax ? (size_t)n2 * sizeof(double) : 0;
    row_sigma_kernel<<<cfg.ndm, 512, sm_sort, s>>>(sc.sigma_b, nb, sc.nb_stride, cfg.bad_lo,
                                                   cfg.bad_hi, wt, sc.sref, sc.scale, sc.bad,
                                                   sc.bparam);
    const int64_t L = cfg.window_len;
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    const int64_t k0 = fdiv(t_offset, L);
    const int64_t k1 = fdiv(t_offset + Ls - 1, L);
    const size_t sm_box = (size_t)(kChunk + wt.wmax + 1) * sizeof(uint32_t);
    boxcar_kernel<false><<<dim3((unsigned)(k1 - k0 + 1), (unsigned)cfg.ndm), kBoxThreads, sm_box, s>>>(
        D, stride, Ls, B, sc.nb_stride, t_offset, L, k0, k1 - k0 + 1, 1, wt, sc.bparam, sc.scale,
        cfg.threshold,
        nullptr, cands, ncand, max_cands);
    return cudaGetLastError();
}

}  // namespace gsp
