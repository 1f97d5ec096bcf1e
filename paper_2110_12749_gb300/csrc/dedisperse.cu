// Brute-force incoherent dedispersion kernels (Sec. 2.3, Alg. 2/3):
//   D[dm][t] = sum_c X[c][t + delay[dm][c]],  t < n_out = n_in - max delay.
//
// The tiled kernel (dd_tiled_kernel) is the performance path.  Each CTA owns
// a tile of KW*8 consecutive DM trials x T_EFF output samples and streams the
// channels through a ring of shared-memory stages (32 channels per stage).
// A producer warp fills a stage with one TMA bulk copy per channel: the
// bytes X[c][s_c .. s_c + L) where s_c = floor16(t0 + min delay of the DM
// block), which cover every delay of the block.  Eight consumer warps each
// own KW DM trials; lane l of a warp owns the 4-sample words w = l + 32k
// (k < M) of the tile.  For a (channel, DM) pair the word a lane needs starts
// q = t0 + delay - s_c bytes into the window; the kernel reads the aligned
// word at q & ~3 and files its bytes under the phase p = q & 3 (output
// sample of byte i is 4w + i - p).  Channels are visited sorted by phase, so
// each phase accumulates into its own registers and the byte shift is
// resolved once per 256 channels, not per add.
//
// Accumulation (exact, SWAR): per word two 32-bit views are summed over
// channels: the raw word, S = sum w, and the odd bytes, O = sum (b1 + 2^16 b3)
// placed in 16-bit lanes by one byte permute.  A 16-bit lane holds at most
// 256 * 255 < 2^16, so every 256 channels the views are flushed into int32
// accumulators: b1 = O & 0xffff, b3 = O >> 16, and with E = S - (O << 8)
// (mod 2^32, the exact sum of b0 + 2^16 b2), b0 = E & 0xffff, b2 = E >> 16.
// Per word this is one shared load, one permute (ALU), half an IADD3 (ALU)
// and one multiply-add (x * 1 + acc on the IMAD pipe).  Other variants keep a
// masked even-byte view instead of the raw one.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dd_tiled.cuh"
#include "gsp_internal.cuh"

namespace gsp {

// ---------------------------------------------------------------------------
// Simple kernel: the direct form of Alg. 3.  One thread per (dm, 4 outputs),
// channel loop in registers, byte loads through L1.  Kept as a second,
// independent device implementation (GSP_FLAG_SIMPLE_DD) and as the path
// for delay tables whose spread within a DM block does not fit the tiles.
__global__ void __launch_bounds__(256) dd_simple_kernel(const uint8_t *__restrict__ x,
                                                        int64_t x_stride,
                                                        const int32_t *__restrict__ delays,
                                                        int nchan, int64_t n_out,
                                                        int32_t *__restrict__ out,
                                                        int64_t out_stride) {
    const int dm = blockIdx.y;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (t >= n_out) return;
    const int32_t *dl = delays + (int64_t)dm * nchan;
    int32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const bool full = t + 4 <= n_out;
    for (int c = 0; c < nchan; c++) {
        const uint8_t *p = x + (int64_t)c * x_stride + t + __ldg(dl + c);
        a0 += __ldg(p);
        if (full) {
            a1 += __ldg(p + 1);
            a2 += __ldg(p + 2);
            a3 += __ldg(p + 3);
        } else {
            if (t + 1 < n_out) a1 += __ldg(p + 1);
            if (t + 2 < n_out) a2 += __ldg(p + 2);
        }
    }
    int32_t *o = out + (int64_t)dm * out_stride + t;
    if (full) {
        *reinterpret_cast<int4 *>(o) = make_int4(a0, a1, a2, a3);
    } else {
        o[0] = a0;
        if (t + 1 < n_out) o[1] = a1;
        if (t + 2 < n_out) o[2] = a2;
    }
}

cudaError_t launch_dedisperse_simple(const gsp_plan_s *p, const uint8_t *x, int64_t x_stride,
                                     int64_t n_out, int32_t *out, int64_t out_stride,
                                     cudaStream_t s, int32_t *nlaunch) {
    const int64_t quads = (n_out + 3) / 4;
    dim3 grid((unsigned)((quads + 255) / 256), (unsigned)p->desc.ndm);
    dd_simple_kernel<<<grid, 256, 0, s>>>(x, x_stride, p->d_delays, p->desc.nchan, n_out, out,
                                          out_stride);
    *nlaunch += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tiled kernel.
namespace {

constexpr int kMaxBatchBeams = 32;  // beams per launch

// One beam of a launch: its input, delay tables, output and tiling.
struct BeamTile {
    const uint8_t *x;
    int64_t x_stride;
    int64_t n_in;
    int64_t n_out;
    const int32_t *delays;  // [ndm][nchan]
    const int32_t *blkmin;  // [nblk][nchan]
    const int32_t *dpos;    // [ndm][nchan] (delay << 8) | list position (stages of the variant's width)
    const uint32_t *fcnt;   // [ndm][nst] channels per phase family, 4 x 8 bits
    const int32_t *stspread;  // [nst] largest in-block delay spread of each stage's channels
    int32_t *out;
    int64_t out_stride;
    unsigned long long *bsum;  // optional [ndm][nb_max][3] block sums {S0, S1, S2}
    int64_t nb_max;
    int64_t Ls;      // searched length: block_len * floor(n_out / block_len)
    int64_t ntiles;  // time tiles
    int64_t item0;   // first work item of this beam
    int ndm;
    int nblk;
    int grp;         // DM blocks per launch group (groups sweep all time tiles in turn)
    int B;           // block_len (>= stored tile length, so a tile touches at most two blocks)
};

// A launch: one or more beams (same channel count) and their work items, one
// item per (beam, time tile, DM block).  With one CTA per item (grid = items)
// or persistent CTAs striding over the items (grid < items); the staging ring
// then runs on across items, so a CTA's next tile is prefetched while its
// current one is summed.
struct TiledArgs {
    BeamTile beam[kMaxBatchBeams];
    int nbeams;
    int nchan;
    int win;       // bytes per channel window (multiple of 16)
    int stages;    // ring depth
    uint32_t one;  // 1, passed at run time so that x * one + acc stays on the multiply-add pipe
    int *err;      // set to 1 if a bounded wait gave up
    int64_t items;
    long long budget;  // SM clock cycles a pipeline wait may take before it gives up
    int starve;        // failure-path test: the producer issues nothing, so every stage wait
                       // runs out (no copy is ever in flight)
};

// Work item -> beam, time tile and DM block.  Inside a beam: groups of `grp`
// DM blocks; inside a group, time tiles with the group's DM blocks fastest, so
// that items that run together read input spans whose union (over the group's
// delays) stays resident in L2.
__device__ __forceinline__ void decode_item(const TiledArgs &a, int64_t item, int *bi,
                                            int64_t *tile, int *blk) {
    int b = 0;
    while (b + 1 < a.nbeams && item >= a.beam[b + 1].item0) b++;
    const BeamTile &bt = a.beam[b];
    const int64_t idx = item - bt.item0;
    const int64_t nfull = bt.nblk / bt.grp;
    const int64_t per_group = bt.ntiles * bt.grp;
    if (idx < nfull * per_group) {
        const int64_t g = idx / per_group, r = idx - g * per_group;
        *tile = r / bt.grp;
        *blk = (int)(g * bt.grp + (r - *tile * bt.grp));
    } else {
        const int64_t rem = bt.nblk - nfull * bt.grp;
        const int64_t r = idx - nfull * per_group;
        *tile = r / rem;
        *blk = (int)(nfull * bt.grp + (r - *tile * rem));
    }
    *bi = b;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void fail(int *err) { atomicExch(err, 1); }

// Accumulate two words of one phase into the odd-byte view O (bytes 1 and 3
// in 16-bit lanes, one byte permute per word) and into E.  For ACC 0-2, E is
// the even-byte view (bytes 0 and 2, one LOP3 per word) and ACC chooses the
// pipe of the additions: 0 = IADD3 on the integer ALU, 1 = E on the ALU and
// O as x * 1 + acc on the multiply-add pipe, 2 = both on the multiply-add
// pipe.  For ACC 3, E is the raw sum of the words (IADD3, no extraction) and
// O is summed on the multiply-add pipe (ACC 4: O with IADD3 on the ALU too); since w = (b0 + 2^16 b2) + 2^8 O(w),
// the even-byte sums are E - (O << 8) mod 2^32, exact while the 16-bit lanes
// cannot overflow.
// Flush one phase family P into the int32 accumulators: recover the four
// byte sums of each word, add the ones that belong to this lane's word, and
// pass the ones that belong to the previous word (phase P > 0 only) one lane
// down: the previous word of (lane, k) is (lane - 1, k), or (31, k - 1) for
// lane 0.
template <int P, int M, int ACC>
__device__ __forceinline__ void flush_family(uint32_t (&E)[M], uint32_t (&O)[M],
                                             uint32_t (&acc)[M][4], int lane) {
    uint32_t sp[M][3];
#pragma unroll
    for (int k = 0; k < M; k++) {
        sp[k][0] = sp[k][1] = sp[k][2] = 0;
        const uint32_t o = O[k];
        const uint32_t e = ACC >= 3 ? E[k] - (o << 8) : E[k];
        const uint32_t b[4] = {e & 0xffffu, o & 0xffffu, e >> 16, o >> 16};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int jj = q - P;
            if (jj >= 0) acc[k][jj] += b[q];
            else sp[k][jj + 3] += b[q];
        }
        E[k] = O[k] = 0;
    }
    if (P > 0) {
#pragma unroll
        for (int k = 0; k < M; k++) {
#pragma unroll
            for (int jj = 3 - P; jj < 3; jj++) {
                const uint32_t r = __shfl_sync(0xffffffffu, sp[k][jj], (lane + 1) & 31);
                const uint32_t rn =
                    (k + 1 < M) ? __shfl_sync(0xffffffffu, sp[(k + 1) % M][jj], (lane + 1) & 31) : 0u;
                if (lane < 31) acc[k][jj + 1] += r;
                else if (k + 1 < M) acc[k][jj + 1] += rn;
            }
        }
    }
}

// The same with the family chosen at run time (a constant after unrolling).
template <int M, int ACC>
__device__ __forceinline__ void flush_family_p(int P, uint32_t (&E)[M], uint32_t (&O)[M],
                                               uint32_t (&acc)[M][4], int lane) {
    switch (P) {
        case 0: flush_family<0, M, ACC>(E, O, acc, lane); break;
        case 1: flush_family<1, M, ACC>(E, O, acc, lane); break;
        case 2: flush_family<2, M, ACC>(E, O, acc, lane); break;
        default: flush_family<3, M, ACC>(E, O, acc, lane); break;
    }
}

template <int ACC>
__device__ __forceinline__ void acc_pair(uint32_t &E, uint32_t &O, uint32_t w1, uint32_t w2,
                                         uint32_t one) {
    const uint32_t e1 = w1 & 0x00ff00ffu, e2 = w2 & 0x00ff00ffu;
    const uint32_t o1 = __byte_perm(w1, 0, 0x4341), o2 = __byte_perm(w2, 0, 0x4341);
    if (ACC == 3) {
        // raw view: E holds sum w; the even bytes are recovered at the flush
        E += w1 + w2;
        O = ptx::imadd(o1, one, ptx::imadd(o2, one, O));
    } else if (ACC == 4) {
        // raw view, both sums as three-input adds on the integer ALU
        E += w1 + w2;
        O += o1 + o2;
    } else if (ACC == 0) {
        E += e1 + e2;
        O += o1 + o2;
    } else if (ACC == 1) {
        E += e1 + e2;
        O = ptx::imadd(o1, one, ptx::imadd(o2, one, O));
    } else {
        E = ptx::imadd(e1, one, ptx::imadd(e2, one, E));
        O = ptx::imadd(o1, one, ptx::imadd(o2, one, O));
    }
}

// Merged flush (raw + odd views): combine the four phase families in 16-bit
// lanes before unpacking.  Every channel belongs to exactly one family, so
// the contributions of all families to one output slot still come from at
// most 256 channels and fit a 16-bit lane.  With e_P = E_P - (O_P << 8)
// (bytes 0 and 2 of family P) and o_P = O_P (bytes 1 and 3), byte q of family
// P lands in slot q - P, so for this word
//   A = [slot 0 | slot 2] = e0 + o1 + (e2 >> 16) + (o3 >> 16)
//   B = [slot 1 | slot 3] = o0 + (e1 >> 16) + (o2 >> 16)
// and the bytes that land in the previous word (negative slots) are
//   SA = [0 | slot 2] = (e2 + o3) << 16,  SB = [slot 1 | slot 3] = e3 + ((e1 + o2) << 16).
// The int32 accumulators then take lo + 2^16 hi (acc[k][0], acc[k][1]) and
// hi (acc[k][2], acc[k][3]); merged_decode() recovers lo at the end.
template <int M>
__device__ __forceinline__ void flush_merged(uint32_t (&E)[4][M], uint32_t (&O)[4][M],
                                             uint32_t (&acc)[M][4], int lane) {
    uint32_t A[M], B[M], SA[M], SB[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        const uint32_t o0 = O[0][k], o1 = O[1][k], o2 = O[2][k], o3 = O[3][k];
        const uint32_t e0 = E[0][k] - (o0 << 8), e1 = E[1][k] - (o1 << 8);
        const uint32_t e2 = E[2][k] - (o2 << 8), e3 = E[3][k] - (o3 << 8);
        A[k] = e0 + o1 + (e2 >> 16) + (o3 >> 16);
        B[k] = o0 + (e1 >> 16) + (o2 >> 16);
        SA[k] = (e2 + o3) << 16;
        SB[k] = e3 + ((e1 + o2) << 16);
#pragma unroll
        for (int P = 0; P < 4; P++) E[P][k] = O[P][k] = 0;
    }
    // previous word of (lane, k) is (lane - 1, k), or (31, k - 1) for lane 0
    uint32_t rA[M], rB[M];
#pragma unroll
    for (int k = 0; k < M; k++) {
        rA[k] = __shfl_sync(0xffffffffu, SA[k], (lane + 1) & 31);
        rB[k] = __shfl_sync(0xffffffffu, SB[k], (lane + 1) & 31);
    }
#pragma unroll
    for (int k = 0; k < M; k++) {
        const uint32_t xa = lane < 31 ? rA[k] : (k + 1 < M ? rA[(k + 1) % M] : 0u);
        const uint32_t xb = lane < 31 ? rB[k] : (k + 1 < M ? rB[(k + 1) % M] : 0u);
        const uint32_t a = A[k] + xa, b = B[k] + xb;
        acc[k][0] += a;
        acc[k][2] += a >> 16;
        acc[k][1] += b;
        acc[k][3] += b >> 16;
    }
}

// acc[k][0] = sum lo + 2^16 sum hi (mod 2^32) and acc[k][2] = sum hi: slot 0
// is acc[k][0] - (acc[k][2] << 16), exact since the true sum is below 2^32.
template <int M>
__device__ __forceinline__ void merged_decode(uint32_t (&acc)[M][4]) {
#pragma unroll
    for (int k = 0; k < M; k++) {
        acc[k][0] -= acc[k][2] << 16;
        acc[k][1] -= acc[k][3] << 16;
    }
}

// KW: DM trials per consumer warp; kCW = KDM / KW consumer warps + 1 producer.
// QUAD: visit channels four at a time (more loads in flight per warp).
// M: 4-sample words per lane, T = 128 M output samples computed per tile and
// T - 4 stored (the tile's last word is incomplete by construction).
// CB: channels per shared-memory stage (a multiple of 32).
// FF: flush each phase family only when its own channel count would pass 256
// (instead of all families every 256 channels).
// PRE: the phase-sorted channel lists come from the plan's precomputed list
// positions (the phase of a (channel, DM) pair is delay & 3 in every tile,
// since tiles start at multiples of 4 samples), not from a per-stage ballot sort.
// MF: merged flush of the four phase families (flush_merged).
// KDM: DM trials per CTA.  UNR: unroll depth of the two-channel loop (A32).
// IMA: per-channel address adds as x * 1 + y on the multiply-add pipe (A32).
template <int KW, bool QUAD, int ACC, bool A32 = false, int M = 4, int CB = 32, bool FF = false,
          bool PRE = false, bool MF = false, int KDM = 16, int UNR = 2, bool IMA = false>
__global__ void __launch_bounds__((KDM / KW + 1) * 32, (KDM / KW + 1) * 32 <= 256 ? 2 : 1)
    dd_tiled_kernel(const TiledArgs a) {
    static_assert(!PRE || (KW == 1 && (CB == 64 || CB == 32)),
                  "precomputed lists: one DM per warp, 32- or 64-channel stages");
    static_assert(!MF || (ACC >= 3 && !FF), "merged flush: raw + odd views, all families together");
    constexpr int kCB = CB;
    constexpr int kH = CB / 32;                  // channels per lane per stage
    constexpr int kFlushStages = 256 / kCB;      // stages between SWAR flushes (256 channels)
    constexpr int kM = M;
    constexpr int kT = 128 * kM;
    constexpr int kTEff = kT - 4;
    constexpr int kKW = KW;
    static_assert(KDM % KW == 0, "DM trials per CTA: a multiple of the DM trials per warp");
    constexpr int kCW = KDM / KW;
    extern __shared__ __align__(128) uint8_t smem[];
    const int slot_bytes = kCB * a.win;
    int32_t *lists = reinterpret_cast<int32_t *>(smem + (size_t)a.stages * slot_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(lists + kCW * kKW * 4 * kCB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nst = (a.nchan + kCB - 1) / kCB;
    auto full = [&](int i) { return ptx::smem_addr(bars + i); };
    auto empty = [&](int i) { return ptx::smem_addr(bars + a.stages + i); };

    if (threadIdx.x == 0) {
        for (int i = 0; i < a.stages; i++) {
            ptx::mbar_init(full(i), 32);
            ptx::mbar_init(empty(i), kCW);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();

    if (warp == kCW) {
        // ------------------------------------------------------- producer warp
        if (a.starve) return;  // failure-path test: nothing issued, nothing in flight
        int64_t gst = 0;  // stages issued by this CTA so far (across items)
        int slot = 0;           // ring slot of the next stage
        uint32_t rpar = 0;      // parity of the slot's current round
        bool wrapped = false;   // the ring has been filled once
        bool ok = true;
        for (int64_t item = blockIdx.x; item < a.items && ok; item += gridDim.x) {
        int bi, blk;
        int64_t tile;
        decode_item(a, item, &bi, &tile, &blk);
        const BeamTile &bt = a.beam[bi];
        const int64_t t0 = tile * kTEff;
        const int32_t *bmin = bt.blkmin + (int64_t)blk * a.nchan;
        for (int st = 0; st < nst && ok; st++, gst++) {
            if (wrapped) {
                const bool w = ptx::mbar_wait(empty(slot), rpar ^ 1u, a.budget);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
            }
            // this stage's window: the tile plus the largest in-block delay spread of
            // its own channels (at most a.win, the slot pitch set by the widest stage)
            const int64_t wst = min((int64_t)a.win, (int64_t)((kT + 30 + bt.stspread[st]) & ~15));
            int64_t s_c[kH], avail[kH];
            uint32_t len16[kH];
            uint32_t tot = 0;
#pragma unroll
            for (int h = 0; h < kH; h++) {
                const int c = st * kCB + h * 32 + lane;
                s_c[h] = 0;
                avail[h] = 0;
                len16[h] = 0;
                if (c < a.nchan) {
                    s_c[h] = (t0 + bmin[c]) & ~(int64_t)15;
                    avail[h] = bt.n_in - s_c[h];
                    len16[h] = (uint32_t)min(wst, avail[h] & ~(int64_t)15);
                }
                tot += len16[h];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lane == 0)
                asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(full(slot)),
                             "r"(tot)
                             : "memory");
            __syncwarp();
#pragma unroll
            for (int h = 0; h < kH; h++) {
                const int c = st * kCB + h * 32 + lane;
                uint8_t *dst = smem + (size_t)slot * slot_bytes + (size_t)(h * 32 + lane) * a.win;
                if (len16[h] > 0) {
                    const uint8_t *src = bt.x + (int64_t)c * bt.x_stride + s_c[h];
                    ptx::bulk_g2s(ptx::smem_addr(dst), src, len16[h], full(slot));
                }
                if (c < a.nchan) {
                    const int64_t end = min(wst, avail[h]);
                    for (int64_t i = len16[h]; i < end; i++)
                        dst[i] = bt.x[(int64_t)c * bt.x_stride + s_c[h] + i];
                }
            }
            ptx::mbar_arrive(full(slot));
            if (++slot == a.stages) {
                slot = 0;
                rpar ^= 1u;
                wrapped = true;
            }
        }
        }
        if (!ok && lane == 0) fail(a.err);
        // never leave with copies in flight: wait for the last phase of each slot (with
        // the full limit, whatever a.budget is; the CTA's shared memory stays allocated
        // until this warp returns, even if the consumer warps have given up and left)
        for (int64_t st = max((int64_t)0, gst - a.stages); st < gst; st++) {
            const bool w = ptx::mbar_wait(full((int)(st % a.stages)), (uint32_t)((st / a.stages) & 1),
                                          kWaitLimit);
            if (!__all_sync(0xffffffffu, w)) {
                if (lane == 0) fail(a.err);
                break;
            }
        }
        return;
    }

    // ------------------------------------------------------- consumer warps
    int32_t *mylist = lists + warp * (kKW * 4 * kCB);
    const uint32_t one = a.one;
    const uint32_t lmask = lanemask_lt();
    const uint32_t smem32 = ptx::smem_addr(smem);
    const uint32_t lane4 = 4u * lane;
    int slot = 0;       // ring slot of the next stage (no 64-bit division per stage)
    uint32_t rpar = 0;  // parity of the slot's current round
    for (int64_t item = blockIdx.x; item < a.items; item += gridDim.x) {
    int bi, blk;
    int64_t tile;
    decode_item(a, item, &bi, &tile, &blk);
    const BeamTile &bt = a.beam[bi];
    const int64_t t0 = tile * kTEff;
    const int dm0 = blk * KDM;
    const int32_t *bmin = bt.blkmin + (int64_t)blk * a.nchan;
    const int dmw = dm0 + warp * kKW;
    uint32_t acc[kKW][kM][4];
    uint32_t E[kKW][4][kM], O[kKW][4][kM];
#pragma unroll
    for (int i = 0; i < kKW; i++)
#pragma unroll
        for (int k = 0; k < kM; k++) {
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][k][j] = 0;
#pragma unroll
            for (int p = 0; p < 4; p++) E[i][p][k] = O[i][p][k] = 0;
        }
    int famcnt[kKW][4];  // channels accumulated per family since its last flush (FF)
#pragma unroll
    for (int i = 0; i < kKW; i++)
#pragma unroll
        for (int P = 0; P < 4; P++) famcnt[i][P] = 0;
    // delays of the next stage are loaded one stage ahead (hides L2 latency)
    // PRE: nx_dl holds the packed (delay << 8) | list position instead of the delay
    const int32_t *dtab = PRE ? bt.dpos : bt.delays;
    const uint32_t *fcrow = PRE ? bt.fcnt + (int64_t)min(dmw, bt.ndm - 1) * nst : nullptr;
    int nx_min[kH], nx_dl[kKW][kH];
    uint32_t nx_fc = PRE ? fcrow[0] : 0u;
#pragma unroll
    for (int h = 0; h < kH; h++) {
        const int c0 = h * 32 + lane;
        const bool v0 = c0 < a.nchan;
        nx_min[h] = v0 ? bmin[c0] : 0;
#pragma unroll
        for (int i = 0; i < kKW; i++)
            nx_dl[i][h] = v0 ? dtab[(int64_t)min(dmw + i, bt.ndm - 1) * a.nchan + c0] : 0;
    }

    for (int st = 0; st < nst; st++) {
        int cur_min[kH], cur_dl[kKW][kH];
        // the same word in every lane; a warp reduction makes that visible to the compiler,
        // so the family loops below branch on a warp-uniform count
        const uint32_t cur_fc = PRE ? __reduce_or_sync(0xffffffffu, nx_fc) : 0u;
        if (PRE && st + 1 < nst) nx_fc = fcrow[st + 1];
#pragma unroll
        for (int h = 0; h < kH; h++) {
            cur_min[h] = nx_min[h];
#pragma unroll
            for (int i = 0; i < kKW; i++) cur_dl[i][h] = nx_dl[i][h];
            const int cn = (st + 1) * kCB + h * 32 + lane;
            const bool vn = cn < a.nchan;
            nx_min[h] = vn ? bmin[cn] : 0;
#pragma unroll
            for (int i = 0; i < kKW; i++)
                nx_dl[i][h] = vn ? dtab[(int64_t)min(dmw + i, bt.ndm - 1) * a.nchan + cn] : 0;
        }
        int cnt[kKW][4];
#pragma unroll
        for (int i = 0; i < kKW; i++)
#pragma unroll
            for (int P = 0; P < 4; P++) cnt[i][P] = PRE ? (int)((cur_fc >> (8 * P)) & 0xffu) : 0;
        if constexpr (PRE) {
            // each lane files its channel's aligned word at the precomputed position
            // (family P occupies entries [P * kCB, P * kCB + count_P) of the list)
            const uint32_t t0lo = (uint32_t)t0;
#pragma unroll
            for (int h = 0; h < kH; h++) {
                const int c = st * kCB + h * 32 + lane;
                const uint32_t pk = (uint32_t)cur_dl[0][h];
                const uint32_t q = (t0lo + (pk >> 8)) - ((t0lo + (uint32_t)cur_min[h]) & ~15u);
                const int boff = slot * slot_bytes + (h * 32 + lane) * a.win + (int)(q & ~3u);
                if (c < a.nchan) mylist[pk & 0xffu] = A32 ? (int)(smem32 + boff) : (boff >> 2);
            }
        } else
#pragma unroll
        for (int h = 0; h < kH; h++) {
            const int c = st * kCB + h * 32 + lane;
            const bool valid = c < a.nchan;
            const int64_t s_c = valid ? ((t0 + cur_min[h]) & ~(int64_t)15) : 0;
#pragma unroll
            for (int i = 0; i < kKW; i++) {
                const int dl = valid ? cur_dl[i][h] : 0;
                const int q = (int)(t0 + dl - s_c);
                const int p = q & 3;
                // the aligned word of this (channel, DM) in shared memory: its word
                // index, or (A32) its 32-bit shared-window byte address
                const int boff = slot * slot_bytes + (h * 32 + lane) * a.win + (q & ~3);
                const int entry = A32 ? (int)(smem32 + boff) : (boff >> 2);
#pragma unroll
                for (int P = 0; P < 4; P++) {
                    const uint32_t m = __ballot_sync(0xffffffffu, valid && p == P);
                    if (valid && p == P)
                        mylist[(i * 4 + P) * kCB + cnt[i][P] + __popc(m & lmask)] = entry;
                    cnt[i][P] += __popc(m);
                }
            }
        }
        __syncwarp();
        const bool landed = ptx::mbar_wait(full(slot), rpar, a.budget);
        if (!__all_sync(0xffffffffu, landed)) {
            if (lane == 0) fail(a.err);
            return;
        }
        const uint32_t *lanebase = reinterpret_cast<const uint32_t *>(smem) + lane;
        if constexpr (A32) {
            // explicit 32-bit shared addresses, immediate offsets per word
#pragma unroll
            for (int i = 0; i < kKW; i++) {
#pragma unroll
                for (int P = 0; P < 4; P++) {
                    const int n = cnt[i][P];
                    if constexpr (FF) {
                        if (famcnt[i][P] + n > 256) {
                            flush_family_p<kM, ACC>(P, E[i][P], O[i][P], acc[i], lane);
                            famcnt[i][P] = 0;
                        }
                        famcnt[i][P] += n;
                    }
                    const int32_t *lp = mylist + (i * 4 + P) * kCB;
                    int j = 0;
                    if constexpr (QUAD) {
                        // four channels per step (one 16-byte entry load)
                        for (; j + 4 <= n; j += 4) {
                            const int4 e = *reinterpret_cast<const int4 *>(lp + j);
                            uint32_t w1[kM], w2[kM], w3[kM], w4[kM];
                            ptx::lds_words<kM>((uint32_t)e.x + lane4, w1);
                            ptx::lds_words<kM>((uint32_t)e.y + lane4, w2);
                            ptx::lds_words<kM>((uint32_t)e.z + lane4, w3);
                            ptx::lds_words<kM>((uint32_t)e.w + lane4, w4);
#pragma unroll
                            for (int k = 0; k < kM; k++) {
                                acc_pair<ACC>(E[i][P][k], O[i][P][k], w1[k], w2[k], one);
                                acc_pair<ACC>(E[i][P][k], O[i][P][k], w3[k], w4[k], one);
                            }
                        }
                    }
#pragma unroll UNR
                    for (; j + 2 <= n; j += 2) {
                        const int2 e = *reinterpret_cast<const int2 *>(lp + j);
                        const uint32_t a1 = IMA ? ptx::imadd((uint32_t)e.x, one, lane4)
                                                : (uint32_t)e.x + lane4;
                        const uint32_t a2 = IMA ? ptx::imadd((uint32_t)e.y, one, lane4)
                                                : (uint32_t)e.y + lane4;
                        uint32_t w1[kM], w2[kM];
                        ptx::lds_words<kM>(a1, w1);
                        ptx::lds_words<kM>(a2, w2);
#pragma unroll
                        for (int k = 0; k < kM; k++) acc_pair<ACC>(E[i][P][k], O[i][P][k], w1[k], w2[k], one);
                    }
                    if (j < n) {
                        uint32_t w1[kM];
                        ptx::lds_words<kM>((uint32_t)lp[j] + lane4, w1);
#pragma unroll
                        for (int k = 0; k < kM; k++) {
                            E[i][P][k] += ACC >= 3 ? w1[k] : (w1[k] & 0x00ff00ffu);
                            if (IMA)
                                O[i][P][k] = ptx::imadd(__byte_perm(w1[k], 0, 0x4341), one, O[i][P][k]);
                            else
                                O[i][P][k] += __byte_perm(w1[k], 0, 0x4341);
                        }
                    }
                }
            }
        } else

#pragma unroll
        for (int i = 0; i < kKW; i++) {
#pragma unroll
            for (int P = 0; P < 4; P++) {
                const int n = cnt[i][P];
                if constexpr (FF) {
                    if (famcnt[i][P] + n > 256) {
                        flush_family_p<kM, ACC>(P, E[i][P], O[i][P], acc[i], lane);
                        famcnt[i][P] = 0;
                    }
                    famcnt[i][P] += n;
                }
                const int32_t *lp = mylist + (i * 4 + P) * kCB;
                int j = 0;
                if (QUAD) {
                    for (; j + 4 <= n; j += 4) {
                        const int4 e = *reinterpret_cast<const int4 *>(lp + j);
                        const uint32_t *p1 = lanebase + e.x;
                        const uint32_t *p2 = lanebase + e.y;
                        const uint32_t *p3 = lanebase + e.z;
                        const uint32_t *p4 = lanebase + e.w;
#pragma unroll
                        for (int k = 0; k < kM; k++) {
                            const uint32_t w1 = p1[32 * k], w2 = p2[32 * k];
                            const uint32_t w3 = p3[32 * k], w4 = p4[32 * k];
                            acc_pair<ACC>(E[i][P][k], O[i][P][k], w1, w2, one);
                            acc_pair<ACC>(E[i][P][k], O[i][P][k], w3, w4, one);
                        }
                    }
                }
                for (; j + 2 <= n; j += 2) {
                    const int2 e = *reinterpret_cast<const int2 *>(lp + j);
                    const uint32_t *p1 = lanebase + e.x;
                    const uint32_t *p2 = lanebase + e.y;
#pragma unroll
                    for (int k = 0; k < kM; k++) {
                        const uint32_t w1 = p1[32 * k], w2 = p2[32 * k];
                        acc_pair<ACC>(E[i][P][k], O[i][P][k], w1, w2, one);
                    }
                }
                if (j < n) {
                    const uint32_t *p1 = lanebase + lp[j];
#pragma unroll
                    for (int k = 0; k < kM; k++) {
                        const uint32_t w1 = p1[32 * k];
                        E[i][P][k] += ACC >= 3 ? w1 : (w1 & 0x00ff00ffu);
                        O[i][P][k] += __byte_perm(w1, 0, 0x4341);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(empty(slot));
        if (++slot == a.stages) {
            slot = 0;
            rpar ^= 1u;
        }

        if (MF && ((st + 1) % kFlushStages == 0 || st == nst - 1)) {
#pragma unroll
            for (int i = 0; i < kKW; i++) flush_merged<kM>(E[i], O[i], acc[i], lane);
        } else if (FF && st == nst - 1) {
#pragma unroll
            for (int i = 0; i < kKW; i++) {
                flush_family<0, kM, ACC>(E[i][0], O[i][0], acc[i], lane);
                flush_family<1, kM, ACC>(E[i][1], O[i][1], acc[i], lane);
                flush_family<2, kM, ACC>(E[i][2], O[i][2], acc[i], lane);
                flush_family<3, kM, ACC>(E[i][3], O[i][3], acc[i], lane);
            }
        } else if (!MF && !FF && ((st + 1) % kFlushStages == 0 || st == nst - 1)) {
#pragma unroll
            for (int i = 0; i < kKW; i++) {
                uint32_t sp[kM][3];
#pragma unroll
                for (int k = 0; k < kM; k++) {
                    sp[k][0] = sp[k][1] = sp[k][2] = 0;
#pragma unroll
                    for (int P = 0; P < 4; P++) {
                        const uint32_t o = O[i][P][k];
                        const uint32_t e = ACC >= 3 ? E[i][P][k] - (o << 8) : E[i][P][k];
                        uint32_t b[4];
                        b[0] = e & 0xffffu;
                        b[1] = o & 0xffffu;
                        b[2] = e >> 16;
                        b[3] = o >> 16;
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            const int jj = q - P;  // output slot, negative = previous word
                            if (jj >= 0) acc[i][k][jj] += b[q];
                            else sp[k][jj + 3] += b[q];
                        }
                        E[i][P][k] = O[i][P][k] = 0;
                    }
                }
                // previous word of (lane, k) is (lane - 1, k), or (31, k - 1) for lane 0
#pragma unroll
                for (int k = 0; k < kM; k++) {
#pragma unroll
                    for (int jj = 0; jj < 3; jj++) {
                        const uint32_t r = __shfl_sync(0xffffffffu, sp[k][jj], (lane + 1) & 31);
                        const uint32_t rn =
                            (k + 1 < kM) ? __shfl_sync(0xffffffffu, sp[(k + 1) % kM][jj], (lane + 1) & 31) : 0u;
                        if (lane < 31) acc[i][k][jj + 1] += r;
                        else if (k + 1 < kM) acc[i][k][jj + 1] += rn;
                    }
                }
            }
        }
    }

    if constexpr (MF) {
#pragma unroll
        for (int i = 0; i < kKW; i++) merged_decode<kM>(acc[i]);
    }

    // ------------------------------------------------------- store the tile
#pragma unroll
    for (int i = 0; i < kKW; i++) {
        const int d = dmw + i;
        if (d >= bt.ndm) continue;
        if (bt.bsum != nullptr) {
            // exact sums of the stored samples for the (at most two) search blocks
            // the tile touches: S0 = sum D, S1 = sum j D (j inside the block), S2 = sum D^2
            const int64_t ba = t0 / bt.B;
            const int64_t tb = (ba + 1) * bt.B;
            long long sm[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
            for (int k = 0; k < kM; k++) {
                const int w = lane + 32 * k;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int64_t t = t0 + 4 * w + j;
                    if (4 * w + j < kTEff && t < bt.Ls) {
                        const long long v = (long long)(int32_t)acc[i][k][j];
                        if (t < tb) {
                            sm[0][0] += v;
                            sm[0][1] += (t - ba * bt.B) * v;
                            sm[0][2] += v * v;
                        } else {
                            sm[1][0] += v;
                            sm[1][1] += (t - tb) * v;
                            sm[1][2] += v * v;
                        }
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; h++)
#pragma unroll
                for (int f = 0; f < 3; f++) {
                    long long v = sm[h][f];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    sm[h][f] = v;
                }
            if (lane == 0) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int64_t b = ba + h;
                    if (b * bt.B < bt.Ls) {
                        unsigned long long *q = bt.bsum + ((int64_t)d * bt.nb_max + b) * 3;
#pragma unroll
                        for (int f = 0; f < 3; f++) atomicAdd(q + f, (unsigned long long)sm[h][f]);
                    }
                }
            }
        }
        int32_t *orow = bt.out + (int64_t)d * bt.out_stride;
#pragma unroll
        for (int k = 0; k < kM; k++) {
            const int w = lane + 32 * k;
            const int64_t tt = t0 + 4 * w;
            if (4 * w + 3 < kTEff && tt + 3 < bt.n_out) {
                // streaming store: the series is not re-read by this kernel
                __stcs(reinterpret_cast<int4 *>(orow + tt),
                       make_int4((int)acc[i][k][0], (int)acc[i][k][1], (int)acc[i][k][2],
                                 (int)acc[i][k][3]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (4 * w + j < kTEff && tt + j < bt.n_out) orow[tt + j] = (int32_t)acc[i][k][j];
            }
        }
    }
    }  // items
}

// Per-DM-block minimum delay per channel, the largest spread of delays within
// a block, and from it the shared-memory window per channel and ring depth.
typedef void (*TiledKernel)(const TiledArgs);

struct TiledVariant {
    TiledKernel fn;
    int kw;
    int m;
    int cb;
    bool pre = false;  // needs the plan's precomputed list positions
    int kdm = 16;      // DM trials per CTA (one of kKdmSizes)
};

// Tuning variants of the tiled kernel (same result, different schedule).
const TiledVariant kVariants[] = {
    {dd_tiled_kernel<2, false, 0>, 2, 4, 32},
    {dd_tiled_kernel<1, false, 0>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 1>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 2>, 1, 4, 32},
    {dd_tiled_kernel<2, false, 1>, 2, 4, 32},
    {dd_tiled_kernel<1, true, 1>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 2, true>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 2, true, 8>, 1, 8, 32},
    {dd_tiled_kernel<1, false, 3>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 3, true>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 3, false, 4, 64>, 1, 4, 64},
    {dd_tiled_kernel<1, true, 3, false, 4, 64>, 1, 4, 64},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, true>, 1, 4, 64},
    {dd_tiled_kernel<1, false, 3, false, 4, 32, true>, 1, 4, 32},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, false, true, false>, 1, 4, 64, true},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, false, true, true>, 1, 4, 64, true},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, false, false, true>, 1, 4, 64},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, true, true>, 1, 4, 64, true},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, false, true>, 1, 4, 64},
    {dd_tiled_kernel<1, true, 3, true, 4, 64, false, true, true>, 1, 4, 64, true},
    {dd_tiled_kernel<1, true, 3, true, 4, 64, false, false, true>, 1, 4, 64},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, false, true, 15>, 1, 4, 64, false, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, true, true, 15>, 1, 4, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, false, false, true, 15>, 1, 4, 64, false, 15},
    {dd_tiled_kernel<1, true, 3, true, 4, 64, false, false, true, 15>, 1, 4, 64, false, 15},
    {dd_tiled_kernel<1, false, 3, false, 4, 64, false, true, true, 15>, 1, 4, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 32, false, false, true, 15>, 1, 4, 32, false, 15},
    {dd_tiled_kernel<1, false, 3, true, 8, 64, false, true, true, 15>, 1, 8, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, false, 8, 64, false, true, true, 15>, 1, 8, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, true, true, 15, 4>, 1, 4, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, true, true, 15, 1>, 1, 4, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 64, false, true, true, 15, 2, true>, 1, 4, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 64, false, true, true, 15, 2, true>, 1, 6, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 64, false, true, true, 15, 1, true>, 1, 6, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 32, false, false, true, 15, 2, true>, 1, 6, 32, false, 15},
    {dd_tiled_kernel<1, false, 3, true, 7, 64, false, true, true, 15, 2, true>, 1, 7, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 64, false, true, true, 15, 3, true>, 1, 6, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 64, false, true, true, 15, 4, true>, 1, 6, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 5, 64, false, true, true, 15, 2, true>, 1, 5, 64, true, 15},
    {dd_tiled_kernel<1, false, 4, true, 6, 64, false, true, true, 15, 2, true>, 1, 6, 64, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 32, false, false, true, 7, 2, true>, 1, 6, 32, false, 7},
    {dd_tiled_kernel<1, false, 3, true, 4, 32, false, false, true, 7, 2, true>, 1, 4, 32, false, 7},
    // 32-channel stages with precomputed lists (plans whose delay spread leaves
    // the 64-channel stages fewer than two ring slots: wide bands, coarse DM steps)
    {dd_tiled_kernel<1, false, 3, true, 6, 32, false, true, true, 15, 2, true>, 1, 6, 32, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 4, 32, false, true, true, 15, 2, true>, 1, 4, 32, true, 15},
    {dd_tiled_kernel<1, false, 3, true, 6, 32, false, true, true, 7, 2, true>, 1, 6, 32, true, 7},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

constexpr int kDefaultVariant = 32;  // 15 DMs x 768 samples, 64-channel stages, precomputed lists

// Variants tried in order when a plan is created; the first whose stages fit
// at least two ring slots is taken: the default; the same tile with 32-channel
// stages (half the shared memory per stage); ballot-sorted lists for delays of
// 2^23 samples or more; 7-DM blocks (half the in-block spread).  Measured on
// GB300 (fraction of the integer-issue roofline): 64-channel stages with two
// slots 0.675 against 0.617 for 32-channel stages with five (2500 trials to DM
// 1500); on the wide band 32-channel stages with two slots 0.610, 7-DM blocks
// 0.40 (one CTA per SM) and 0.49 (two per SM, 4 words per lane).
const int kAutoList[] = {kDefaultVariant, 42, 34, 44, 40, 41};

// Variants the batch autotuner times (those that fit the batch are timed).
const int kTuneList[] = {kDefaultVariant, 42, 35, 31, 22, 43, 44, 36, 34, 40};

// Shared memory of one CTA: all of an SM's 227 KB, or half of it (less the
// per-CTA reserve) for CTAs of at most 8 warps that run two per SM.
constexpr int64_t kSmemOne = 227 * 1024;
constexpr int64_t kSmemTwo = 112 * 1024;

TileFit fit_variant(const TiledVariant &v, int64_t spread) {
    TileFit f;
    const int kT = 128 * v.m;
    const int64_t win = (kT + 15 + spread + 15) & ~(int64_t)15;
    const int64_t fixed = (int64_t)v.kdm * 4 * v.cb * 4 + 2 * 8 * 8;
    const bool small = (v.kdm / v.kw + 1) * 32 <= 256;
    // small CTAs run two per SM when two stages fit in half the shared memory,
    // else one per SM with all of it
    for (int two = small ? 1 : 0; two >= 0; two--) {
        const int64_t budget = two ? kSmemTwo : kSmemOne;
        const int64_t stages = std::min<int64_t>(8, (budget - fixed) / ((int64_t)v.cb * win));
        if (stages >= 2) {
            f.ok = true;
            f.win = (int)win;
            f.stages = (int)stages;
            f.smem = (int)(stages * v.cb * win + fixed);
            f.ctas_per_sm = two ? 2 : 1;
            return f;
        }
    }
    return f;
}

bool lists_ok(const TiledVariant &v, bool have_lists) { return !v.pre || have_lists; }

// The first variant of the automatic list that fits; -1 if none does.
int choose_auto(const int64_t (&spread)[kNumKdm], const bool (&have_lists)[kNumCb]) {
    for (int v : kAutoList) {
        const TiledVariant &tv = kVariants[v];
        if (!lists_ok(tv, have_lists[cb_index(tv.cb)])) continue;
        if (fit_variant(tv, spread[kdm_index(tv.kdm)]).ok) return v;
    }
    return -1;
}

}  // namespace

void plan_phase_lists(const gsp_plan_s *p, int cb, std::vector<int32_t> *dpos,
                      std::vector<uint32_t> *fcnt) {
    // Phase-sorted lists of cb-channel stages, per DM: channel c of stage st
    // (in channel order within its family) is filed at position
    // P * cb + rank, P = delay & 3, and the stage's four family sizes are
    // packed 8 bits each.  The phase of a (channel, DM) pair is the same in
    // every time tile because tiles start at multiples of 4 samples and the
    // staged windows at multiples of 16 bytes.
    const int C = p->desc.nchan, ndm = p->desc.ndm;
    const int nst = (C + cb - 1) / cb;
    dpos->clear();
    fcnt->clear();
    if (p->max_delay >= ((int64_t)1 << 23)) return;  // packed delay field is 23 bits
    dpos->resize((size_t)ndm * C);
    fcnt->resize((size_t)ndm * nst);
    for (int d = 0; d < ndm; d++) {
        const int32_t *dl = p->delays_h.data() + (size_t)d * C;
        for (int st = 0; st < nst; st++) {
            uint32_t cnt[4] = {0, 0, 0, 0};
            for (int c = st * cb; c < std::min(C, st * cb + cb); c++) {
                const int P = dl[c] & 3;
                (*dpos)[(size_t)d * C + c] = (int32_t)(((uint32_t)dl[c] << 8) | (uint32_t)(P * cb + cnt[P]));
                cnt[P]++;
            }
            (*fcnt)[(size_t)d * nst + st] = cnt[0] | (cnt[1] << 8) | (cnt[2] << 16) | (cnt[3] << 24);
        }
    }
}

bool plan_dedisperse_tiled(gsp_plan_s *p, TiledTables *tab) {
    const int C = p->desc.nchan, ndm = p->desc.ndm;
    DDGeom &g = p->geom;
    // DM blocks of each supported block size: per-block minimum delay of every
    // channel, the largest delay spread inside a block (overall and per stage
    // of either width), and the L2 grouping
    for (int o = 0; o < kNumKdm; o++) {
        const int kdm = kKdmSizes[o];
        const int nblk = (ndm + kdm - 1) / kdm;
        std::vector<int32_t> &bm = tab->blkmin[o];
        bm.assign((size_t)nblk * C, 0);
        std::vector<int64_t> chspread((size_t)C, 0);  // per channel, over all blocks
        for (int b = 0; b < nblk; b++) {
            for (int c = 0; c < C; c++) {
                int32_t lo = INT32_MAX, hi = 0;
                for (int d = b * kdm; d < std::min(ndm, (b + 1) * kdm); d++) {
                    const int32_t v = p->delays_h[(size_t)d * C + c];
                    lo = std::min(lo, v);
                    hi = std::max(hi, v);
                }
                bm[(size_t)b * C + c] = lo;
                chspread[c] = std::max<int64_t>(chspread[c], (int64_t)hi - lo);
            }
        }
        int64_t spread = 0;
        for (int c = 0; c < C; c++) spread = std::max(spread, chspread[c]);
        for (int i = 0; i < kNumCb; i++) {
            const int cb = kCbSizes[i];
            std::vector<int32_t> &ss = tab->stspread[o][i];
            ss.assign((size_t)((C + cb - 1) / cb), 0);
            for (int c = 0; c < C; c++)
                ss[c / cb] = std::max(ss[c / cb], (int32_t)chspread[c]);
        }
        g.nblk[o] = nblk;
        g.spread[o] = spread;
        // largest group of DM blocks whose per-tile input union (sum over channels
        // of the delay range across the group plus a 512-sample window) stays
        // within ~24 MB of L2
        const int64_t win = (512 + 15 + spread + 15) & ~(int64_t)15;
        g.grp[o] = 1;
        for (int G = nblk; G >= 1; G--) {
            int64_t worst = 0;
            for (int b0 = 0; b0 < nblk; b0 += G) {
                int64_t u = 0;
                const int d_hi = std::min(ndm, (b0 + G) * kdm) - 1;
                for (int c = 0; c < C; c++) {
                    const int64_t lo = bm[(size_t)b0 * C + c];
                    const int64_t hi = p->delays_h[(size_t)d_hi * C + c];
                    u += std::max<int64_t>(hi - lo, 0) + win;
                }
                worst = std::max(worst, u);
            }
            if (worst <= ((int64_t)24 << 20) || G == 1) {
                g.grp[o] = G;
                break;
            }
        }
    }
    bool have_lists[kNumCb];
    for (int i = 0; i < kNumCb; i++) {
        plan_phase_lists(p, kCbSizes[i], &tab->dpos[i], &tab->fcnt[i]);
        have_lists[i] = !tab->dpos[i].empty();
    }
    // GSP_DD_VARIANT selects a tuning variant of the tiled kernel if it fits
    // this plan; otherwise the automatic choice.
    int variant = -1;
    if (const char *v = std::getenv("GSP_DD_VARIANT")) {
        const int k = std::atoi(v);
        if (k >= 0 && k < kNumVariants && lists_ok(kVariants[k], have_lists[cb_index(kVariants[k].cb)]) &&
            fit_variant(kVariants[k], g.spread[kdm_index(kVariants[k].kdm)]).ok)
            variant = k;
    }
    if (variant < 0) variant = choose_auto(g.spread, have_lists);
    if (variant < 0) {
        *tab = TiledTables();
        return false;
    }
    const TiledVariant &v = kVariants[variant];
    const TileFit f = fit_variant(v, g.spread[kdm_index(v.kdm)]);
    g.kdm = v.kdm;
    g.t_cta = 128 * v.m;
    g.t_eff = 128 * v.m - 4;
    g.cb = v.cb;
    g.win = f.win;
    g.stages = f.stages;
    g.smem = f.smem;
    g.ctas_per_sm = f.ctas_per_sm;
    g.variant = variant;
    return true;
}

int dedisperse_num_variants() { return kNumVariants; }

int dedisperse_tune_candidates(const int **list) {
    *list = kTuneList;
    return (int)(sizeof(kTuneList) / sizeof(kTuneList[0]));
}

TileFit dedisperse_fit(int variant, const int64_t (&spread)[kNumKdm]) {
    if (variant < 0 || variant >= kNumVariants) return TileFit();
    const TiledVariant &v = kVariants[variant];
    return fit_variant(v, spread[kdm_index(v.kdm)]);
}

bool dedisperse_variant_usable(const gsp_plan_s *p, int variant) {
    if (!p || p->simple_dd || variant < 0 || variant >= kNumVariants) return false;
    const TiledVariant &v = kVariants[variant];
    const int o = kdm_index(v.kdm), ci = cb_index(v.cb);
    if (!p->d_blkmin[o] || !p->d_stspread[o][ci]) return false;
    if (v.pre && (!p->d_dpos[ci] || !p->d_fcnt[ci])) return false;
    return fit_variant(v, p->geom.spread[o]).ok;
}

void dedisperse_set_variant(gsp_plan_s *p, int variant) {
    const TiledVariant &v = kVariants[variant];
    const TileFit f = fit_variant(v, p->geom.spread[kdm_index(v.kdm)]);
    DDGeom &g = p->geom;
    g.kdm = v.kdm;
    g.t_cta = 128 * v.m;
    g.t_eff = 128 * v.m - 4;
    g.cb = v.cb;
    g.win = f.win;
    g.stages = f.stages;
    g.smem = f.smem;
    g.ctas_per_sm = f.ctas_per_sm;
    g.variant = variant;
}

int dedisperse_choose_variant(const gsp_plan_s *const *plans, int nplans) {
    if (nplans < 1) return -1;
    int64_t spread[kNumKdm] = {};
    bool have_lists[kNumCb] = {true, true};
    for (int i = 0; i < nplans; i++) {
        if (!plans[i] || plans[i]->simple_dd) return -1;
        for (int o = 0; o < kNumKdm; o++) spread[o] = std::max(spread[o], plans[i]->geom.spread[o]);
        for (int c = 0; c < kNumCb; c++) have_lists[c] = have_lists[c] && plans[i]->d_dpos[c];
    }
    // the plans' common variant if it fits the batch, else the automatic choice
    const int v0 = plans[0]->geom.variant;
    bool same = true;
    for (int i = 1; i < nplans; i++) same = same && plans[i]->geom.variant == v0;
    if (same && lists_ok(kVariants[v0], have_lists[cb_index(kVariants[v0].cb)]) &&
        fit_variant(kVariants[v0], spread[kdm_index(kVariants[v0].kdm)]).ok)
        return v0;
    return choose_auto(spread, have_lists);
}

cudaError_t launch_dedisperse_batch(const BeamLaunch *beams, int nbeams, int variant,
                                    bool persistent, int num_sms, int *err, cudaStream_t s,
                                    int32_t *nlaunch) {
    if (nbeams < 1 || nbeams > kMaxBatchBeams || variant < 0 || variant >= kNumVariants)
        return cudaErrorInvalidValue;
    const TiledVariant &v = kVariants[variant];
    const int o = kdm_index(v.kdm), ci = cb_index(v.cb);
    const int t_cta = 128 * v.m, t_eff = t_cta - 4;
    const int nchan = beams[0].plan->desc.nchan;
    int64_t spread = 0;
    for (int b = 0; b < nbeams; b++) {
        const gsp_plan_s *p = beams[b].plan;
        if (p->desc.nchan != nchan || !p->d_blkmin[o] || !p->d_stspread[o][ci])
            return cudaErrorInvalidValue;
        if (v.pre && (!p->d_dpos[ci] || !p->d_fcnt[ci])) return cudaErrorInvalidValue;
        spread = std::max(spread, p->geom.spread[o]);
    }
    const TileFit f = fit_variant(v, spread);
    if (!f.ok) return cudaErrorInvalidValue;
    {
        cudaError_t e = ensure_kernel_smem(reinterpret_cast<const void *>(v.fn), f.smem);
        if (e != cudaSuccess) return e;
    }
    TiledArgs a;
    std::memset(&a, 0, sizeof(a));
    int64_t items = 0;
    for (int b = 0; b < nbeams; b++) {
        const BeamLaunch &in = beams[b];
        const gsp_plan_s *p = in.plan;
        BeamTile &bt = a.beam[b];
        bt.x = in.x;
        bt.x_stride = in.x_stride;
        bt.n_in = in.n_in;
        bt.n_out = in.n_out;
        bt.delays = p->d_delays;
        bt.blkmin = p->d_blkmin[o];
        bt.dpos = p->d_dpos[ci];
        bt.fcnt = p->d_fcnt[ci];
        bt.stspread = p->d_stspread[o][ci];
        bt.out = in.out;
        bt.out_stride = in.out_stride;
        bt.bsum = in.bsum;
        bt.nb_max = p->nb_max;
        bt.B = p->desc.block_len;
        bt.Ls = (in.n_out / bt.B) * bt.B;
        bt.ntiles = (in.n_out + t_eff - 1) / t_eff;
        bt.item0 = items;
        bt.ndm = p->desc.ndm;
        bt.nblk = p->geom.nblk[o];
        bt.grp = p->geom.grp[o];
        if (in.bsum && bt.B < t_eff) return cudaErrorInvalidValue;
        items += bt.ntiles * bt.nblk;
    }
    a.nbeams = nbeams;
    a.nchan = nchan;
    a.win = f.win;
    a.stages = f.stages;
    a.one = 1u;
    a.err = err;
    a.items = items;
    a.budget = beams[0].plan->wait_budget;
    a.starve = beams[0].plan->wait_starve;
    int64_t grid = persistent ? std::min<int64_t>(items, (int64_t)num_sms * f.ctas_per_sm) : items;
    if (grid < 1 || grid > 0x7fffffffll) return cudaErrorInvalidConfiguration;
    v.fn<<<(unsigned)grid, (v.kdm / v.kw + 1) * 32, f.smem, s>>>(a);
    *nlaunch += 1;
    return cudaGetLastError();
}

cudaError_t launch_dedisperse_tiled(const gsp_plan_s *p, const uint8_t *x, int64_t n_in,
                                    int64_t x_stride, int64_t n_out, int32_t *out,
                                    int64_t out_stride, unsigned long long *bsum,
                                    cudaStream_t s, int32_t *nlaunch) {
    BeamLaunch b;
    b.plan = p;
    b.x = x;
    b.n_in = n_in;
    b.x_stride = x_stride;
    b.n_out = n_out;
    b.out = out;
    b.out_stride = out_stride;
    b.bsum = bsum;
    return launch_dedisperse_batch(&b, 1, p->geom.variant, false, p->num_sms, p->d_err, s,
                                   nlaunch);
}

}  // namespace gsp
