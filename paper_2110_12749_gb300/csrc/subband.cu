// DDplan ranges (time downsampling, one plan per DM range) and two-stage
// sub-band dedispersion: the survey plan of Sec. 3.1 (Tables 2 and 3: per
// range a DM step and a downsampling factor) and the sub-band algorithm of
// PRESTO's prepsubband that GSP accelerates (Sec. 2.3).
//
// Sub-band dedispersion.  The channels form nsub sub-bands of cs = nchan/nsub
// consecutive channels; the reference channel of a sub-band is its highest-
// frequency channel.  DM trials are taken in groups of `group` consecutive
// trials, and the middle trial of each group is its sub-band DM:
//   stage 1: S[s][g][t] = sum_{c in s} X[c][t + d1[g][c]],
//            d1[g][c] = delay_c(sdm_g) - delay_ref(s)(sdm_g),
//   stage 2: D[d][t]    = sum_s S[s][g(d)][t + d2[d][s]],  d2[d][s] = delay_ref(s)(DM_d).
// Stage 1 is the tiled dedispersion kernel itself, launched over the
// sub-bands as the "beams" of one persistent batched launch (one internal
// plan per sub-band, with the explicit delay table d1).  Stage 2 is
// subband_sum_kernel below.  A trial that is its group's sub-band DM gets
// exactly the brute-force delay of every channel; the others are
// approximated with the sub-band's reference delay (smearing within a
// sub-band), which is what makes the method cheaper: nsdm*nchan + ndm*nsub
// additions per output sample instead of ndm*nchan.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gsp_internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Time downsampling: out[c][t] = floor((2 * sum_{k<ds} x[c][t*ds + k] + ds) / (2*ds)),
// the mean rounded half up.  One thread per four output samples of a channel.
__global__ void __launch_bounds__(256) downsample_kernel(const uint8_t *__restrict__ x,
                                                         int64_t x_stride, int64_t n_ds, int ds,
                                                         uint8_t *__restrict__ out,
                                                         int64_t out_stride, bool word_out) {
    const int64_t c = blockIdx.y;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (t >= n_ds) return;
    const uint8_t *xc = x + c * x_stride + t * ds;
    const uint32_t two_ds = 2u * (uint32_t)ds;
    uint32_t word = 0;
    const int nj = (int)min((int64_t)4, n_ds - t);
    for (int j = 0; j < nj; j++) {
        const uint8_t *p = xc + (int64_t)j * ds;
        uint32_t sum = 0;
        for (int k = 0; k < ds; k++) sum += __ldg(p + k);
        word |= ((2u * sum + (uint32_t)ds) / two_ds) << (8 * j);
    }
    uint8_t *o = out + c * out_stride + t;
    if (word_out && nj == 4) {
        *reinterpret_cast<uint32_t *>(o) = word;
    } else {
        for (int j = 0; j < nj; j++) o[j] = (uint8_t)(word >> (8 * j));
    }
}

// ---------------------------------------------------------------------------
// Stage 2 of sub-band dedispersion.  One CTA per (group g, 1024 output
// samples); thread i owns outputs t0 + i + 256 j (j < 4) of every trial of
// the group.  The group's rows S[s][g][t0 + min2[g][s] .. + 1024 + spread)
// are staged in shared memory a chunk of sub-bands at a time, so the rows
// are read from L2 once per group instead of once per trial; a trial then
// reads its row at the offset off2[d][s] = d2[d][s] - min2[g][s].
constexpr int kMaxGroup = 16;
constexpr int kS2Threads = 256;
constexpr int kS2Tile = 4 * kS2Threads;

__global__ void __launch_bounds__(kS2Threads) subband_sum_kernel(
    const int32_t *__restrict__ S, int64_t s_stride, int nsdm, int nsub, int64_t n1,
    const int32_t *__restrict__ min2, const int32_t *__restrict__ off2, int ndm, int group,
    int row_len, int chunk, int64_t n_out, int32_t *__restrict__ D, int64_t d_stride) {
    extern __shared__ __align__(16) int32_t sm[];
    int32_t *soff = sm;                         // [group][nsub] offsets of the group's trials
    int32_t *rows = sm + kMaxGroup * nsub;      // [chunk][row_len]
    const int g = blockIdx.y;
    const int64_t t0 = (int64_t)blockIdx.x * kS2Tile;
    const int d0 = g * group;
    const int gcount = min(group, ndm - d0);
    for (int i = threadIdx.x; i < gcount * nsub; i += kS2Threads)
        soff[i] = off2[(int64_t)d0 * nsub + i];
    int32_t acc[kMaxGroup][4];
#pragma unroll
    for (int i = 0; i < kMaxGroup; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0;
    for (int s0 = 0; s0 < nsub; s0 += chunk) {
        const int sc = min(chunk, nsub - s0);
        __syncthreads();  // previous chunk consumed (and soff written)
        for (int r = 0; r < sc; r++) {
            const int s = s0 + r;
            const int64_t base = t0 + min2[(int64_t)g * nsub + s];
            const int32_t *src = S + ((int64_t)s * nsdm + g) * s_stride;
            int32_t *dst = rows + r * row_len;
            for (int i = threadIdx.x; i < row_len; i += kS2Threads) {
                const int64_t t = base + i;
                dst[i] = t < n1 ? __ldg(src + t) : 0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kMaxGroup; i++) {
            if (i < gcount) {
                for (int r = 0; r < sc; r++) {
                    const int32_t *row = rows + r * row_len + soff[i * nsub + s0 + r] + threadIdx.x;
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] += row[kS2Threads * j];
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kMaxGroup; i++) {
        if (i < gcount) {
            int32_t *o = D + (int64_t)(d0 + i) * d_stride;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int64_t t = t0 + threadIdx.x + kS2Threads * j;
                if (t < n_out) o[t] = acc[i][j];
            }
        }
    }
}

}  // namespace

struct gsp_subband_s {
    int32_t nchan = 0, nsub = 0, cs = 0, group = 0, ndm = 0, nsdm = 0;
    int64_t nsamp_max = 0;
    int64_t max1 = 0, max2 = 0;   // largest stage-1 / stage-2 delay
    std::vector<int32_t> d1, d2, sdm_idx, min2, off2;
    std::vector<gsp_plan_t> stage1;  // one plan per sub-band (explicit delays d1)
    int32_t *d_S = nullptr;          // [nsub][nsdm][s_stride] stage-1 series
    int64_t s_stride = 0;
    int32_t *d_min2 = nullptr;       // [nsdm][nsub]
    int32_t *d_off2 = nullptr;       // [ndm][nsub]
    int *d_err = nullptr;
    int row_len = 0, chunk = 0, smem = 0;
    int num_sms = 0;
    int32_t launches = 0;
};

namespace {

void free_subband(gsp_subband_s *b) {
    if (!b) return;
    for (gsp_plan_t p : b->stage1)
        if (p) gsp_plan_destroy(p);
    cudaFree(b->d_S);
    cudaFree(b->d_min2);
    cudaFree(b->d_off2);
    cudaFree(b->d_err);
    delete b;
}

template <typename T>
gsp_status sb_alloc(T **ptr, size_t count) {
    cudaError_t e = cudaMalloc((void **)ptr, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        gsp::record_error(e, "cudaMalloc");
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
    }
    return GSP_OK;
}

bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" {

gsp_status gsp_downsample(const uint8_t *d_x, int32_t nchan, int64_t n_in, int64_t x_stride,
                          int32_t ds, uint8_t *d_out, int64_t out_stride, void *stream) {
    // ds <= 2^20 keeps 2 * sum + ds (at most 2 * 255 * ds + ds) within 32 bits
    if (!d_x || !d_out || nchan <= 0 || n_in < 0 || ds < 1 || ds > (1 << 20) ||
        x_stride < n_in || out_stride < n_in / ds || nchan > 65535)
        return GSP_ERR_INVALID_ARG;
    const int64_t n_ds = n_in / ds;
    if (n_ds == 0) return GSP_OK;
    const int64_t quads = (n_ds + 3) / 4;
    dim3 grid((unsigned)((quads + 255) / 256), (unsigned)nchan);
    const bool word_out = ((uintptr_t)d_out & 3u) == 0 && (out_stride & 3) == 0;
    downsample_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_x, x_stride, n_ds, ds, d_out,
                                                              out_stride, word_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gsp::record_error(e, "downsample launch");
        return GSP_ERR_CUDA;
    }
    return GSP_OK;
}

gsp_status gsp_subband_create(gsp_subband_t *out, const gsp_plan_desc *desc, int32_t nsub,
                              int32_t group) {
    if (!out || !desc) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (desc->delays || desc->nchan <= 0 || desc->ndm <= 0 || nsub <= 0 ||
        desc->nchan % nsub != 0 || group < 1 || group > kMaxGroup || desc->nsamp_max <= 0)
        return GSP_ERR_INVALID_ARG;
    const int C = desc->nchan, ndm = desc->ndm;
    // brute-force delay table of every trial (the sub-band DMs are trials)
    std::vector<int32_t> T((size_t)C * ndm);
    double margin = 1.0;
    gsp_status st = gsp_compute_delays(desc, T.data(), &margin);
    if (st != GSP_OK) return st;
    if (margin < 1e-9) return GSP_ERR_TIE;
    gsp_subband_s *b = new (std::nothrow) gsp_subband_s();
    if (!b) return GSP_ERR_OOM;
    b->nchan = C;
    b->nsub = nsub;
    b->cs = C / nsub;
    b->group = group;
    b->ndm = ndm;
    b->nsdm = (ndm + group - 1) / group;
    b->nsamp_max = desc->nsamp_max;
    const int cs = b->cs, nsdm = b->nsdm;
    auto ref = [&](int s) { return desc->freq_descending ? s * cs : s * cs + cs - 1; };
    b->sdm_idx.resize(nsdm);
    for (int g = 0; g < nsdm; g++) b->sdm_idx[g] = std::min(g * group + group / 2, ndm - 1);
    b->d1.resize((size_t)nsdm * C);
    b->d2.resize((size_t)ndm * nsub);
    for (int s = 0; s < nsub; s++) {
        const int r = ref(s);
        for (int g = 0; g < nsdm; g++) {
            const int32_t *row = T.data() + (size_t)b->sdm_idx[g] * C;
            for (int c = s * cs; c < s * cs + cs; c++) {
                const int32_t v = row[c] - row[r];
                if (v < 0) {
                    free_subband(b);
                    return GSP_ERR_INVALID_ARG;
                }
                b->d1[(size_t)g * C + c] = v;
                b->max1 = std::max<int64_t>(b->max1, v);
            }
        }
        for (int d = 0; d < ndm; d++) {
            b->d2[(size_t)d * nsub + s] = T[(size_t)d * C + r];
            b->max2 = std::max<int64_t>(b->max2, T[(size_t)d * C + r]);
        }
    }
    // stage-2 offsets: per (group, sub-band) the smallest stage-2 delay, and
    // per trial its offset from it
    b->min2.assign((size_t)nsdm * nsub, INT32_MAX);
    b->off2.resize((size_t)ndm * nsub);
    int64_t spread = 0;
    for (int d = 0; d < ndm; d++)
        for (int s = 0; s < nsub; s++) {
            int32_t &m = b->min2[(size_t)(d / group) * nsub + s];
            m = std::min(m, b->d2[(size_t)d * nsub + s]);
        }
    for (int d = 0; d < ndm; d++)
        for (int s = 0; s < nsub; s++) {
            const int32_t o = b->d2[(size_t)d * nsub + s] - b->min2[(size_t)(d / group) * nsub + s];
            b->off2[(size_t)d * nsub + s] = o;
            spread = std::max<int64_t>(spread, o);
        }
    b->row_len = (int)(((int64_t)kS2Tile + spread + 3) & ~(int64_t)3);
    const int64_t fixed = (int64_t)kMaxGroup * nsub * 4;
    const int64_t budget = 100 * 1024 - fixed;
    b->chunk = (int)std::max<int64_t>(1, std::min<int64_t>(nsub, budget / ((int64_t)b->row_len * 4)));
    b->smem = (int)(fixed + (int64_t)b->chunk * b->row_len * 4);
    if (spread > (1 << 20) || b->smem > 227 * 1024) {
        free_subband(b);
        return GSP_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        gsp::record_error(e, "cudaGetDevice");
        free_subband(b);
        return GSP_ERR_CUDA;
    }
    // stage-1 plans: the channels of one sub-band, the sub-band DMs, delays d1
    std::vector<int32_t> cols((size_t)nsdm * cs);
    for (int s = 0; s < nsub; s++) {
        for (int g = 0; g < nsdm; g++)
            std::memcpy(cols.data() + (size_t)g * cs, b->d1.data() + (size_t)g * C + s * cs,
                        (size_t)cs * sizeof(int32_t));
        gsp_plan_desc pd = *desc;
        pd.nchan = cs;
        pd.ndm = nsdm;
        pd.dms = nullptr;
        pd.delays = cols.data();
        pd.max_cands = 1;
        pd.flags = 0;
        gsp_plan_t p = nullptr;
        st = gsp_plan_create(&p, &pd);
        if (st != GSP_OK) {
            free_subband(b);
            return st;
        }
        b->stage1.push_back(p);
    }
    b->s_stride = (desc->nsamp_max + 3) & ~(int64_t)3;
    st = sb_alloc(&b->d_S, (size_t)nsub * nsdm * b->s_stride);
    if (st == GSP_OK) st = sb_alloc(&b->d_min2, b->min2.size());
    if (st == GSP_OK) st = sb_alloc(&b->d_off2, b->off2.size());
    if (st == GSP_OK) st = sb_alloc(&b->d_err, 1);
    if (st != GSP_OK) {
        free_subband(b);
        return st;
    }
    e = cudaMemcpy(b->d_min2, b->min2.data(), b->min2.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_off2, b->off2.data(), b->off2.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(int));
    if (e == cudaSuccess && b->smem > 48 * 1024)
        e = cudaFuncSetAttribute(subband_sum_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 b->smem);
    if (e != cudaSuccess) {
        gsp::record_error(e, "subband upload");
        free_subband(b);
        return GSP_ERR_CUDA;
    }
    *out = b;
    return GSP_OK;
}

gsp_status gsp_subband_destroy(gsp_subband_t b) {
    if (!b) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    free_subband(b);
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

int64_t gsp_subband_nout(gsp_subband_t b, int64_t n_in) {
    if (!b) return -1;
    return n_in - b->max1 - b->max2;
}

gsp_status gsp_subband_delays(gsp_subband_t b, int32_t *d1, int32_t *d2, int32_t *sdm_idx) {
    if (!b) return GSP_ERR_INVALID_ARG;
    if (d1) std::memcpy(d1, b->d1.data(), b->d1.size() * sizeof(int32_t));
    if (d2) std::memcpy(d2, b->d2.data(), b->d2.size() * sizeof(int32_t));
    if (sdm_idx) std::memcpy(sdm_idx, b->sdm_idx.data(), b->sdm_idx.size() * sizeof(int32_t));
    return GSP_OK;
}

gsp_status gsp_subband_dedisperse(gsp_subband_t b, const uint8_t *d_x, int64_t n_in,
                                  int64_t x_stride, int32_t *d_out, int64_t out_stride,
                                  void *stream) {
    if (!b || !d_x || !d_out || n_in <= 0 || n_in > b->nsamp_max || x_stride < n_in)
        return GSP_ERR_INVALID_ARG;
    if (!al16(d_x) || (x_stride & 15) || ((uintptr_t)d_out & 3)) return GSP_ERR_ALIGN;
    const int64_t n1 = n_in - b->max1;
    const int64_t n_out = n1 - b->max2;
    if (n_out <= 0) return GSP_ERR_TOO_SHORT;
    if (out_stride < n_out) return GSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    b->launches = 0;
    // stage 1: every sub-band's channels at the sub-band DMs
    std::vector<gsp::BeamLaunch> bl;
    for (int sb = 0; sb < b->nsub; sb++) {
        gsp_plan_s *p = b->stage1[sb];
        const uint8_t *xs = d_x + (int64_t)sb * b->cs * x_stride;
        int32_t *Ss = b->d_S + (int64_t)sb * b->nsdm * b->s_stride;
        if (p->simple_dd) {
            gsp_status st = gsp_dedisperse(p, xs, n_in, x_stride, Ss, b->s_stride, stream);
            if (st != GSP_OK) return st;
            b->launches += gsp_plan_launches(p);
            continue;
        }
        bl.push_back(gsp::BeamLaunch{p, xs, n_in, x_stride, n_in - p->max_delay, Ss, b->s_stride,
                                     nullptr});
    }
    for (size_t i = 0; i < bl.size(); i += 32) {
        const int n = (int)std::min<size_t>(32, bl.size() - i);
        // one variant that fits every sub-band of this launch
        std::vector<const gsp_plan_s *> ps((size_t)n);
        for (int k = 0; k < n; k++) ps[k] = bl[i + k].plan;
        const int variant = gsp::dedisperse_choose_variant(ps.data(), n);
        cudaError_t e = variant < 0 ? cudaErrorInvalidValue
                                    : gsp::launch_dedisperse_batch(bl.data() + i, n, variant, true,
                                                                   b->num_sms, b->d_err, s,
                                                                   &b->launches);
        if (e != cudaSuccess) {
            gsp::record_error(e, "sub-band stage 1 launch");
            return GSP_ERR_CUDA;
        }
    }
    // stage 2: sums of the sub-band series, shifted by the reference delays
    dim3 grid((unsigned)((n_out + kS2Tile - 1) / kS2Tile), (unsigned)b->nsdm);
    subband_sum_kernel<<<grid, kS2Threads, b->smem, s>>>(
        b->d_S, b->s_stride, b->nsdm, b->nsub, n1, b->d_min2, b->d_off2, b->ndm, b->group,
        b->row_len, b->chunk, n_out, d_out, out_stride);
    b->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gsp::record_error(e, "sub-band stage 2 launch");
        return GSP_ERR_CUDA;
    }
    return GSP_OK;
}

gsp_status gsp_subband_finish(gsp_subband_t b, void *stream) {
    if (!b) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        gsp::record_error(e, "sub-band finish");
        return GSP_ERR_CUDA;
    }
    if (flag) {
        cudaMemset(b->d_err, 0, sizeof(int));
        return GSP_ERR_TIMEOUT;
    }
    return GSP_OK;
}

int32_t gsp_subband_launches(gsp_subband_t b) { return b ? b->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// DDplan: a survey plan of DM ranges, each with its own DM step and time
// downsampling factor (Sec. 3.1, Tables 2-3).  One plan per range searches
// the input downsampled by the range's factor (computed once per distinct
// factor and search call).

struct gsp_ddplan_s {
    int32_t nchan = 0;
    int64_t nsamp_max = 0;
    std::vector<gsp_plan_t> plans;
    std::vector<int32_t> ds;
    std::vector<int64_t> dm0;      // first global trial index of each range
    std::vector<uint8_t *> buf;    // downsampled input per range (shared by equal factors)
    std::vector<int> owner;        // range whose buffer a range reads (-1 for ds == 1)
    std::vector<int64_t> stride;   // row stride of each buffer
};

namespace {

void free_ddplan(gsp_ddplan_s *d) {
    if (!d) return;
    for (gsp_plan_t p : d->plans)
        if (p) gsp_plan_destroy(p);
    for (size_t r = 0; r < d->buf.size(); r++)
        if (d->owner[r] == (int)r) cudaFree(d->buf[r]);
    delete d;
}

}  // namespace

extern "C" {

gsp_status gsp_ddplan_create(gsp_ddplan_t *out, const gsp_plan_desc *base,
                             const gsp_ddplan_range *ranges, int32_t nranges) {
    if (!out || !base || !ranges || nranges < 1 || nranges > 64 || base->delays ||
        base->nchan <= 0 || base->nsamp_max <= 0)
        return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    gsp_ddplan_s *d = new (std::nothrow) gsp_ddplan_s();
    if (!d) return GSP_ERR_OOM;
    d->nchan = base->nchan;
    d->nsamp_max = base->nsamp_max;
    int64_t next = 0;
    for (int r = 0; r < nranges; r++) {
        const gsp_ddplan_range &R = ranges[r];
        if (R.downsamp < 1 || R.downsamp > (1 << 20) || R.ndm < 1 || !(R.dm_step >= 0.0) ||
            base->nsamp_max / R.downsamp < 1) {
            free_ddplan(d);
            return GSP_ERR_INVALID_ARG;
        }
        gsp_plan_desc pd = *base;
        pd.t_samp_s = base->t_samp_s * (double)R.downsamp;
        pd.nsamp_max = base->nsamp_max / R.downsamp;
        pd.ndm = R.ndm;
        pd.dms = nullptr;
        pd.dm_lo = R.dm_lo;
        pd.dm_step = R.dm_step;
        gsp_plan_t p = nullptr;
        gsp_status st = gsp_plan_create(&p, &pd);
        if (st != GSP_OK) {
            free_ddplan(d);
            return st;
        }
        d->plans.push_back(p);
        d->ds.push_back(R.downsamp);
        d->dm0.push_back(next);
        next += R.ndm;
        int own = R.downsamp == 1 ? -1 : r;
        for (int q = 0; q < r && own == r; q++)
            if (d->ds[q] == R.downsamp) own = q;
        d->owner.push_back(own);
        d->buf.push_back(nullptr);
        d->stride.push_back(0);
        if (own == r) {
            const int64_t stride = (pd.nsamp_max + 15) & ~(int64_t)15;
            cudaError_t e = cudaMalloc((void **)&d->buf[r], (size_t)stride * base->nchan);
            if (e != cudaSuccess) {
                gsp::record_error(e, "cudaMalloc");
                (void)cudaGetLastError();
                free_ddplan(d);
                return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
            }
            d->stride[r] = stride;
        } else if (own >= 0) {
            d->buf[r] = d->buf[own];
            d->stride[r] = d->stride[own];
        }
    }
    *out = d;
    return GSP_OK;
}

gsp_status gsp_ddplan_destroy(gsp_ddplan_t d) {
    if (!d) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    free_ddplan(d);
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

gsp_status gsp_ddplan_search(gsp_ddplan_t d, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                             int64_t t_offset, void *stream) {
    if (!d || !d_x || n_in <= 0 || n_in > d->nsamp_max || x_stride < n_in || t_offset < 0)
        return GSP_ERR_INVALID_ARG;
    for (size_t r = 0; r < d->plans.size(); r++)
        if (t_offset % d->ds[r]) return GSP_ERR_INVALID_ARG;
    for (size_t r = 0; r < d->plans.size(); r++) {
        const int ds = d->ds[r];
        gsp_status st;
        if (ds == 1) {
            st = gsp_search(d->plans[r], d_x, n_in, x_stride, t_offset, nullptr, 0, stream);
        } else {
            if (d->owner[r] == (int)r) {
                st = gsp_downsample(d_x, d->nchan, n_in, x_stride, ds, d->buf[r], d->stride[r],
                                    stream);
                if (st != GSP_OK) return st;
            }
            st = gsp_search(d->plans[r], d->buf[r], n_in / ds, d->stride[r], t_offset / ds,
                            nullptr, 0, stream);
        }
        if (st != GSP_OK) return st;
    }
    return GSP_OK;
}

gsp_status gsp_ddplan_candidates(gsp_ddplan_t d, gsp_cand *host_out, int64_t cap,
                                 int64_t *n_total) {
    if (!d || !n_total || cap < 0 || (cap > 0 && !host_out)) return GSP_ERR_INVALID_ARG;
    int64_t total = 0;
    bool truncated = false;
    for (size_t r = 0; r < d->plans.size(); r++) {
        int64_t n = 0;
        gsp_status st = gsp_candidates(d->plans[r], nullptr, 0, &n);
        if (st != GSP_OK && st != GSP_ERR_CAPACITY) return st;
        std::vector<gsp_cand> v((size_t)n);
        int64_t n2 = 0;
        st = gsp_candidates(d->plans[r], v.data(), n, &n2);
        if (st == GSP_ERR_CAPACITY) truncated = true;
        else if (st != GSP_OK) return st;
        const int64_t kept = std::min(n, n2);
        for (int64_t i = 0; i < kept; i++) {
            gsp_cand c = v[(size_t)i];
            c.dm_idx += (int32_t)d->dm0[r];
            c.t *= d->ds[r];
            c.width *= d->ds[r];
            c.beam = (int32_t)r;
            if (total + i < cap) host_out[total + i] = c;
        }
        total += n2;
    }
    *n_total = total;
    return (truncated || total > cap) ? GSP_ERR_CAPACITY : GSP_OK;
}

}  // extern "C"
