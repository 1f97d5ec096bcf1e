// C ABI of libgsp: plans, host-side delay table, argument checking, and the
// orchestration of the dedispersion and search kernels (include/gsp.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "gsp_internal.cuh"

namespace {

thread_local char g_err[512] = "";

void set_err(cudaError_t e, const char *what) {
    std::snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
}

#define GSP_CK(call)                          \
    do {                                      \
        cudaError_t e_ = (call);              \
        if (e_ != cudaSuccess) {              \
            set_err(e_, #call);               \
            return GSP_ERR_CUDA;              \
        }                                     \
    } while (0)

const int32_t kDefaultWidths[13] = {1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150};

// Host-side fault hook for failure-path tests: GSP_FAULT=alloc makes plan
// allocation report GSP_ERR_OOM, GSP_FAULT=launch makes the first kernel
// launch of a call report GSP_ERR_CUDA, before any GPU work is enqueued.
bool fault(const char *what) {
    const char *f = std::getenv("GSP_FAULT");
    return f && std::strcmp(f, what) == 0;
}

// Delay table (Sec. 2.3: a numdm x numchan integer matrix of per-channel
// shifts).  Cold-plasma law relative to the highest channel centre, in
// samples, rounded half away from zero; FP64, no contraction (the library is
// compiled with -ffp-contract=off for host code).
gsp_status compute_delays(const gsp_plan_desc *d, const std::vector<double> &dms,
                          int32_t *out, double *min_margin) {
    const int64_t C = d->nchan;
    const double df = (d->f_hi_mhz - d->f_lo_mhz) / (double)C;
    const double ftop = d->f_lo_mhz + ((double)(C - 1) + 0.5) * df;
    const double inv_top2 = 1.0 / (ftop * ftop);
    double margin = 1.0;
    for (size_t i = 0; i < dms.size(); i++) {
        const double dm = dms[i];
        for (int64_t c = 0; c < C; c++) {
            const int64_t k = d->freq_descending ? (C - 1 - c) : c;
            const double f = d->f_lo_mhz + ((double)k + 0.5) * df;
            const double x = 4.148808e3 * dm * (1.0 / (f * f) - inv_top2) / d->t_samp_s;
            const double fl = std::floor(x);
            const double m = std::fabs((x - fl) - 0.5);
            if (m < margin) margin = m;
            const double r = std::floor(x + 0.5);
            if (!(r >= 0.0) || r > 2147483647.0) return GSP_ERR_INVALID_ARG;
            out[i * C + c] = (int32_t)r;
        }
    }
    if (min_margin) *min_margin = margin;
    return GSP_OK;
}

gsp_status desc_dms(const gsp_plan_desc *d, std::vector<double> *dms) {
    if (d->ndm <= 0) return GSP_ERR_INVALID_ARG;
    dms->resize((size_t)d->ndm);
    for (int32_t i = 0; i < d->ndm; i++) {
        double v = d->dms ? d->dms[i] : d->dm_lo + (double)i * d->dm_step;
        if (!std::isfinite(v) || v < 0.0) return GSP_ERR_INVALID_ARG;
        (*dms)[i] = v;
    }
    return GSP_OK;
}

gsp_status check_band(const gsp_plan_desc *d) {
    if (d->nchan <= 0 || !(d->f_lo_mhz > 0.0) || !(d->f_hi_mhz > d->f_lo_mhz) ||
        !std::isfinite(d->f_hi_mhz) || !(d->t_samp_s > 0.0) || !std::isfinite(d->t_samp_s))
        return GSP_ERR_INVALID_ARG;
    return GSP_OK;
}

void free_plan(gsp_plan_s *p) {
    if (!p) return;
    cudaFree(p->d_delays);
    for (auto *b : p->d_blkmin) cudaFree(b);
    for (auto *b : p->d_dpos) cudaFree(b);
    for (auto *b : p->d_fcnt) cudaFree(b);
    for (auto &row : p->d_stspread)
        for (auto *b : row) cudaFree(b);
    cudaFree(p->d_err);
    cudaFree(p->d_prefix);
    cudaFree(p->d_order);
    cudaFree(p->d_order_hist);
    cudaFree(p->d_sinv);
    cudaFree(p->d_bsum);
    cudaFree(p->d_sigma_b);
    cudaFree(p->d_bad);
    cudaFree(p->d_bparam);
    cudaFree(p->d_scale);
    cudaFree(p->d_sref);
    cudaFree(p->d_cands);
    cudaFree(p->d_ncand);
    cudaFree(p->d_slots);
    cudaFree(p->d_chunk);
    cudaFree(p->d_D);
    cudaFree(p->d_xstage);
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : p->h2d_ev)
        if (e) cudaEventDestroy(e);
    if (p->h2d_stream) cudaStreamDestroy(p->h2d_stream);
    delete p;
}

template <typename T>
gsp_status dalloc(T **ptr, size_t count) {
    if (fault("alloc")) return GSP_ERR_OOM;
    cudaError_t e = cudaMalloc((void **)ptr, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        set_err(e, "cudaMalloc");
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSP_ERR_OOM : GSP_ERR_CUDA;
    }
    return GSP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// After a synchronisation: did a kernel report a bounded wait that gave up?
// The flag is cleared so that the plan stays usable.
gsp_status take_kernel_error(gsp_plan_s *p) {
    int e = 0;
    cudaError_t ce = cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
        set_err(ce, "read kernel status");
        return GSP_ERR_CUDA;
    }
    if (e != 0) {
        cudaMemset(p->d_err, 0, sizeof(int));
        return GSP_ERR_TIMEOUT;
    }
    return GSP_OK;
}

gsp_status check_dd_args(gsp_plan_s *p, const uint8_t *x, int64_t n_in, int64_t x_stride,
                         const int32_t *out, int64_t out_stride, int64_t *n_out) {
    if (!p || !x || n_in <= 0 || n_in > p->desc.nsamp_max || x_stride < n_in)
        return GSP_ERR_INVALID_ARG;
    if (n_in <= p->max_delay) return GSP_ERR_TOO_SHORT;
    *n_out = n_in - p->max_delay;
    if (out && out_stride < *n_out) return GSP_ERR_INVALID_ARG;
    if (!aligned16(x) || (x_stride & 15)) return GSP_ERR_ALIGN;
    if (out && (!aligned16(out) || (out_stride & 3))) return GSP_ERR_ALIGN;
    return GSP_OK;
}

gsp_status ensure_scratch_D(gsp_plan_s *p, int64_t n_out) {
    size_t need = (size_t)p->desc.ndm * (size_t)n_out;
    if (need <= p->d_D_elems) return GSP_OK;
    cudaFree(p->d_D);
    p->d_D = nullptr;
    p->d_D_elems = 0;
    // size for the largest call the plan admits, so that it is allocated once
    const int64_t row = (std::max<int64_t>(p->desc.nsamp_max - p->max_delay, n_out) + 3) & ~(int64_t)3;
    const size_t full = (size_t)p->desc.ndm * (size_t)row;
    gsp_status st = dalloc(&p->d_D, full);
    if (st != GSP_OK) return st;
    p->d_D_elems = full;
    return GSP_OK;
}

// Block sums are fused into the tiled kernel when it can produce them (a
// tile of 508 samples then touches at most two search blocks).
bool fused_stats(const gsp_plan_s *p) {
    return !p->simple_dd && p->d_bsum != nullptr && p->desc.block_len >= p->geom.t_eff;
}

gsp_status run_dedisperse(gsp_plan_s *p, const uint8_t *x, int64_t n_in, int64_t x_stride,
                          int64_t n_out, int32_t *out, int64_t out_stride,
                          unsigned long long *bsum, cudaStream_t s) {
    if (fault("launch")) return GSP_ERR_CUDA;
    cudaError_t e;
    if (p->simple_dd)
        e = gsp::launch_dedisperse_simple(p, x, x_stride, n_out, out, out_stride, s, &p->launches);
    else
        e = gsp::launch_dedisperse_tiled(p, x, n_in, x_stride, n_out, out, out_stride, bsum, s,
                                         &p->launches);
    if (e != cudaSuccess) {
        set_err(e, "dedisperse launch");
        return GSP_ERR_CUDA;
    }
    return GSP_OK;
}

gsp_status run_search(gsp_plan_s *p, const int32_t *D, int64_t n_out, int64_t stride,
                      int64_t t_offset, float *snr_out, const unsigned long long *bsum,
                      cudaStream_t s) {
    if (fault("launch")) return GSP_ERR_CUDA;
    cudaError_t e =
        gsp::launch_search(p, D, n_out, stride, t_offset, snr_out, bsum, s, &p->launches);
    if (e != cudaSuccess) {
        set_err(e, "search launch");
        return GSP_ERR_CUDA;
    }
    p->last_stream = s;
    p->last_D = D;
    p->last_stride = stride;
    p->last_nout = n_out;
    p->last_nb = n_out / p->desc.block_len;
    p->have_search = true;
    p->search_seq++;
    return GSP_OK;
}

}  // namespace

namespace gsp {

void record_error(cudaError_t e, const char *what) { set_err(e, what); }

cudaError_t ensure_kernel_smem(const void *fn, int smem, bool max_carveout) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> done;  // (device, kernel) -> bytes
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find({dev, fn});
    if (it != done.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && max_carveout)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done[{dev, fn}] = smem;
    return e;
}

// Used by the batch module: make sure the plan's series scratch exists and
// tell whether block sums can be fused into the tiled dedispersion kernel.
gsp_status plan_prepare_search(gsp_plan_s *p, int64_t n_out, int32_t **D, int64_t *stride,
                               unsigned long long **bsum) {
    gsp_status st = ensure_scratch_D(p, n_out);
    if (st != GSP_OK) return st;
    *D = p->d_D;
    *stride = (n_out + 3) & ~(int64_t)3;
    *bsum = (fused_stats(p) && n_out / p->desc.block_len > 0) ? p->d_bsum : nullptr;
    return GSP_OK;
}

gsp_status plan_check_input(gsp_plan_s *p, const uint8_t *x, int64_t n_in, int64_t x_stride,
                            int64_t *n_out) {
    return check_dd_args(p, x, n_in, x_stride, nullptr, 0, n_out);
}

}  // namespace gsp

extern "C" {

gsp_status gsp_plan_desc_init(gsp_plan_desc *d) {
    if (!d) return GSP_ERR_INVALID_ARG;
    std::memset(d, 0, sizeof(*d));
    d->widths = nullptr;
    d->nwidths = 0;
    d->block_len = 1024;
    d->window_len = 1024;
    d->threshold = 6.0f;
    d->bad_lo = 0.5f;
    d->bad_hi = 2.5f;
    d->max_cands = 1 << 20;
    return GSP_OK;
}

gsp_status gsp_compute_delays(const gsp_plan_desc *d, int32_t *host_out, double *min_margin) {
    if (!d || !host_out) return GSP_ERR_INVALID_ARG;
    gsp_status st = check_band(d);
    if (st != GSP_OK) return st;
    std::vector<double> dms;
    st = desc_dms(d, &dms);
    if (st != GSP_OK) return st;
    return compute_delays(d, dms, host_out, min_margin);
}

gsp_status gsp_plan_create(gsp_plan_t *out, const gsp_plan_desc *d) {
    if (!out || !d) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->nchan <= 0 || d->ndm <= 0 || d->nsamp_max <= 0 || d->max_cands <= 0 ||
        d->block_len <= 0 || d->window_len <= 0 || !(d->bad_lo <= d->bad_hi) ||
        !std::isfinite(d->threshold) || d->nwidths < 0 || d->nwidths > gsp::kMaxWidths)
        return GSP_ERR_INVALID_ARG;
    if ((int64_t)d->nchan * (int64_t)d->ndm > ((int64_t)1 << 31) || d->ndm > 65535)
        return GSP_ERR_INVALID_ARG;
    gsp_plan_s *p = new (std::nothrow) gsp_plan_s();
    if (!p) return GSP_ERR_OOM;
    p->desc = *d;
    p->desc.dms = nullptr;
    p->desc.delays = nullptr;
    p->desc.widths = nullptr;
    // widths
    if (d->widths && d->nwidths > 0) {
        p->widths.assign(d->widths, d->widths + d->nwidths);
    } else {
        p->widths.assign(kDefaultWidths, kDefaultWidths + 13);
    }
    p->desc.nwidths = (int32_t)p->widths.size();
    for (size_t i = 0; i < p->widths.size(); i++) {
        if (p->widths[i] < 1 || (i && p->widths[i] <= p->widths[i - 1])) {
            delete p;
            return GSP_ERR_INVALID_ARG;
        }
    }
    if (p->widths.back() > d->block_len || p->widths.back() > 1024) {
        delete p;
        return GSP_ERR_INVALID_ARG;
    }
    // delay table
    const int64_t C = d->nchan, ndm = d->ndm;
    p->delays_h.resize((size_t)(C * ndm));
    if (d->delays) {
        for (int64_t i = 0; i < C * ndm; i++) {
            if (d->delays[i] < 0) {
                delete p;
                return GSP_ERR_INVALID_ARG;
            }
            p->delays_h[i] = d->delays[i];
        }
    } else {
        gsp_status st = check_band(d);
        if (st == GSP_OK) st = desc_dms(d, &p->dms);
        double margin = 1.0;
        if (st == GSP_OK) st = compute_delays(d, p->dms, p->delays_h.data(), &margin);
        if (st == GSP_OK && margin < 1e-9) st = GSP_ERR_TIE;
        if (st != GSP_OK) {
            delete p;
            return st;
        }
    }
    p->max_delay = *std::max_element(p->delays_h.begin(), p->delays_h.end());
    p->simple_dd = (d->flags & GSP_FLAG_SIMPLE_DD) != 0;
    p->timed = (d->flags & GSP_FLAG_TIMING) != 0;

    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        set_err(e, "cudaGetDevice");
        (void)cudaGetLastError();
        delete p;
        return GSP_ERR_CUDA;
    }
    // tiled-kernel tables; the simple kernel only when asked for, or when no
    // tiled variant fits the delay spread (gsp_dedisperse_variants reports it)
    gsp::TiledTables tab;
    if (!p->simple_dd && !gsp::plan_dedisperse_tiled(p, &tab)) p->simple_dd = true;

    p->nb_max = std::max<int64_t>(d->nsamp_max / d->block_len, 1);
    const size_t rows_blocks = (size_t)ndm * (size_t)p->nb_max;
    gsp_status st = GSP_OK;
    if (st == GSP_OK) st = dalloc(&p->d_delays, (size_t)(C * ndm));
    for (int o = 0; o < gsp::kNumKdm; o++) {
        if (st == GSP_OK && !tab.blkmin[o].empty()) st = dalloc(&p->d_blkmin[o], tab.blkmin[o].size());
        for (int i = 0; i < gsp::kNumCb; i++)
            if (st == GSP_OK && !tab.stspread[o][i].empty())
                st = dalloc(&p->d_stspread[o][i], tab.stspread[o][i].size());
    }
    for (int i = 0; i < gsp::kNumCb; i++) {
        if (st == GSP_OK && !tab.dpos[i].empty()) st = dalloc(&p->d_dpos[i], tab.dpos[i].size());
        if (st == GSP_OK && !tab.fcnt[i].empty()) st = dalloc(&p->d_fcnt[i], tab.fcnt[i].size());
    }
    if (st == GSP_OK) st = dalloc(&p->d_sigma_b, rows_blocks);
    if (st == GSP_OK) st = dalloc(&p->d_bad, rows_blocks);
    if (st == GSP_OK) st = dalloc(&p->d_bparam, rows_blocks);
    if (st == GSP_OK) st = dalloc(&p->d_scale, (size_t)ndm * p->widths.size());
    if (st == GSP_OK) st = dalloc(&p->d_sref, (size_t)ndm);
    if (st == GSP_OK) st = dalloc(&p->d_cands, (size_t)d->max_cands);
    if (st == GSP_OK) st = dalloc(&p->d_ncand, 1);
    p->nwin_max = d->nsamp_max / d->window_len + 2;
    const size_t nslots = (size_t)ndm * (size_t)p->nwin_max;
    if (st == GSP_OK && nslots >= ((size_t)1 << 31)) st = GSP_ERR_INVALID_ARG;
    if (st == GSP_OK) st = dalloc(&p->d_slots, nslots);
    if (st == GSP_OK) st = dalloc(&p->d_chunk, (nslots + 1023) / 1024);
    if (st == GSP_OK) st = dalloc(&p->d_err, 1);
    if (st == GSP_OK && !p->simple_dd) st = dalloc(&p->d_bsum, rows_blocks * 3);
    if (st != GSP_OK) {
        free_plan(p);
        return st;
    }
    e = cudaMemcpy(p->d_delays, p->delays_h.data(), (size_t)(C * ndm) * sizeof(int32_t),
                   cudaMemcpyHostToDevice);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes > 0) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    for (int o = 0; o < gsp::kNumKdm; o++) {
        up(p->d_blkmin[o], tab.blkmin[o].data(), tab.blkmin[o].size() * sizeof(int32_t));
        for (int i = 0; i < gsp::kNumCb; i++)
            up(p->d_stspread[o][i], tab.stspread[o][i].data(), tab.stspread[o][i].size() * sizeof(int32_t));
    }
    for (int i = 0; i < gsp::kNumCb; i++) {
        up(p->d_dpos[i], tab.dpos[i].data(), tab.dpos[i].size() * sizeof(int32_t));
        up(p->d_fcnt[i], tab.fcnt[i].data(), tab.fcnt[i].size() * sizeof(uint32_t));
    }
    if (e == cudaSuccess) e = cudaMemset(p->d_ncand, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    for (int i = 0; i < 3 && e == cudaSuccess; i++) e = cudaEventCreate(&p->ev[i]);
    if (e != cudaSuccess) {
        set_err(e, "plan upload");
        free_plan(p);
        return GSP_ERR_CUDA;
    }
    *out = p;
    return GSP_OK;
}

gsp_status gsp_plan_destroy(gsp_plan_t p) {
    if (!p) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(p);
    if (e != cudaSuccess) {
        set_err(e, "cudaDeviceSynchronize");
        return GSP_ERR_CUDA;
    }
    return GSP_OK;
}

int64_t gsp_plan_max_delay(gsp_plan_t p) { return p ? p->max_delay : -1; }

int64_t gsp_plan_nout(gsp_plan_t p, int64_t n_in) { return p ? n_in - p->max_delay : -1; }

gsp_status gsp_plan_delays(gsp_plan_t p, int32_t *host_out) {
    if (!p || !host_out) return GSP_ERR_INVALID_ARG;
    std::memcpy(host_out, p->delays_h.data(), p->delays_h.size() * sizeof(int32_t));
    return GSP_OK;
}

gsp_status gsp_dedisperse(gsp_plan_t p, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                          int32_t *d_out, int64_t out_stride, void *stream) {
    int64_t n_out = 0;
    if (!d_out) return GSP_ERR_INVALID_ARG;
    gsp_status st = check_dd_args(p, d_x, n_in, x_stride, d_out, out_stride, &n_out);
    if (st != GSP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    p->launches = 0;
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[0], s));
    st = run_dedisperse(p, d_x, n_in, x_stride, n_out, d_out, out_stride, nullptr, s);
    if (st != GSP_OK) return st;
    if (p->timed) {
        GSP_CK(cudaEventRecord(p->ev[1], s));
        GSP_CK(cudaEventRecord(p->ev[2], s));
    }
    p->last_stream = s;
    return GSP_OK;
}

gsp_status gsp_search(gsp_plan_t p, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                      int64_t t_offset, int32_t *d_out, int64_t out_stride, void *stream) {
    int64_t n_out = 0;
    gsp_status st = check_dd_args(p, d_x, n_in, x_stride, d_out, out_stride, &n_out);
    if (st != GSP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *D = d_out;
    int64_t stride = out_stride;
    if (!D) {
        st = ensure_scratch_D(p, n_out);
        if (st != GSP_OK) return st;
        D = p->d_D;
        stride = (n_out + 3) & ~(int64_t)3;
    }
    p->launches = 0;
    unsigned long long *bsum = nullptr;
    const int64_t nb = n_out / p->desc.block_len;
    if (fused_stats(p) && nb > 0) {
        bsum = p->d_bsum;
        GSP_CK(cudaMemsetAsync(bsum, 0, (size_t)p->desc.ndm * p->nb_max * 3 * sizeof(*bsum), s));
    }
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[0], s));
    st = run_dedisperse(p, d_x, n_in, x_stride, n_out, D, stride, bsum, s);
    if (st != GSP_OK) return st;
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[1], s));
    st = run_search(p, D, n_out, stride, t_offset, nullptr, bsum, s);
    if (st != GSP_OK) return st;
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[2], s));
    return GSP_OK;
}

gsp_status gsp_search_series(gsp_plan_t p, const int32_t *d_D, int64_t n_out, int64_t stride,
                             int64_t t_offset, void *stream) {
    if (!p || !d_D || n_out <= 0 || stride < n_out) return GSP_ERR_INVALID_ARG;
    if (n_out / p->desc.block_len > p->nb_max) return GSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    p->launches = 0;
    if (p->timed) {
        GSP_CK(cudaEventRecord(p->ev[0], s));
        GSP_CK(cudaEventRecord(p->ev[1], s));
    }
    gsp_status st = run_search(p, d_D, n_out, stride, t_offset, nullptr, nullptr, s);
    if (st != GSP_OK) return st;
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[2], s));
    return GSP_OK;
}

gsp_status gsp_boxcar_snr(gsp_plan_t p, const int32_t *d_D, int64_t n_out, int64_t stride,
                          float *d_snr, void *stream) {
    if (!p || !d_D || !d_snr || n_out <= 0 || stride < n_out) return GSP_ERR_INVALID_ARG;
    if (n_out / p->desc.block_len > p->nb_max) return GSP_ERR_INVALID_ARG;
    p->launches = 0;
    return run_search(p, d_D, n_out, stride, 0, d_snr, nullptr, (cudaStream_t)stream);
}

gsp_status gsp_search_stats(gsp_plan_t p, double *sigma_b, uint8_t *bad, double *sigma_ref,
                            int64_t *nb_out) {
    if (!p) return GSP_ERR_INVALID_ARG;
    if (!p->have_search) return GSP_ERR_STATE;
    GSP_CK(cudaStreamSynchronize(p->last_stream));
    const int64_t nb = p->last_nb, ndm = p->desc.ndm;
    if (nb_out) *nb_out = nb;
    if (sigma_b && nb > 0)
        GSP_CK(cudaMemcpy2D(sigma_b, nb * sizeof(double), p->d_sigma_b, p->nb_max * sizeof(double),
                            nb * sizeof(double), ndm, cudaMemcpyDeviceToHost));
    if (bad && nb > 0)
        GSP_CK(cudaMemcpy2D(bad, nb, p->d_bad, p->nb_max, nb, ndm, cudaMemcpyDeviceToHost));
    if (sigma_ref)
        GSP_CK(cudaMemcpy(sigma_ref, p->d_sref, ndm * sizeof(double), cudaMemcpyDeviceToHost));
    return GSP_OK;
}

gsp_status gsp_candidates(gsp_plan_t p, gsp_cand *host_out, int64_t cap, int64_t *n_total) {
    if (!p || !n_total || cap < 0 || (cap > 0 && !host_out)) return GSP_ERR_INVALID_ARG;
    if (!p->have_search) return GSP_ERR_STATE;
    GSP_CK(cudaStreamSynchronize(p->last_stream));
    gsp_status kst = take_kernel_error(p);
    if (kst != GSP_OK) return kst;
    unsigned long long n = 0;
    GSP_CK(cudaMemcpy(&n, p->d_ncand, sizeof(n), cudaMemcpyDeviceToHost));
    *n_total = (int64_t)n;
    const int64_t kept = std::min<int64_t>((int64_t)n, p->desc.max_cands);
    auto less = [](const gsp_cand &a, const gsp_cand &b) {
        if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
        if (a.t != b.t) return a.t < b.t;
        return a.width < b.width;
    };
    const int64_t m = std::min<int64_t>(kept, cap);
    if (kept <= cap) {
        // everything fits: read straight into the caller's buffer (no staging copy)
        if (kept > 0)
            GSP_CK(cudaMemcpy(host_out, p->d_cands, (size_t)kept * sizeof(gsp_cand),
                              cudaMemcpyDeviceToHost));
        // the device list is already in (dm, t) order; sort only if it is not
        if (!std::is_sorted(host_out, host_out + kept, less)) std::sort(host_out, host_out + kept, less);
    } else {
        // the first cap of the sorted list: sort the whole kept list first
        std::vector<gsp_cand> v((size_t)kept);
        GSP_CK(cudaMemcpy(v.data(), p->d_cands, (size_t)kept * sizeof(gsp_cand),
                          cudaMemcpyDeviceToHost));
        if (!std::is_sorted(v.begin(), v.end(), less)) std::sort(v.begin(), v.end(), less);
        if (m > 0) std::memcpy(host_out, v.data(), (size_t)m * sizeof(gsp_cand));
    }
    return ((int64_t)n > m) ? GSP_ERR_CAPACITY : GSP_OK;
}

// Host input in time chunks: the copy of chunk k + 1 (on a second stream)
// overlaps the dedispersion of chunk k.  Chunk boundaries are multiples of
// lcm(block_len, 16) output samples, so every chunk's input starts 16-byte
// aligned and its block sums land in whole blocks; chunk k needs the input
// columns [a_k, a_{k+1} + max_delay), and its copy brings the columns not yet
// on the device.  The series are exact integer sums, so the result does not
// depend on the chunking.  GSP_HOST_CHUNKS (1..8) sets the number of chunks;
// 1 copies everything first.
constexpr int kHostChunks = 8;

int host_chunks() {
    if (const char *v = std::getenv("GSP_HOST_CHUNKS")) {
        const int k = std::atoi(v);
        if (k >= 1 && k <= kHostChunks) return k;
    }
    return kHostChunks;
}

gsp_status gsp_search_host(gsp_plan_t p, const uint8_t *h_x, int64_t n_in, int64_t x_stride,
                           int64_t t_offset, gsp_cand *host_out, int64_t cap, int64_t *n_total,
                           void *stream) {
    if (!p || !h_x || !n_total || n_in <= 0 || n_in > p->desc.nsamp_max || x_stride < n_in)
        return GSP_ERR_INVALID_ARG;
    const int64_t dstride = (n_in + 15) & ~(int64_t)15;
    const size_t need = (size_t)dstride * (size_t)p->desc.nchan;
    if (need > p->d_xstage_bytes) {
        cudaFree(p->d_xstage);
        p->d_xstage = nullptr;
        p->d_xstage_bytes = 0;
        const int64_t full_stride = (p->desc.nsamp_max + 15) & ~(int64_t)15;
        const size_t full = std::max(need, (size_t)full_stride * (size_t)p->desc.nchan);
        gsp_status st = dalloc(&p->d_xstage, full);
        if (st != GSP_OK) return st;
        p->d_xstage_bytes = full;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_out = n_in - p->max_delay;
    const int64_t B = p->desc.block_len;
    int64_t unit = B;
    while (unit % 16) unit += B;  // lcm(B, 16)
    const int nch = host_chunks();
    const bool pipelined = nch > 1 && !p->simple_dd && n_out >= nch * unit;
    if (!pipelined) {
        if (x_stride == dstride) {
            GSP_CK(cudaMemcpyAsync(p->d_xstage, h_x, need, cudaMemcpyHostToDevice, s));
        } else {
            GSP_CK(cudaMemcpy2DAsync(p->d_xstage, dstride, h_x, x_stride, n_in, p->desc.nchan,
                                     cudaMemcpyHostToDevice, s));
        }
        gsp_status st = gsp_search(p, p->d_xstage, n_in, dstride, t_offset, nullptr, 0, stream);
        if (st != GSP_OK) return st;
        return gsp_candidates(p, host_out, cap, n_total);
    }
    if (!p->h2d_stream) GSP_CK(cudaStreamCreateWithFlags(&p->h2d_stream, cudaStreamNonBlocking));
    for (auto &e : p->h2d_ev)
        if (!e) GSP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // chunk sizes in the weights 1, 1, 2, 4, 8, 8, ...: the first dedispersion
    // launch waits only for a small copy (its columns plus the max_delay
    // overhang), and each later copy is at most the size of the launch it hides
    // behind; equal chunks when the series is too short for the smallest ones
    int64_t wts[kHostChunks], wsum = 0;
    for (int k = 0; k < nch; k++) {
        wts[k] = k == 0 ? 1 : std::min<int64_t>((int64_t)1 << (k - 1), 8);
        wsum += wts[k];
    }
    const bool grow = n_out >= wsum * unit;
    int64_t a[kHostChunks + 1];
    a[0] = 0;
    for (int k = 0, cum = 0; k < nch; k++) {
        cum += (int)wts[k];
        a[k + 1] = (grow ? n_out * cum / wsum : n_out * (k + 1) / nch) / unit * unit;
    }
    a[nch] = n_out;
    // the copies start after the caller's earlier work on s (which may still
    // read the staging buffer)
    GSP_CK(cudaEventRecord(p->h2d_ev[kHostChunks], s));
    GSP_CK(cudaStreamWaitEvent(p->h2d_stream, p->h2d_ev[kHostChunks], 0));
    int64_t copied = 0;
    for (int k = 0; k < nch; k++) {
        const int64_t upto = std::min(n_in, a[k + 1] + p->max_delay);
        if (upto > copied)
            GSP_CK(cudaMemcpy2DAsync(p->d_xstage + copied, dstride, h_x + copied, x_stride,
                                     upto - copied, p->desc.nchan, cudaMemcpyHostToDevice,
                                     p->h2d_stream));
        copied = std::max(copied, upto);
        GSP_CK(cudaEventRecord(p->h2d_ev[k], p->h2d_stream));
    }
    gsp_status st = ensure_scratch_D(p, n_out);
    if (st != GSP_OK) return st;
    int32_t *D = p->d_D;
    const int64_t stride = (n_out + 3) & ~(int64_t)3;
    p->launches = 0;
    unsigned long long *bsum = nullptr;
    if (fused_stats(p) && n_out / B > 0) {
        bsum = p->d_bsum;
        GSP_CK(cudaMemsetAsync(bsum, 0, (size_t)p->desc.ndm * p->nb_max * 3 * sizeof(*bsum), s));
    }
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[0], s));
    for (int k = 0; k < nch; k++) {
        GSP_CK(cudaStreamWaitEvent(s, p->h2d_ev[k], 0));
        const int64_t len = a[k + 1] - a[k];
        st = run_dedisperse(p, p->d_xstage + a[k], len + p->max_delay, dstride, len, D + a[k],
                            stride, bsum ? bsum + (a[k] / B) * 3 : nullptr, s);
        if (st != GSP_OK) return st;
    }
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[1], s));
    st = run_search(p, D, n_out, stride, t_offset, nullptr, bsum, s);
    if (st != GSP_OK) return st;
    if (p->timed) GSP_CK(cudaEventRecord(p->ev[2], s));
    return gsp_candidates(p, host_out, cap, n_total);
}

gsp_status gsp_plan_timing(gsp_plan_t p, float *ms_dd, float *ms_search) {
    if (!p) return GSP_ERR_INVALID_ARG;
    if (!p->timed) return GSP_ERR_STATE;
    GSP_CK(cudaEventSynchronize(p->ev[2]));
    gsp_status kst = take_kernel_error(p);
    if (kst != GSP_OK) return kst;
    float a = 0.f, b = 0.f;
    GSP_CK(cudaEventElapsedTime(&a, p->ev[0], p->ev[1]));
    GSP_CK(cudaEventElapsedTime(&b, p->ev[1], p->ev[2]));
    if (ms_dd) *ms_dd = a;
    if (ms_search) *ms_search = b;
    return GSP_OK;
}

int32_t gsp_plan_launches(gsp_plan_t p) { return p ? p->launches : -1; }

gsp_status gsp_plan_set_wait_limit(gsp_plan_t p, int64_t cycles, int32_t starve) {
    if (!p || cycles < 1 || cycles > gsp::kWaitLimit || starve < 0 || starve > 1)
        return GSP_ERR_INVALID_ARG;
    p->wait_budget = cycles;
    p->wait_starve = starve;
    return GSP_OK;
}

gsp_status gsp_plan_set_snippet_path(gsp_plan_t p, int32_t path) {
    if (!p || path < 0 || path > 2) return GSP_ERR_INVALID_ARG;
    p->snippet_path = path;
    return GSP_OK;
}

gsp_status gsp_plan_series(gsp_plan_t p, const int32_t **d_D, int64_t *stride, int64_t *n_out) {
    if (!p || !d_D || !stride || !n_out) return GSP_ERR_INVALID_ARG;
    if (!p->have_search) return GSP_ERR_STATE;
    *d_D = p->last_D;
    *stride = p->last_stride;
    *n_out = p->last_nout;
    return GSP_OK;
}

// Tile-variant autotuning of one plan on the caller's input: every tiled
// variant that fits the plan is timed kPlanTuneReps times (after one warm-up
// run) over the first kPlanTuneSamples output samples, into the plan's series
// scratch; the one with the smallest median becomes the plan's variant.
constexpr int64_t kPlanTuneSamples = 131072;
constexpr int kPlanTuneReps = 3;

gsp_status gsp_plan_tune(gsp_plan_t p, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                         void *stream, int32_t *variant, float *best_ms) {
    int64_t n_out = 0;
    gsp_status st = check_dd_args(p, d_x, n_in, x_stride, nullptr, 0, &n_out);
    if (st != GSP_OK) return st;
    if (p->simple_dd) return GSP_ERR_STATE;
    st = ensure_scratch_D(p, n_out);
    if (st != GSP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = std::min(n_out, kPlanTuneSamples);
    const int64_t stride = (n_out + 3) & ~(int64_t)3;
    const int *cand = nullptr;
    const int ncand = gsp::dedisperse_tune_candidates(&cand);
    const int keep = p->geom.variant;
    int best = -1;
    float best_t = 0.f;
    for (int ci = 0; ci < ncand; ci++) {
        if (!gsp::dedisperse_variant_usable(p, cand[ci])) continue;
        gsp::dedisperse_set_variant(p, cand[ci]);
        std::vector<float> ms;
        for (int r = 0; r <= kPlanTuneReps; r++) {
            int32_t nl = 0;
            GSP_CK(cudaEventRecord(p->ev[0], s));
            cudaError_t e = gsp::launch_dedisperse_tiled(p, d_x, n + p->max_delay, x_stride, n,
                                                         p->d_D, stride, nullptr, s, &nl);
            if (e != cudaSuccess) {
                gsp::dedisperse_set_variant(p, keep);
                set_err(e, "tuning launch");
                return GSP_ERR_CUDA;
            }
            GSP_CK(cudaEventRecord(p->ev[1], s));
            GSP_CK(cudaEventSynchronize(p->ev[1]));
            float t = 0.f;
            GSP_CK(cudaEventElapsedTime(&t, p->ev[0], p->ev[1]));
            if (r > 0) ms.push_back(t);
        }
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (best < 0 || med < best_t) {
            best = cand[ci];
            best_t = med;
        }
    }
    gsp_status kst = take_kernel_error(p);
    gsp::dedisperse_set_variant(p, best >= 0 ? best : keep);
    if (kst != GSP_OK) return kst;
    if (variant) *variant = p->geom.variant;
    if (best_ms) *best_ms = best_t;
    return GSP_OK;
}

int32_t gsp_dedisperse_variants(gsp_plan_t p, int32_t *in_use) {
    if (p && in_use) *in_use = p->simple_dd ? -1 : p->geom.variant;
    return gsp::dedisperse_num_variants();
}

const char *gsp_status_string(gsp_status s) {
    switch (s) {
        case GSP_OK: return "ok";
        case GSP_ERR_INVALID_ARG: return "invalid argument";
        case GSP_ERR_OOM: return "out of memory";
        case GSP_ERR_CUDA: return "CUDA error";
        case GSP_ERR_TOO_SHORT: return "input shorter than the largest delay";
        case GSP_ERR_CAPACITY: return "candidate capacity exceeded (list truncated)";
        case GSP_ERR_TIMEOUT: return "bounded wait timed out";
        case GSP_ERR_TIE: return "delay table entry within 1e-9 of a rounding tie";
        case GSP_ERR_ALIGN: return "pointer or stride misaligned";
        case GSP_ERR_STATE: return "call out of order";
        case GSP_ERR_TOO_LARGE: return "sizes exceed the static scratch of the no-allocation search";
        case GSP_ERR_BUSY: return "no free chunk buffer (chunk not admitted)";
    }
    return "unknown status";
}

const char *gsp_last_error_string(void) { return g_err; }

int32_t gsp_version(void) { return 100; }

}  // extern "C"
