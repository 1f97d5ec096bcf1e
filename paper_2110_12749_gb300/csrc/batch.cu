// Batched search of many beams (the multi-beam receiver of the survey in
// Sec. 2): every beam has its own plan (DM grid, length), all beams share the
// channel count, and their dedispersion runs as ONE launch of the tiled kernel
// whose CTAs work through a list of (beam, time tile, DM block) items.  With
// GSP_BATCH_PERSISTENT the grid is one CTA per SM striding over the items; with
// GSP_BATCH_GRAPH the whole enqueue sequence (block-sum resets, the batched
// dedispersion, every beam's search kernels) is captured once into a CUDA
// graph and replayed while the inputs stay the same; with GSP_BATCH_AUTOTUNE
// the first call times the dedispersion kernel's tile variants that fit the
// batch (channels per stage, DM trials per block, samples per tile, visiting
// order) on the actual inputs, each three times on every beam's first
// kTuneSamples output samples, and keeps the one with the smallest median.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gsp_internal.cuh"

struct gsp_batch_s {
    std::vector<gsp_plan_t> plans;
    int32_t flags = 0;
    int variant = -1;
    float tuned_ms = 0.f;   // median time of the fastest tuning run (ms)
    int32_t tune_tried = 0;  // variants the autotuner timed
    std::vector<int32_t> tune_variant;  // every timed candidate and its median (ms)
    std::vector<float> tune_ms;
    std::vector<gsp_beam_input> last;  // inputs the graph was captured for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
    bool have_search = false;
    int32_t launches = 0;
    int32_t graph_launches = 0;  // kernels in the captured graph
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // GSP_BATCH_TIMING
};

namespace {

constexpr int64_t kTuneSamples = 65536;  // output samples per beam of a tuning run
constexpr int kTuneReps = 3;             // timed runs per candidate (median kept)

bool same_inputs(const std::vector<gsp_beam_input> &a, const gsp_beam_input *b, size_t n) {
    if (a.size() != n) return false;
    for (size_t i = 0; i < n; i++)
        if (std::memcmp(&a[i], &b[i], sizeof(gsp_beam_input)) != 0) return false;
    return true;
}

void drop_graph(gsp_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Enqueue the whole batch on stream s with dedispersion variant `variant`.
gsp_status enqueue(gsp_batch_s *b, const gsp_beam_input *in, int variant, cudaStream_t s,
                   int32_t *nlaunch) {
    const int nb = (int)b->plans.size();
    std::vector<gsp::BeamLaunch> bl((size_t)nb);
    std::vector<int64_t> n_out((size_t)nb);
    for (int i = 0; i < nb; i++) {
        gsp_plan_s *p = b->plans[i];
        int32_t *D = nullptr;
        int64_t stride = 0;
        unsigned long long *bsum = nullptr;
        gsp_status st = gsp::plan_check_input(p, in[i].d_x, in[i].n_in, in[i].x_stride, &n_out[i]);
        if (st == GSP_OK) st = gsp::plan_prepare_search(p, n_out[i], &D, &stride, &bsum);
        if (st != GSP_OK) return st;
        if (bsum && cudaMemsetAsync(bsum, 0, (size_t)p->desc.ndm * p->nb_max * 3 * sizeof(*bsum), s) !=
                        cudaSuccess)
            return GSP_ERR_CUDA;
        if (cudaMemsetAsync(p->d_ncand, 0, sizeof(unsigned long long), s) != cudaSuccess)
            return GSP_ERR_CUDA;
        bl[i] = gsp::BeamLaunch{p, in[i].d_x, in[i].n_in, in[i].x_stride, n_out[i], D, stride, bsum};
    }
    gsp_plan_s *p0 = b->plans[0];
    const bool timed = (b->flags & GSP_BATCH_TIMING) && b->ev[0];
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return GSP_ERR_CUDA;
    const bool capturing = cst == cudaStreamCaptureStatusActive;
    if (timed && cudaEventRecordWithFlags(b->ev[0], s, capturing ? cudaEventRecordExternal : 0) !=
                     cudaSuccess)
        return GSP_ERR_CUDA;
    if (gsp::launch_dedisperse_batch(bl.data(), nb, variant, (b->flags & GSP_BATCH_PERSISTENT) != 0,
                                     p0->num_sms, p0->d_err, s, nlaunch) != cudaSuccess)
        return GSP_ERR_CUDA;
    if (timed && cudaEventRecordWithFlags(b->ev[1], s, capturing ? cudaEventRecordExternal : 0) !=
                     cudaSuccess)
        return GSP_ERR_CUDA;
    for (int i = 0; i < nb; i++) {
        gsp_plan_s *p = b->plans[i];
        if (gsp::launch_search(p, bl[i].out, n_out[i], bl[i].out_stride, in[i].t_offset, nullptr,
                               bl[i].bsum, s, nlaunch) != cudaSuccess)
            return GSP_ERR_CUDA;
        p->last_stream = s;
        p->last_D = bl[i].out;
        p->last_stride = bl[i].out_stride;
        p->last_nout = n_out[i];
        p->last_nb = n_out[i] / p->desc.block_len;
        p->have_search = true;
    }
    if (timed && cudaEventRecordWithFlags(b->ev[2], s, capturing ? cudaEventRecordExternal : 0) !=
                     cudaSuccess)
        return GSP_ERR_CUDA;
    return GSP_OK;
}

// Median device time (ms) of kTuneReps batched dedispersion launches of
// variant v over every beam's first kTuneSamples output samples (series into
// the plans' scratch, no block sums); < 0 if the variant cannot run.
float time_variant(gsp_batch_s *b, const gsp_beam_input *in, int v, cudaStream_t s,
                   cudaEvent_t e0, cudaEvent_t e1) {
    const int nb = (int)b->plans.size();
    std::vector<gsp::BeamLaunch> bl((size_t)nb);
    for (int i = 0; i < nb; i++) {
        gsp_plan_s *p = b->plans[i];
        if (!gsp::dedisperse_variant_usable(p, v)) return -1.f;
        int64_t n_out = 0, stride = 0;
        int32_t *D = nullptr;
        unsigned long long *bsum = nullptr;
        if (gsp::plan_check_input(p, in[i].d_x, in[i].n_in, in[i].x_stride, &n_out) != GSP_OK ||
            gsp::plan_prepare_search(p, n_out, &D, &stride, &bsum) != GSP_OK)
            return -1.f;
        const int64_t n = std::min<int64_t>(n_out, kTuneSamples);
        bl[i] = gsp::BeamLaunch{p, in[i].d_x, n + p->max_delay, in[i].x_stride, n, D, stride,
                                nullptr};
    }
    gsp_plan_s *p0 = b->plans[0];
    std::vector<float> ms;
    for (int r = 0; r <= kTuneReps; r++) {  // run 0 warms up and sets the kernel's attributes
        int32_t nl = 0;
        if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
        if (gsp::launch_dedisperse_batch(bl.data(), nb, v, (b->flags & GSP_BATCH_PERSISTENT) != 0,
                                         p0->num_sms, p0->d_err, s, &nl) != cudaSuccess) {
            (void)cudaGetLastError();
            return -1.f;
        }
        float t = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return -1.f;
        if (r > 0) ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

}  // namespace

extern "C" {

gsp_status gsp_batch_create(gsp_batch_t *out, const gsp_plan_t *plans, int32_t nbeams,
                            int32_t flags) {
    if (!out || !plans || nbeams < 1 || nbeams > 32) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < nbeams; i++) {
        if (!plans[i] || plans[i]->simple_dd || plans[i]->desc.nchan != plans[0]->desc.nchan)
            return GSP_ERR_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) return GSP_ERR_INVALID_ARG;  // one plan per beam
    }
    // one tile variant for all beams: the beams' own if it fits every beam's
    // delay spread, else the first automatic choice that does
    const int variant = gsp::dedisperse_choose_variant(plans, nbeams);
    if (variant < 0) return GSP_ERR_INVALID_ARG;
    gsp_batch_s *b = new (std::nothrow) gsp_batch_s();
    if (!b) return GSP_ERR_OOM;
    b->plans.assign(plans, plans + nbeams);
    b->flags = flags;
    b->variant = variant;
    if (flags & GSP_BATCH_TIMING)
        for (auto &e : b->ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                delete b;
                return GSP_ERR_CUDA;
            }
    *out = b;
    return GSP_OK;
}

gsp_status gsp_batch_destroy(gsp_batch_t b) {
    if (!b) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    drop_graph(b);
    for (auto &ev : b->ev)
        if (ev) cudaEventDestroy(ev);
    delete b;
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

gsp_status gsp_batch_search(gsp_batch_t b, const gsp_beam_input *in, void *stream) {
    if (!b || !in) return GSP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if ((b->flags & GSP_BATCH_GRAPH) && s == nullptr) return GSP_ERR_INVALID_ARG;  // needs a capturable stream
    const size_t nb = b->plans.size();
    b->launches = 0;
    if ((b->flags & GSP_BATCH_AUTOTUNE) && b->tuned_ms == 0.f) {
        // time every candidate variant that fits this batch; keep the fastest median
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            if (e0) cudaEventDestroy(e0);
            return GSP_ERR_CUDA;
        }
        int best = -1;
        float best_ms = 0.f;
        const int *cand = nullptr;
        const int ncand = gsp::dedisperse_tune_candidates(&cand);
        b->tune_tried = 0;
        b->tune_variant.clear();
        b->tune_ms.clear();
        for (int ci = 0; ci < ncand; ci++) {
            const float ms = time_variant(b, in, cand[ci], s, e0, e1);
            if (ms < 0.f) continue;
            b->tune_tried++;
            b->tune_variant.push_back(cand[ci]);
            b->tune_ms.push_back(ms);
            if (best < 0 || ms < best_ms) {
                best = cand[ci];
                best_ms = ms;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (best < 0) return GSP_ERR_CUDA;
        b->variant = best;
        b->tuned_ms = best_ms;
        drop_graph(b);
    }
    if (b->flags & GSP_BATCH_GRAPH) {
        if (!b->exec || !same_inputs(b->last, in, nb)) {
            drop_graph(b);
            // one uncaptured run configures kernel attributes and allocates scratch
            int32_t nl = 0;
            gsp_status st = enqueue(b, in, b->variant, s, &nl);
            if (st != GSP_OK) return st;
            if (cudaStreamSynchronize(s) != cudaSuccess) return GSP_ERR_CUDA;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                return GSP_ERR_CUDA;
            st = enqueue(b, in, b->variant, s, &b->launches);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != GSP_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return st != GSP_OK ? st : GSP_ERR_CUDA;
            }
            b->graph = g;
            if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
                drop_graph(b);
                return GSP_ERR_CUDA;
            }
            b->last.assign(in, in + nb);
            b->graph_launches = b->launches;
        }
        if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return GSP_ERR_CUDA;
        b->launches = b->graph_launches;
    } else {
        gsp_status st = enqueue(b, in, b->variant, s, &b->launches);
        if (st != GSP_OK) return st;
    }
    b->last_stream = s;
    b->have_search = true;
    for (gsp_plan_s *p : b->plans) p->search_seq++;  // also on graph replays
    return GSP_OK;
}

gsp_status gsp_batch_candidates(gsp_batch_t b, gsp_cand *host_out, int64_t cap, int64_t *n_total) {
    if (!b || !n_total || cap < 0 || (cap > 0 && !host_out)) return GSP_ERR_INVALID_ARG;
    if (!b->have_search) return GSP_ERR_STATE;
    int64_t total = 0, stored = 0;
    gsp_status worst = GSP_OK;
    for (size_t i = 0; i < b->plans.size(); i++) {
        int64_t n = 0;
        gsp_status st = gsp_candidates(b->plans[i], host_out ? host_out + stored : nullptr,
                                       cap - stored, &n);
        if (st != GSP_OK && st != GSP_ERR_CAPACITY) return st;
        if (st == GSP_ERR_CAPACITY) worst = GSP_ERR_CAPACITY;
        const int64_t m = std::min<int64_t>(n, cap - stored);
        for (int64_t k = 0; k < m; k++) host_out[stored + k].beam = (int32_t)i;
        stored += m;
        total += n;
    }
    *n_total = total;
    return worst;
}

gsp_status gsp_batch_timing(gsp_batch_t b, float *ms_dedisperse, float *ms_total) {
    if (!b) return GSP_ERR_INVALID_ARG;
    if (!(b->flags & GSP_BATCH_TIMING) || !b->have_search) return GSP_ERR_STATE;
    if (cudaEventSynchronize(b->ev[2]) != cudaSuccess) return GSP_ERR_CUDA;
    float a = 0.f, t = 0.f;
    if (cudaEventElapsedTime(&a, b->ev[0], b->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, b->ev[0], b->ev[2]) != cudaSuccess)
        return GSP_ERR_CUDA;
    if (ms_dedisperse) *ms_dedisperse = a;
    if (ms_total) *ms_total = t;
    return GSP_OK;
}

int32_t gsp_batch_tune_results(gsp_batch_t b, int32_t *variants, float *ms, int32_t cap) {
    if (!b || cap < 0) return -1;
    const int32_t n = (int32_t)b->tune_variant.size();
    for (int32_t i = 0; i < std::min(n, cap); i++) {
        if (variants) variants[i] = b->tune_variant[i];
        if (ms) ms[i] = b->tune_ms[i];
    }
    return n;
}

gsp_status gsp_batch_info(gsp_batch_t b, int32_t *variant, float *tuned_ms, int32_t *launches) {
    if (!b) return GSP_ERR_INVALID_ARG;
    if (variant) *variant = b->variant;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    if (launches) *launches = b->launches;
    return GSP_OK;
}

}  // extern "C"
