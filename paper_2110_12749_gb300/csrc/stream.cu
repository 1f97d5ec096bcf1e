// Streaming search of one beam: chunks of new samples arrive one after the
// other; every chunk is searched together with the last max_delay samples of
// the previous one (the dispersion-overlap tail, kept on the device), so that
// consecutive chunks cover the output series without gaps or overlaps.  This
// is the device-resident form of the overlapping read blocks of Alg. 2 /
// Alg. 3 (lastdata + data), and of the half-overlap merge of adjacent files
// in Sec. 2.1, for an unbounded stream.
#include <algorithm>
#include <cstring>
#include <new>

#include "gsp_internal.cuh"

struct gsp_stream_s {
    gsp_plan_t plan = nullptr;
    int64_t chunk_out = 0;   // output samples per chunk (multiple of block_len and window_len)
    int64_t tail = 0;        // max delay of the plan
    int64_t stride = 0;      // device row stride (bytes), multiple of 16
    uint8_t *buf[2] = {nullptr, nullptr};  // ping-pong [nchan][stride] inputs
    int cur = 0;             // buffer holding the last chunk
    int64_t chunks = 0;      // chunks pushed
    int32_t beam = 0;
    cudaStream_t last = nullptr;
    int64_t last_offset = 0;  // absolute sample index of the last chunk's output sample 0
};

extern "C" {

gsp_status gsp_stream_create(gsp_stream_t *out, gsp_plan_t plan, int64_t chunk_out, int32_t beam) {
    if (!out || !plan || chunk_out <= 0) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    const int64_t tail = gsp_plan_max_delay(plan);
    const int64_t n_in = chunk_out + tail;
    if (n_in > plan->desc.nsamp_max) return GSP_ERR_INVALID_ARG;
    if (chunk_out % plan->desc.block_len || chunk_out % plan->desc.window_len)
        return GSP_ERR_INVALID_ARG;
    gsp_stream_s *s = new (std::nothrow) gsp_stream_s();
    if (!s) return GSP_ERR_OOM;
    s->plan = plan;
    s->chunk_out = chunk_out;
    s->tail = tail;
    s->stride = (n_in + 15) & ~(int64_t)15;
    s->beam = beam;
    const size_t bytes = (size_t)s->stride * (size_t)plan->desc.nchan;
    for (int i = 0; i < 2; i++) {
        if (cudaMalloc((void **)&s->buf[i], bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(s->buf[0]);
            delete s;
            return GSP_ERR_OOM;
        }
    }
    *out = s;
    return GSP_OK;
}

gsp_status gsp_stream_destroy(gsp_stream_t s) {
    if (!s) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(s->buf[0]);
    cudaFree(s->buf[1]);
    delete s;
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

int64_t gsp_stream_bytes(gsp_plan_t plan, int64_t chunk_out) {
    if (!plan || chunk_out <= 0) return -1;
    const int64_t stride = (chunk_out + gsp_plan_max_delay(plan) + 15) & ~(int64_t)15;
    int64_t bytes = 2 * stride * (int64_t)plan->desc.nchan;
    // the plan's series scratch, allocated on its first search for nsamp_max samples
    if (!plan->d_D) {
        const int64_t row = (std::max<int64_t>(plan->desc.nsamp_max - plan->max_delay, chunk_out) + 3) &
                            ~(int64_t)3;
        bytes += (int64_t)plan->desc.ndm * row * (int64_t)sizeof(int32_t);
    }
    return bytes;
}

int64_t gsp_stream_need(gsp_stream_t s) {
    if (!s) return -1;
    return s->chunks == 0 ? s->chunk_out + s->tail : s->chunk_out;
}

gsp_status gsp_stream_push(gsp_stream_t s, const uint8_t *h_x, int64_t n, int64_t h_stride,
                           void *stream) {
    if (!s || !h_x || h_stride < n || n != gsp_stream_need(s)) return GSP_ERR_INVALID_ARG;
    cudaStream_t cs = (cudaStream_t)stream;
    const int64_t C = s->plan->desc.nchan;
    const int nxt = s->chunks == 0 ? 0 : 1 - s->cur;
    uint8_t *dst = s->buf[nxt];
    cudaError_t e = cudaSuccess;
    if (s->chunks == 0) {
        e = cudaMemcpy2DAsync(dst, s->stride, h_x, h_stride, n, C, cudaMemcpyHostToDevice, cs);
    } else {
        // overlap tail: the last `tail` input samples of the previous chunk
        const uint8_t *prev = s->buf[s->cur];
        if (s->tail > 0)
            e = cudaMemcpy2DAsync(dst, s->stride, prev + s->chunk_out, s->stride, s->tail, C,
                                  cudaMemcpyDeviceToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dst + s->tail, s->stride, h_x, h_stride, n, C,
                                  cudaMemcpyHostToDevice, cs);
    }
    if (e != cudaSuccess) return GSP_ERR_CUDA;
    const int64_t offset = s->chunks * s->chunk_out;
    gsp_status st = gsp_search(s->plan, dst, s->chunk_out + s->tail, s->stride, offset, nullptr,
                               0, stream);
    if (st != GSP_OK) return st;
    s->cur = nxt;
    s->chunks++;
    s->last = cs;
    s->last_offset = offset;
    return GSP_OK;
}

gsp_status gsp_stream_results(gsp_stream_t s, gsp_cand *host_out, int64_t cap, int64_t *n_total,
                              int64_t *t_abs0) {
    if (!s || !n_total) return GSP_ERR_INVALID_ARG;
    if (s->chunks == 0) return GSP_ERR_STATE;
    gsp_status st = gsp_candidates(s->plan, host_out, cap, n_total);
    if (st != GSP_OK && st != GSP_ERR_CAPACITY) return st;
    const int64_t m = *n_total < cap ? *n_total : cap;
    for (int64_t i = 0; i < m; i++) {
        host_out[i].t += s->last_offset;
        host_out[i].beam = s->beam;
    }
    if (t_abs0) *t_abs0 = s->last_offset;
    return st;
}

}  // extern "C"
