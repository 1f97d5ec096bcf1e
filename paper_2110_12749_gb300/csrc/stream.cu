// Streaming search of one beam: chunks of new samples arrive one after the
// other; every chunk is searched together with the last max_delay samples of
// the previous one (the dispersion-overlap tail, kept on the device), so that
// consecutive chunks cover the output series without gaps or overlaps.  This
// is the device-resident form of the overlapping read blocks of Alg. 2 /
// Alg. 3 (lastdata + data), and of the half-overlap merge of adjacent files
// in Sec. 2.1, for an unbounded stream.
//
// A stream either owns two input buffers (ping-pong: the tail is read from
// the previous chunk's buffer), or draws its input buffer chunk by chunk from
// a pool shared by the streams of many beams (gsp_chunkpool_*).  A pooled
// stream keeps only its tail on the device, and a chunk is admitted only when
// a pool buffer is free: the pool's size is the device memory the caller
// grants to chunks in flight, and a push that finds no free buffer is refused
// (GSP_ERR_BUSY) with nothing enqueued, so the caller can queue the chunk.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "gsp_internal.cuh"

struct gsp_chunkpool_s {
    int32_t nchan = 0;
    int64_t chunk_out = 0;
    int64_t max_tail = 0;
    int64_t stride = 0;                // bytes per channel row of a buffer (multiple of 16)
    std::vector<uint8_t *> buf;        // nbuf device buffers [nchan][stride]
    std::vector<cudaEvent_t> done;     // recorded after the last work that reads buffer i
    std::vector<char> busy;            // buffer i holds a chunk whose work may be running
};

struct gsp_stream_s {
    gsp_plan_t plan = nullptr;
    int64_t chunk_out = 0;   // output samples per chunk (multiple of block_len and window_len)
    int64_t tail = 0;        // max delay of the plan
    int64_t stride = 0;      // device row stride (bytes), multiple of 16
    uint8_t *buf[2] = {nullptr, nullptr};  // ping-pong [nchan][stride] inputs (own buffers)
    int cur = 0;             // buffer holding the last chunk
    gsp_chunkpool_s *pool = nullptr;       // pooled: input buffers come from here
    uint8_t *tailbuf = nullptr;            // pooled: [nchan][tail_stride] last tail samples
    int64_t tail_stride = 0;
    int64_t chunks = 0;      // chunks pushed
    int32_t beam = 0;
    cudaStream_t last = nullptr;
    int64_t last_offset = 0;  // absolute sample index of the last chunk's output sample 0
};

namespace {

bool check_chunking(gsp_plan_t plan, int64_t chunk_out) {
    return chunk_out > 0 && chunk_out % plan->desc.block_len == 0 &&
           chunk_out % plan->desc.window_len == 0;
}

// A pool buffer whose last chunk has finished (or that never held one), or -1.
int pool_acquire(gsp_chunkpool_s *p) {
    for (size_t i = 0; i < p->buf.size(); i++) {
        if (p->busy[i]) {
            const cudaError_t e = cudaEventQuery(p->done[i]);
            if (e == cudaErrorNotReady) continue;
            (void)cudaGetLastError();
            p->busy[i] = 0;
        }
        return (int)i;
    }
    return -1;
}

}  // namespace

extern "C" {

int64_t gsp_chunkpool_bytes(int32_t nchan, int64_t chunk_out, int64_t max_tail, int32_t nbuf) {
    if (nchan <= 0 || chunk_out <= 0 || max_tail < 0 || nbuf <= 0) return -1;
    return (int64_t)nbuf * (int64_t)nchan * ((chunk_out + max_tail + 15) & ~(int64_t)15);
}

gsp_status gsp_chunkpool_create(gsp_chunkpool_t *out, int32_t nchan, int64_t chunk_out,
                                int64_t max_tail, int32_t nbuf) {
    if (!out || nchan <= 0 || chunk_out <= 0 || max_tail < 0 || nbuf <= 0 || nbuf > 1024)
        return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    gsp_chunkpool_s *p = new (std::nothrow) gsp_chunkpool_s();
    if (!p) return GSP_ERR_OOM;
    p->nchan = nchan;
    p->chunk_out = chunk_out;
    p->max_tail = max_tail;
    p->stride = (chunk_out + max_tail + 15) & ~(int64_t)15;
    p->buf.assign((size_t)nbuf, nullptr);
    p->done.assign((size_t)nbuf, nullptr);
    p->busy.assign((size_t)nbuf, 0);
    gsp_status st = GSP_OK;
    for (int i = 0; i < nbuf && st == GSP_OK; i++) {
        if (cudaMalloc((void **)&p->buf[i], (size_t)p->stride * (size_t)nchan) != cudaSuccess)
            st = GSP_ERR_OOM;
        else if (cudaEventCreateWithFlags(&p->done[i], cudaEventDisableTiming) != cudaSuccess)
            st = GSP_ERR_CUDA;
    }
    if (st != GSP_OK) {
        (void)cudaGetLastError();
        for (int i = 0; i < nbuf; i++) {
            cudaFree(p->buf[i]);
            if (p->done[i]) cudaEventDestroy(p->done[i]);
        }
        delete p;
        return st;
    }
    *out = p;
    return GSP_OK;
}

gsp_status gsp_chunkpool_destroy(gsp_chunkpool_t p) {
    if (!p) return GSP_ERR_INVALID_ARG;
    const cudaError_t e = cudaDeviceSynchronize();
    for (size_t i = 0; i < p->buf.size(); i++) {
        cudaFree(p->buf[i]);
        cudaEventDestroy(p->done[i]);
    }
    delete p;
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}

int32_t gsp_chunkpool_free(gsp_chunkpool_t p) {
    if (!p) return -1;
    int32_t n = 0;
    for (size_t i = 0; i < p->buf.size(); i++) {
        if (p->busy[i]) {
            const cudaError_t e = cudaEventQuery(p->done[i]);
            if (e == cudaErrorNotReady) continue;
            (void)cudaGetLastError();
            p->busy[i] = 0;
        }
        n++;
    }
    return n;
}

gsp_status gsp_stream_create(gsp_stream_t *out, gsp_plan_t plan, int64_t chunk_out, int32_t beam) {
    if (!out || !plan || chunk_out <= 0) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    const int64_t tail = gsp_plan_max_delay(plan);
    const int64_t n_in = chunk_out + tail;
    if (n_in > plan->desc.nsamp_max) return GSP_ERR_INVALID_ARG;
    if (!check_chunking(plan, chunk_out)) return GSP_ERR_INVALID_ARG;
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

gsp_status gsp_stream_create_pooled(gsp_stream_t *out, gsp_plan_t plan, gsp_chunkpool_t pool,
                                    int32_t beam) {
    if (!out || !plan || !pool) return GSP_ERR_INVALID_ARG;
    *out = nullptr;
    const int64_t tail = gsp_plan_max_delay(plan);
    const int64_t chunk_out = pool->chunk_out;
    if (plan->desc.nchan != pool->nchan || tail > pool->max_tail ||
        chunk_out + tail > plan->desc.nsamp_max || !check_chunking(plan, chunk_out))
        return GSP_ERR_INVALID_ARG;
    gsp_stream_s *s = new (std::nothrow) gsp_stream_s();
    if (!s) return GSP_ERR_OOM;
    s->plan = plan;
    s->chunk_out = chunk_out;
    s->tail = tail;
    s->stride = pool->stride;
    s->pool = pool;
    s->beam = beam;
    s->tail_stride = std::max<int64_t>((tail + 15) & ~(int64_t)15, 16);
    if (cudaMalloc((void **)&s->tailbuf, (size_t)s->tail_stride * (size_t)plan->desc.nchan) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return GSP_ERR_OOM;
    }
    *out = s;
    return GSP_OK;
}

gsp_status gsp_stream_destroy(gsp_stream_t s) {
    if (!s) return GSP_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(s->buf[0]);
    cudaFree(s->buf[1]);
    cudaFree(s->tailbuf);
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

int64_t gsp_stream_pooled_bytes(gsp_plan_t plan, int64_t chunk_out) {
    if (!plan || chunk_out <= 0) return -1;
    const int64_t tail = gsp_plan_max_delay(plan);
    int64_t bytes = std::max<int64_t>((tail + 15) & ~(int64_t)15, 16) * (int64_t)plan->desc.nchan;
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
    int slot = -1;
    uint8_t *dst = nullptr;
    const uint8_t *prev_tail = nullptr;
    int64_t prev_stride = 0;
    if (s->pool) {
        slot = pool_acquire(s->pool);
        if (slot < 0) return GSP_ERR_BUSY;  // not admitted: nothing enqueued
        dst = s->pool->buf[slot];
        prev_tail = s->tailbuf;
        prev_stride = s->tail_stride;
    } else {
        const int nxt = s->chunks == 0 ? 0 : 1 - s->cur;
        dst = s->buf[nxt];
        prev_tail = s->buf[s->cur] + s->chunk_out;
        prev_stride = s->stride;
    }
    cudaError_t e = cudaSuccess;
    if (s->chunks == 0) {
        e = cudaMemcpy2DAsync(dst, s->stride, h_x, h_stride, n, C, cudaMemcpyHostToDevice, cs);
    } else {
        // overlap tail: the last `tail` input samples of the previous chunk
        if (s->tail > 0)
            e = cudaMemcpy2DAsync(dst, s->stride, prev_tail, prev_stride, s->tail, C,
                                  cudaMemcpyDeviceToDevice, cs);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dst + s->tail, s->stride, h_x, h_stride, n, C,
                                  cudaMemcpyHostToDevice, cs);
    }
    // pooled: keep this chunk's tail for the next one before the buffer goes back
    if (e == cudaSuccess && s->pool && s->tail > 0)
        e = cudaMemcpy2DAsync(s->tailbuf, s->tail_stride, dst + s->chunk_out, s->stride, s->tail,
                              C, cudaMemcpyDeviceToDevice, cs);
    if (e != cudaSuccess) {
        gsp::record_error(e, "stream chunk copy");
        return GSP_ERR_CUDA;
    }
    const int64_t offset = s->chunks * s->chunk_out;
    gsp_status st = gsp_search(s->plan, dst, s->chunk_out + s->tail, s->stride, offset, nullptr,
                               0, stream);
    if (s->pool) {
        // the buffer is free again once everything enqueued above has run
        if (cudaEventRecord(s->pool->done[slot], cs) != cudaSuccess) {
            (void)cudaGetLastError();
            if (st == GSP_OK) st = GSP_ERR_CUDA;
            // without the event the buffer cannot be tracked: wait for the stream instead
            cudaStreamSynchronize(cs);
        } else {
            s->pool->busy[slot] = 1;
        }
    }
    if (st != GSP_OK) return st;
    if (!s->pool) s->cur = s->chunks == 0 ? 0 : 1 - s->cur;
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
