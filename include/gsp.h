/*
 * gsp.h - C ABI of libgsp: brute-force incoherent dedispersion of an 8-bit
 * filterbank fused with a single-pulse (boxcar matched-filter) search, on one
 * GB300 (sm_103a).
 *
 * Method: arXiv 2110.12749 ("GSP").  Dedispersion is the sum over channels of
 * time-shifted samples with the shifts taken from a numdm x numchan delay
 * matrix (Sec. 2.3, Alg. 2 and Alg. 3); the single-pulse search that follows
 * it is named in Sec. 2.1-2.2 and specified here by the library (block
 * detrend, robust normalisation, boxcar filter, threshold, per-window
 * maximum).
 *
 * Conventions shared by every entry point
 *   - Input filterbank X: uint8, channel-major, X[c][t] at byte
 *     c * x_stride + t, c in [0, nchan), t in [0, n_in).  The merged buffer of
 *     Alg. 3 generalises to: every DM row uses the same output length
 *     n_out = n_in - max_delay, so that t + delay < n_in for every output.
 *   - Channel c (ascending order) has centre f_lo + (c + 1/2)(f_hi - f_lo)/nchan
 *     MHz; with freq_descending row 0 is the highest channel.  The top channel
 *     (highest centre) has delay 0 and all delays are >= 0.
 *   - Delay of (dm, c) in samples: floor(x + 1/2) with
 *     x = 4.148808e3 * DM * (1/f_c^2 - 1/f_top^2) / t_samp (f in MHz, t_samp in s),
 *     computed on the host in IEEE FP64 without contraction.
 *   - Dedispersed series D: int32 [ndm][n_out], exact integer sums.
 *   - Device pointers are CUDA device (or managed) addresses owned by the
 *     caller; host pointers are ordinary host memory owned by the caller.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it; only the
 *     functions documented as synchronising wait for the GPU.
 *   - Every function returns a gsp_status; nothing aborts, traps or prints.
 *     A CUDA failure returns GSP_ERR_CUDA and its text is available from
 *     gsp_last_error_string() in the calling thread.
 *   - A plan may be used by one host thread and one stream at a time.
 */
#ifndef GSP_H
#define GSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSP_OK = 0,
    GSP_ERR_INVALID_ARG = 1, /* bad pointer, size, stride or descriptor field */
    GSP_ERR_OOM = 2,         /* device or host allocation failed */
    GSP_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    GSP_ERR_TOO_SHORT = 4,   /* n_in <= max delay: no output sample exists */
    GSP_ERR_CAPACITY = 5,    /* more candidates than storage: list truncated */
    GSP_ERR_TIMEOUT = 6,     /* a bounded wait gave up */
    GSP_ERR_TIE = 7,         /* a delay lies within 1e-9 of a rounding tie */
    GSP_ERR_ALIGN = 8,       /* pointer or stride violates a stated alignment */
    GSP_ERR_STATE = 9,       /* call out of order (e.g. no search yet) */
    GSP_ERR_TOO_LARGE = 10,  /* sizes exceed the static scratch of gsp_search_series_static */
    GSP_ERR_BUSY = 11        /* no free chunk buffer: the chunk was not admitted, nothing enqueued */
} gsp_status;

/* Plan flags (gsp_plan_desc.flags). */
#define GSP_FLAG_TIMING 1    /* record CUDA events around each kernel phase */
#define GSP_FLAG_SIMPLE_DD 2 /* use the simple reference dedispersion kernel */

typedef struct gsp_plan_s *gsp_plan_t;
typedef struct gsp_stream_s *gsp_stream_t;
typedef struct gsp_chunkpool_s *gsp_chunkpool_t;
typedef struct gsp_batch_s *gsp_batch_t;
typedef struct gsp_subband_s *gsp_subband_t;
typedef struct gsp_ddplan_s *gsp_ddplan_t;
typedef struct gsp_ranker_s *gsp_ranker_t;

/* Batch flags (gsp_batch_create). */
#define GSP_BATCH_PERSISTENT 1 /* one CTA per SM striding over all beams' work items */
#define GSP_BATCH_GRAPH 2      /* capture the batch into a CUDA graph, replay while inputs repeat */
#define GSP_BATCH_AUTOTUNE 4   /* time the tile variants on the first call, keep the fastest */
#define GSP_BATCH_TIMING 8     /* record CUDA events around the batched dedispersion */

/* Input of one beam of a batch (device filterbank, layout as gsp_dedisperse). */
typedef struct {
    const uint8_t *d_x;
    int64_t n_in;
    int64_t x_stride;
    int64_t t_offset;
} gsp_beam_input;

/* Plan descriptor: host values, copied by gsp_plan_create.  Fill it with
 * gsp_plan_desc_init() first; then set the band, sampling and DM grid. */
typedef struct {
    int32_t nchan;           /* channels C >= 1 */
    double f_lo_mhz;         /* bottom edge of the band */
    double f_hi_mhz;         /* top edge of the band (> f_lo_mhz > 0) */
    int32_t freq_descending; /* 0: row 0 = lowest channel; 1: row 0 = highest */
    double t_samp_s;         /* sampling time (s) */
    int32_t ndm;             /* number of DM trials >= 1 */
    const double *dms;       /* [ndm] DM values (pc cm^-3), or NULL for dm_lo + i*dm_step */
    double dm_lo, dm_step;
    const int32_t *delays;   /* optional explicit delay table [ndm][nchan] (>= 0);
                                overrides the band/DM description (Sec. 2.3 matrix) */
    int64_t nsamp_max;       /* largest n_in any call will pass (sizes scratch) */
    const int32_t *widths;   /* boxcar widths, ascending, 1..min(block_len, 1024); NULL = default 13 */
    int32_t nwidths;
    int32_t block_len;       /* detrend block B (default 1024, >= max width) */
    int32_t window_len;      /* candidate window L_win (default 1024) */
    float threshold;         /* event if S/N >= threshold (default 6) */
    float bad_lo, bad_hi;    /* block bad if sigma_b outside [bad_lo, bad_hi]*sigma_ref
                                (default 0.5, 2.5) */
    int64_t max_cands;       /* device candidate capacity (default 1<<20) */
    int32_t flags;           /* GSP_FLAG_* */
} gsp_plan_desc;

/* One single-pulse candidate: the best (t, width) of one DM row inside one
 * candidate window (fields after the per-candidate record of Sec. 2.2). */
typedef struct {
    int32_t dm_idx; /* DM trial index */
    int32_t width;  /* boxcar width (samples) */
    int64_t t;      /* start sample of the boxcar, relative to D[.][0] */
    float snr;      /* matched-filter S/N */
    int32_t beam;   /* beam label (0 for single-beam calls) */
} gsp_cand;

/* Fill *desc with defaults (13 widths {1,2,3,4,6,9,14,20,30,45,70,100,150},
 * B = L_win = 1024, threshold 6, bad bounds 0.5/2.5, max_cands 2^20) and
 * zeros elsewhere.  Host only. */
gsp_status gsp_plan_desc_init(gsp_plan_desc *desc);

/* Compute the delay table [ndm][nchan] of a descriptor on the host, exactly
 * as gsp_plan_create does (Sec. 2.3 delay matrix).  min_margin (optional)
 * receives min |frac(x) - 1/2| over the table.  No GPU is touched. */
gsp_status gsp_compute_delays(const gsp_plan_desc *desc, int32_t *host_out,
                              double *min_margin);

/* Create a plan: validate the descriptor, compute the delay table (returns
 * GSP_ERR_TIE if any entry is within 1e-9 of a rounding tie), choose tiles,
 * and allocate device memory for the delay table, search statistics and the
 * candidate buffer.  The dedispersed-series scratch used by gsp_search when
 * the caller passes no output buffer is allocated on first use.  Uses the
 * current CUDA device. */
gsp_status gsp_plan_create(gsp_plan_t *out, const gsp_plan_desc *desc);

/* Free everything the plan owns (synchronises the device first). */
gsp_status gsp_plan_destroy(gsp_plan_t plan);

/* Largest entry of the delay table, or -1 for a NULL plan. */
int64_t gsp_plan_max_delay(gsp_plan_t plan);

/* n_out = n_in - max_delay (may be <= 0), or -1 for a NULL plan. */
int64_t gsp_plan_nout(gsp_plan_t plan, int64_t n_in);

/* Copy the plan's delay table [ndm][nchan] to host memory. */
gsp_status gsp_plan_delays(gsp_plan_t plan, int32_t *host_out);

/* Dedispersion only (Sec. 2.3, Alg. 3 semantics):
 *   d_out[dm * out_stride + t] = sum_c X[c][t + delay[dm][c]],  t < n_out.
 * d_x: device, n_in <= nsamp_max samples per channel, x_stride >= n_in bytes.
 * d_out: device int32, out_stride >= n_out elements.
 * Alignment: d_x and x_stride multiples of 16 bytes, d_out 16-byte aligned
 * and out_stride a multiple of 4 (else GSP_ERR_ALIGN).
 * GSP_ERR_TOO_SHORT if n_in <= max delay.  Asynchronous on stream. */
gsp_status gsp_dedisperse(gsp_plan_t plan, const uint8_t *d_x, int64_t n_in,
                          int64_t x_stride, int32_t *d_out, int64_t out_stride,
                          void *stream);

/* Dedispersion fused with the single-pulse search (the whole hot path).
 * D goes to d_out (same layout rules as gsp_dedisperse) or, if d_out is
 * NULL, to plan-owned scratch.  t_offset is the absolute sample index of
 * output sample 0 (candidate windows are aligned to absolute indices).
 * Candidates stay on the device until gsp_candidates.  Search steps per DM
 * row: blocks of B samples (samples beyond the last whole block are not
 * searched); least-squares line per block, residual RMS sigma_b; sigma_ref =
 * lower median of sigma_b; blocks outside [bad_lo, bad_hi]*sigma_ref are
 * zeroed; S/N(t, w) = sum_{k<w} r[t+k] / (sigma_ref sqrt(w)); best width per t
 * (ties: smaller w); event if S/N >= threshold; per window the largest event
 * (ties: smaller t).  Asynchronous on stream. */
gsp_status gsp_search(gsp_plan_t plan, const uint8_t *d_x, int64_t n_in,
                      int64_t x_stride, int64_t t_offset, int32_t *d_out,
                      int64_t out_stride, void *stream);

/* Search only, on caller-provided dedispersed series d_D [ndm][stride]
 * (int32, device), n_out samples per row.  Same search as gsp_search. */
gsp_status gsp_search_series(gsp_plan_t plan, const int32_t *d_D, int64_t n_out,
                             int64_t stride, int64_t t_offset, void *stream);

/* S/N of every (dm, width, t) for caller-provided series (parity surface):
 * d_snr[(dm * nwidths + iw) * Ls + t], Ls = B * floor(n_out / B), float,
 * NaN where t + w > Ls, 0 for rows with sigma_ref == 0.  Also leaves the
 * candidates of this search in the plan.  Asynchronous on stream. */
gsp_status gsp_boxcar_snr(gsp_plan_t plan, const int32_t *d_D, int64_t n_out,
                          int64_t stride, float *d_snr, void *stream);

/* Per-row statistics of the last search, copied to host (synchronises):
 * sigma_b [ndm][nb] (nb = floor(n_out/B)), bad [ndm][nb] (1 = bad block),
 * sigma_ref [ndm].  Any pointer may be NULL; nb_out receives nb. */
gsp_status gsp_search_stats(gsp_plan_t plan, double *sigma_b, uint8_t *bad,
                            double *sigma_ref, int64_t *nb_out);

/* Candidates of the last search (synchronises with its stream).  Copies up
 * to cap records, sorted by (dm_idx, t, width), to host_out and the true
 * count to *n_total.  Returns GSP_ERR_CAPACITY if the device buffer
 * (max_cands) or cap was too small; the stored prefix is then the first
 * records in sorted order among those the device kept. */
gsp_status gsp_candidates(gsp_plan_t plan, gsp_cand *host_out, int64_t cap,
                          int64_t *n_total);

/* End-to-end call on HOST data: copies h_x (host, pinned or pageable,
 * x_stride bytes per channel) to plan-owned device memory, runs gsp_search
 * and returns the candidates as gsp_candidates does.  Synchronises.  With the
 * tiled kernel the input is copied in time chunks (8 by default; environment
 * variable GSP_HOST_CHUNKS = 1..8, 1 = copy everything first) on a second
 * stream, each chunk's dedispersion starting when its columns have arrived,
 * so that the copy of chunk k + 1 overlaps the dedispersion of chunk k
 * (overlap needs pinned host memory).  The result does not depend on the
 * chunking. */
gsp_status gsp_search_host(gsp_plan_t plan, const uint8_t *h_x, int64_t n_in,
                           int64_t x_stride, int64_t t_offset, gsp_cand *host_out,
                           int64_t cap, int64_t *n_total, void *stream);

/* Device durations (ms) of the dedispersion kernel and of the search
 * kernels of the last gsp_search / gsp_dedisperse call, measured with CUDA
 * events on its stream; requires GSP_FLAG_TIMING (else GSP_ERR_STATE).
 * Synchronises. */
gsp_status gsp_plan_timing(gsp_plan_t plan, float *ms_dedisperse, float *ms_search);

/* Kernel launches the last gsp_search / gsp_dedisperse call made. */
int32_t gsp_plan_launches(gsp_plan_t plan);

/* Limits of the bounded waits of the plan's tiled dedispersion pipeline (a
 * test knob for the failure path; the paper has no counterpart).  Every wait of
 * a consumer warp for a staged copy, and of the producer warp for a free ring
 * slot, gives up after `cycles` SM clock cycles (1 .. 4e9, default 4e9, about
 * 2 s): the kernel then sets the plan's error flag and its warps leave, and the
 * next synchronising call (gsp_candidates, gsp_plan_timing) returns
 * GSP_ERR_TIMEOUT and clears the flag, so the plan stays usable.  The producer
 * always waits for every copy it issued to land (with the full limit) before
 * its CTA can end, so no copy is ever in flight into released shared memory.
 * With starve = 1 the producer issues no copies at all, so every consumer's
 * first wait runs out (a failure made on purpose, with nothing in flight);
 * starve = 0 restores normal operation.  Host only. */
gsp_status gsp_plan_set_wait_limit(gsp_plan_t plan, int64_t cycles, int32_t starve);

/* Tile variants of the dedispersion kernel (a tuning knob with no paper
 * counterpart; every variant computes the same bit-exact series).  Returns
 * the number of variants; if plan is not NULL and in_use is not NULL, writes
 * the variant the plan uses, or -1 if it uses the simple kernel.  A plan's
 * variant is chosen at gsp_plan_create: the index in the environment variable
 * GSP_DD_VARIANT if that is in range and fits the plan, else the first of a
 * preference list (64-channel stages; 32-channel stages; 7-DM blocks) whose
 * shared-memory stages hold the plan's largest in-block delay spread with at
 * least two ring slots.  The simple kernel (-1) is used only with
 * GSP_FLAG_SIMPLE_DD or when no tiled variant fits the spread (a 7-DM block
 * spread of more than about 3000 samples), never silently otherwise. */
int32_t gsp_dedisperse_variants(gsp_plan_t plan, int32_t *in_use);

/* Autotune the plan's tile variant on the caller's input (a tuning knob with
 * no paper counterpart): every variant of the tuning list that fits the plan
 * runs once to warm up and three times timed, with CUDA events on stream, over
 * the first 131072 output samples of d_x (layout and limits as gsp_dedisperse)
 * into the plan's series scratch (allocated here if needed); the variant with
 * the smallest median becomes the plan's.  *variant and *best_ms (optional)
 * receive it and its median.  Synchronises.  GSP_ERR_STATE for a plan on the
 * simple kernel. */
gsp_status gsp_plan_tune(gsp_plan_t plan, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                         void *stream, int32_t *variant, float *best_ms);

/* The series of the plan's last search (gsp_search, gsp_search_host,
 * gsp_search_series, or a batch search of this plan): its device address, row
 * stride (elements) and n_out.  The address is the caller's d_out or the
 * plan's scratch; it stays valid until the plan is destroyed or searches
 * again.  GSP_ERR_STATE before the first search.  Host only. */
gsp_status gsp_plan_series(gsp_plan_t plan, const int32_t **d_D, int64_t *stride,
                           int64_t *n_out);

/* Search of caller-provided dedispersed series that allocates nothing: for
 * callers that may not call cudaMalloc (for instance a real-time ingest loop
 * whose latency budget a device allocation would break, or an application
 * that owns all device memory through its own pool).  The paper has no
 * counterpart; this is a deployment variant of gsp_search_series.
 *   d_D       device int32 [ndm][stride], n_out samples per row (input);
 *   t_offset  absolute sample index of D[.][0] (windows are absolute);
 *   widths    host array of nwidths ascending widths (NULL: the default 13);
 *   block_len, window_len, threshold, bad_lo, bad_hi: as in gsp_plan_desc;
 *   d_cands   device gsp_cand [max_cands] (output, unsorted, at most one per
 *             (DM row, window));
 *   d_ncand   device uint64 (output): the true number of candidates; records
 *             beyond max_cands are dropped.
 * Working memory is one static device array inside the library, about 7 MB on
 * every GPU that loads it, which limits a call to ndm <= 4096 rows and
 * ndm * floor(n_out / block_len) <= 2^18 search blocks, and the candidate
 * windows of a row to fewer than 2^31; larger calls return GSP_ERR_TOO_LARGE.
 * threshold must be finite (as in gsp_plan_desc).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and caches it
 * for the life of the process; with lazy module loading that call also loads
 * the library's device code, array included, on that device.  So make that
 * first call before any stream capture, and do not use this entry point on a
 * device after cudaDeviceReset.  All calls share the array: calls whose
 * kernels overlap on the GPU race on it, calls queued one after another on
 * one stream do not.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Asynchronous on stream. */
gsp_status gsp_search_series_static(const int32_t *d_D, int32_t ndm, int64_t n_out,
                                    int64_t stride, int64_t t_offset, const int32_t *widths,
                                    int32_t nwidths, int32_t block_len, int32_t window_len,
                                    float threshold, float bad_lo, float bad_hi,
                                    gsp_cand *d_cands, int64_t max_cands,
                                    unsigned long long *d_ncand, void *stream);

/* Streaming search of one beam (the device-resident form of the overlapping
 * read blocks of Alg. 2/3 and of the overlapped merge of adjacent files of
 * Sec. 2.1).  A stream owns two device input buffers of
 * nchan x round16(chunk_out + max_delay) bytes and uses the plan (one stream
 * per plan).  chunk_out must be a multiple of block_len and window_len, and
 * chunk_out + max_delay <= nsamp_max.  Chunk k covers output samples
 * [k chunk_out, (k+1) chunk_out) of the stream; its detrend blocks and candidate
 * windows are aligned to absolute sample indices.  The normalisation
 * (sigma_ref) is per chunk. */
gsp_status gsp_stream_create(gsp_stream_t *out, gsp_plan_t plan, int64_t chunk_out, int32_t beam);

/* Device bytes a new stream of chunk_out samples on this plan will allocate:
 * its two input buffers, plus the plan's series scratch if the plan has not
 * searched yet.  For admitting beams by memory (compare with cudaMemGetInfo).
 * -1 for a NULL plan or chunk_out <= 0.  Host only. */
int64_t gsp_stream_bytes(gsp_plan_t plan, int64_t chunk_out);

/* A pool of nbuf device input buffers, each nchan x round16(chunk_out +
 * max_tail) bytes, shared by the pooled streams of many beams (admission by
 * memory, chunk by chunk).  A pooled stream keeps only its overlap tail on the
 * device; each push takes a pool buffer whose previous chunk has finished, or
 * is refused with GSP_ERR_BUSY and enqueues nothing, so that the caller can
 * queue the chunk and retry.  The buffer returns to the pool when the chunk's
 * copies and search have run on the GPU (an event recorded on the push's
 * stream).  A pool is used from one host thread at a time.  Allocates. */
gsp_status gsp_chunkpool_create(gsp_chunkpool_t *out, int32_t nchan, int64_t chunk_out,
                                int64_t max_tail, int32_t nbuf);
gsp_status gsp_chunkpool_destroy(gsp_chunkpool_t pool);

/* Device bytes of a pool (host only; -1 for invalid sizes). */
int64_t gsp_chunkpool_bytes(int32_t nchan, int64_t chunk_out, int64_t max_tail, int32_t nbuf);

/* Pool buffers free now (polls the buffers' events; -1 for NULL). */
int32_t gsp_chunkpool_free(gsp_chunkpool_t pool);

/* A stream of the plan's beam whose input buffers come from the pool: chunks
 * of the pool's chunk_out samples (a multiple of block_len and window_len);
 * the plan's max delay must be <= the pool's max_tail and chunk_out +
 * max_delay <= nsamp_max.  Owns a device tail buffer of nchan x
 * round16(max_delay) bytes.  Pushes and results as for gsp_stream_create. */
gsp_status gsp_stream_create_pooled(gsp_stream_t *out, gsp_plan_t plan, gsp_chunkpool_t pool,
                                    int32_t beam);

/* Device bytes a new pooled stream will allocate: its tail buffer, plus the
 * plan's series scratch if the plan has not searched yet.  Host only. */
int64_t gsp_stream_pooled_bytes(gsp_plan_t plan, int64_t chunk_out);

/* Free the stream's buffers (synchronises the device; the plan is not freed). */
gsp_status gsp_stream_destroy(gsp_stream_t s);

/* Samples per channel the next push must supply: chunk_out + max_delay for
 * the first push, chunk_out afterwards (-1 for a NULL stream). */
int64_t gsp_stream_need(gsp_stream_t s);

/* Admit the next chunk: h_x is host memory [nchan][h_stride] holding
 * gsp_stream_need(s) new samples per channel (pinned memory makes the copy
 * asynchronous).  Enqueues on stream: the copy of the previous chunk's last
 * max_delay samples (device to device), the host-to-device copy of the new
 * samples, and gsp_search (a pooled stream also keeps the new tail).  Returns
 * GSP_ERR_INVALID_ARG if n differs from gsp_stream_need(s), and for a pooled
 * stream GSP_ERR_BUSY if no pool buffer is free (nothing enqueued).  Read the
 * chunk's results (gsp_stream_results) before the next push of this stream. */
gsp_status gsp_stream_push(gsp_stream_t s, const uint8_t *h_x, int64_t n, int64_t h_stride,
                           void *stream);

/* Candidates of the last pushed chunk, as gsp_candidates, with t converted to
 * the stream's absolute sample index and beam set to the stream's label;
 * *t_abs0 (optional) receives the absolute index of the chunk's first output
 * sample.  Synchronises. */
gsp_status gsp_stream_results(gsp_stream_t s, gsp_cand *host_out, int64_t cap, int64_t *n_total,
                              int64_t *t_abs0);

/* Batched search of up to 32 beams, one plan per beam (each plan its own DM
 * grid and maximum length; all plans the same channel count and tiled
 * dedispersion).  The dedispersion of all beams is one kernel launch over a
 * work list of (beam, time tile, DM block) items (the multi-beam receiver of
 * Sec. 2 searched in one pass); every beam is then searched with its plan's
 * settings and its candidates stay in its plan. */
gsp_status gsp_batch_create(gsp_batch_t *out, const gsp_plan_t *plans, int32_t nbeams,
                            int32_t flags);
gsp_status gsp_batch_destroy(gsp_batch_t b);

/* Search every beam: inputs[i] for plan i (same rules as gsp_search, series
 * into each plan's scratch).  With GSP_BATCH_GRAPH the enqueue sequence is
 * captured on the first call (and again whenever an input changes) and
 * replayed, which needs a created stream (not the legacy NULL stream); with
 * GSP_BATCH_AUTOTUNE the first call also times the tile
 * variants on these inputs.  The first call may therefore allocate and
 * synchronise; later calls with the same inputs are asynchronous on stream. */
gsp_status gsp_batch_search(gsp_batch_t b, const gsp_beam_input *inputs, void *stream);

/* Candidates of the last batch search, sorted by (beam, dm_idx, t), beam set to
 * the plan's index in the batch; *n_total = the true total.  Synchronises. */
gsp_status gsp_batch_candidates(gsp_batch_t b, gsp_cand *host_out, int64_t cap, int64_t *n_total);

/* Device durations (ms) of the batched dedispersion launch and of the whole
 * batch of the last call (events recorded on its stream, replayed with the
 * graph); requires GSP_BATCH_TIMING.  Synchronises. */
gsp_status gsp_batch_timing(gsp_batch_t b, float *ms_dedisperse, float *ms_total);

/* The dedispersion variant in use, the autotuner's best median tuning time
 * (ms, 0 if not tuned) and the kernel launches of the last call (captured ones
 * counted). */
gsp_status gsp_batch_info(gsp_batch_t b, int32_t *variant, float *tuned_ms, int32_t *launches);

/* The autotuner's measurements (a tuning knob with no paper counterpart):
 * writes up to cap (variant, median ms) pairs, one per tile variant it timed,
 * to the host arrays variants and ms (either may be NULL) and returns how many
 * it timed (0 before tuning, -1 for a NULL batch or cap < 0).  A variant is
 * timed if it fits every beam's largest in-block delay spread; each is run
 * three times over every beam's first 65536 output samples. */
int32_t gsp_batch_tune_results(gsp_batch_t b, int32_t *variants, float *ms, int32_t cap);

/* Ingest transpose (the optional first step of the path): time-major 8-bit
 * samples d_in[t][c] (the order of PSRFITS files and of Alg. 2's numpts x
 * numchan input matrix, Sec. 2.3), t < n_samp, c < nchan, row stride in_stride
 * >= nchan bytes, into the channel-major d_out[c][t] the other entry points
 * read (row stride out_stride >= n_samp bytes; a multiple of 16 for them).
 * Device pointers; asynchronous on stream. */
gsp_status gsp_ingest_transpose(const uint8_t *d_in, int64_t n_samp, int32_t nchan,
                                int64_t in_stride, uint8_t *d_out, int64_t out_stride,
                                void *stream);

/* ------------------------------------------------------------------------
 * DDplan ranges and sub-band dedispersion (Sec. 3.1, Tables 2-3; Sec. 2.3).
 * ------------------------------------------------------------------------ */

/* Time downsampling of a filterbank, as used by the DDplan ranges of Sec. 3.1
 * (Tables 2-3, column DownSamp): d_out[c][t] = the mean of d_x[c][t*ds ..
 * t*ds + ds - 1] rounded half up, i.e. floor((2*sum + ds) / (2*ds)), for
 * t < floor(n_in / ds).  d_x, d_out: device uint8 [nchan][stride];
 * 1 <= ds <= 2^20.  Asynchronous on stream. */
gsp_status gsp_downsample(const uint8_t *d_x, int32_t nchan, int64_t n_in, int64_t x_stride,
                          int32_t ds, uint8_t *d_out, int64_t out_stride, void *stream);

/* One DM range of a survey plan (a row of Tables 2-3): trial DMs
 * dm_lo + i * dm_step (i < ndm), searched at the sampling time multiplied by
 * downsamp. */
typedef struct {
    double dm_lo;
    double dm_step;
    int32_t ndm;
    int32_t downsamp;
} gsp_ddplan_range;

/* A DDplan: one plan per range, built from base (band, sampling time,
 * nsamp_max in input samples, search settings; its DM fields are ignored and
 * base->delays must be NULL).  Range r's plan has t_samp * downsamp,
 * nsamp_max / downsamp samples, and its search lengths (block, window,
 * widths) count downsampled samples.  Each distinct factor owns a device
 * buffer of nchan x round16(nsamp_max / downsamp) bytes. */
gsp_status gsp_ddplan_create(gsp_ddplan_t *out, const gsp_plan_desc *base,
                             const gsp_ddplan_range *ranges, int32_t nranges);
gsp_status gsp_ddplan_destroy(gsp_ddplan_t d);

/* Search every range: downsample d_x once per distinct factor, then
 * gsp_search each range's plan on its series (same input rules as
 * gsp_search; t_offset must be a multiple of every factor).  Asynchronous. */
gsp_status gsp_ddplan_search(gsp_ddplan_t d, const uint8_t *d_x, int64_t n_in, int64_t x_stride,
                             int64_t t_offset, void *stream);

/* Candidates of all ranges in range order (each sorted as gsp_candidates):
 * dm_idx indexes the concatenated trial list, t and width are in input
 * samples (downsampled index x factor), beam = range index.  Synchronises. */
gsp_status gsp_ddplan_candidates(gsp_ddplan_t d, gsp_cand *host_out, int64_t cap,
                                 int64_t *n_total);

/* Two-stage sub-band dedispersion (the algorithm of PRESTO's prepsubband that
 * GSP accelerates, Sec. 2.3).  The nchan channels (storage order) form nsub
 * sub-bands of nchan/nsub consecutive channels (nsub must divide nchan); the
 * reference channel of a sub-band is its highest-frequency channel.  Trials
 * are taken in groups of `group` (1..16) consecutive trials; the sub-band DM
 * of group g is trial min(g*group + group/2, ndm - 1).  With Delta_c(DM) the
 * plan's delay table,
 *   stage 1: S[s][g][t] = sum_{c in s} X[c][t + d1[g][c]],
 *            d1[g][c] = Delta_c(sdm_g) - Delta_ref(s)(sdm_g)
 *   stage 2: D[d][t] = sum_s S[s][g(d)][t + d2[d][s]],  d2[d][s] = Delta_ref(s)(DM_d)
 * for t < n_out = n_in - max d1 - max d2.  A trial that is its group's
 * sub-band DM gets exactly the brute-force series; the others are the
 * sub-band approximation.  desc: as for gsp_plan_create (band and DM grid;
 * desc->delays must be NULL).  Owns nsub internal plans and a stage-1 buffer of
 * nsub x nsdm x round4(nsamp_max) int32. */
gsp_status gsp_subband_create(gsp_subband_t *out, const gsp_plan_desc *desc, int32_t nsub,
                              int32_t group);
gsp_status gsp_subband_destroy(gsp_subband_t b);

/* n_out for an input of n_in samples (may be <= 0), -1 for NULL. */
int64_t gsp_subband_nout(gsp_subband_t b, int64_t n_in);

/* Host copies of d1 [nsdm][nchan], d2 [ndm][nsub] and the sub-band DM trial
 * indices [nsdm] (any pointer may be NULL). */
gsp_status gsp_subband_delays(gsp_subband_t b, int32_t *d1, int32_t *d2, int32_t *sdm_idx);

/* Two-stage dedispersion of d_x (device uint8 [nchan][x_stride], d_x and
 * x_stride 16-byte aligned, else GSP_ERR_ALIGN) into d_out (device int32
 * [ndm][out_stride], out_stride >= n_out, 4-byte aligned).  Stage 1 is one
 * persistent launch of the tiled dedispersion kernel over all sub-bands (up
 * to 32 per launch); stage 2 one launch.  GSP_ERR_TOO_SHORT if n_out <= 0.
 * Asynchronous on stream; search the result with gsp_search_series. */
gsp_status gsp_subband_dedisperse(gsp_subband_t b, const uint8_t *d_x, int64_t n_in,
                                  int64_t x_stride, int32_t *d_out, int64_t out_stride,
                                  void *stream);

/* Synchronise stream and report GSP_ERR_TIMEOUT if a bounded wait of a stage-1
 * kernel gave up (the flag is then cleared). */
gsp_status gsp_subband_finish(gsp_subband_t b, void *stream);

/* Kernel launches of the last gsp_subband_dedisperse call. */
int32_t gsp_subband_launches(gsp_subband_t b);

/* ------------------------------------------------------------------------
 * Candidate ranker building blocks (the project's own design; see the
 * ranker entry points below).
 * ------------------------------------------------------------------------ */

/* BF16 GEMM on the tcgen05 tensor cores with FP32 accumulation in tensor
 * memory: d_C[m][n] = sum_k A[m][k] * B[n][k] (+ d_bias[n], then ReLU if relu),
 * m < M, n < N.  d_A: device bf16 [M][lda], d_B: device bf16 [N][ldb], both
 * 16-byte aligned with lda, ldb and K multiples of 8 (else GSP_ERR_ALIGN);
 * d_C: device float [M][ldc].  splitk > 1 splits K over CTAs that add their
 * partial tiles atomically into d_C, which must then hold zeros and gets no
 * bias or ReLU.  d_err (device int32, optional) is set to 1 if a bounded wait
 * gave up.  Asynchronous on stream. */
gsp_status gsp_gemm_bf16(const void *d_A, int64_t lda, const void *d_B, int64_t ldb,
                         float *d_C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                         const float *d_bias, int32_t relu, int32_t splitk, int32_t *d_err,
                         void *stream);

/* Candidate ranker: a small CNN that scores candidates by their 64 x 64
 * DM-time snippets (the project's own design for the ranking step the paper
 * motivates in Sec. 1-2; it ranks the threshold output and never replaces it).
 * Network: three conv 3x3 (pad 1) + bias + ReLU + 2x2 max-pool layers (1 -> 8 ->
 * 16 -> 32 channels), fc 2048 -> 96 + ReLU, fc 96 -> 2 (class 1 = pulse),
 * 202,786 parameters.  All
 * products run with bf16 operands (rounded to nearest even) and FP32
 * accumulation, the convolutions and fc 2048 -> 96 (forward and backward) as
 * tcgen05 GEMMs.  An inference pass (gsp_ranker_forward) fuses each conv
 * layer with its bias, ReLU and pool at the same rounding points: the
 * one-input-channel first layer on the CUDA cores, the other two as implicit
 * tcgen05 GEMMs.  Parameters are one FP32 vector of gsp_ranker_num_params()
 * values in the order w1 b1 w2 b2 w3 b3 w4 b4 w5 b5, conv weights as
 * [co][ci][ky][kx], fc weights as [out][in] with the fc 2048 input index
 * (y * 8 + x) * 32 + c of the last pooled 8 x 8 x 32 map.  Training is mean
 * softmax cross-entropy with Adam (beta1 0.9, beta2 0.999, eps 1e-8). */
int64_t gsp_ranker_num_params(void);

/* Create a ranker for batches of up to max_batch (1..4096) snippets; weights
 * He-uniform from seed, biases 0.  Allocates all device memory. */
gsp_status gsp_ranker_create(gsp_ranker_t *out, int32_t max_batch, uint64_t seed);
gsp_status gsp_ranker_destroy(gsp_ranker_t r);

/* Host copies in and out of the parameter vector; set_params also resets
 * Adam's moments and step count.  get_params optionally returns the
 * gradients of the last training step (either pointer may be NULL).
 * Synchronise the device. */
gsp_status gsp_ranker_set_params(gsp_ranker_t r, const float *host_params);
gsp_status gsp_ranker_get_params(gsp_ranker_t r, float *host_params, float *host_grads);

/* Snippets of n device candidates d_cands (as gsp_candidates returns them)
 * from the series d_D (device int32 [ndm][stride]) of the plan's last search:
 * d_out[k][i][j] (device float [n][64][64]) = sum over the f = max(1,
 * width / 4) samples s of time bin j, centred on t + width / 2, of the
 * normalised series of DM row dm_idx - 32 + i (detrended residual / sigma_ref;
 * 0 in bad blocks, outside the rows or past the searched length), divided by
 * sqrt(f).  Every bin is summed as exact integer runs inside one search block.
 * Two paths give the same floats: direct reads of the 64 f samples of each
 * row (bulk copies through shared memory), or two to three reads per bin of
 * block-local prefix sums of the series, which the plan builds once per
 * search and series (one read and one write of the series into plan memory
 * allocated on first use, ndm x searched length int32).  The prefix path is
 * taken when n * 64 * 64 * 4 samples exceed twice the series (or as
 * gsp_plan_set_snippet_path says).  GSP_ERR_STATE if the plan has not
 * searched, GSP_ERR_OOM if the prefix memory cannot be allocated.  A bounded
 * wait of the direct path that gives up sets the plan's error flag (reported
 * by gsp_candidates or gsp_plan_timing as GSP_ERR_TIMEOUT).  Asynchronous. */
gsp_status gsp_ranker_snippets(gsp_plan_t plan, const int32_t *d_D, int64_t stride,
                               const gsp_cand *d_cands, int32_t n, float *d_out, void *stream);

/* Snippet path of gsp_ranker_snippets for this plan (a test and tuning knob;
 * the paper has no counterpart): 0 automatic (default), 1 direct reads,
 * 2 prefix sums.  Host only. */
gsp_status gsp_plan_set_snippet_path(gsp_plan_t plan, int32_t path);

/* Logits (device float [n][2]) of n snippets (device float [n][64][64]).
 * Asynchronous. */
gsp_status gsp_ranker_forward(gsp_ranker_t r, const float *d_x, int32_t n, float *d_logits,
                              void *stream);

/* One training step on n snippets with labels d_labels (device int32, 0 or
 * 1): forward, gradients of the mean cross-entropy, one Adam update with
 * learning rate lr.  d_loss (device float, optional) receives the batch loss.
 * Asynchronous. */
gsp_status gsp_ranker_train_step(gsp_ranker_t r, const float *d_x, const int32_t *d_labels,
                                 int32_t n, float lr, float *d_loss, void *stream);

/* Synchronise stream; GSP_ERR_TIMEOUT if a tensor-core wait gave up. */
gsp_status gsp_ranker_finish(gsp_ranker_t r, void *stream);

/* Kernel launches of the last forward or training step. */
int32_t gsp_ranker_launches(gsp_ranker_t r);

/* Host copy of an intermediate tensor of the last pass (a parity surface: the
 * paper has no counterpart), for n = the last pass's snippets:
 *   "a0" "a1" "a2"  bf16 pooled outputs of the conv layers, NHWC
 *                   [n][32][32][8], [n][16][16][16], [n][8][8][32];
 *   "z4" float [n][96] ReLU(fc1 + bias), "a4" bf16 [n][96] the same rounded
 *                   to bf16, "z5" float [n][2] logits;
 * and after a training step also
 *   "z0" "z1" "z2"  float ReLU(conv + bias) before pooling, NHWC [n][H][H][C];
 *   "idx0" .. "idx2" uint8 pooling argmax (0..3) per pooled output;
 *   "g5" float [n][2] gradient of the mean loss w.r.t. the logits;
 *   "g4" bf16 [n][96] gradient w.r.t. fc1's output before ReLU;
 *   "ga0" .. "ga2"  float gradient w.r.t. the pooled output of conv layer l;
 *   "gz0" .. "gz2"  bf16 gradient w.r.t. the pre-pool output of conv layer l.
 * *bytes receives the size; GSP_ERR_CAPACITY (nothing copied) if host_out is
 * NULL or cap_bytes is smaller, GSP_ERR_STATE before any pass or for a
 * training tensor after an inference pass, GSP_ERR_INVALID_ARG for an unknown
 * name.  Synchronises the device. */
gsp_status gsp_ranker_tensor(gsp_ranker_t r, const char *name, void *host_out, int64_t cap_bytes,
                             int64_t *bytes);

/* Static text for a status code. */
const char *gsp_status_string(gsp_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *gsp_last_error_string(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t gsp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GSP_H */
