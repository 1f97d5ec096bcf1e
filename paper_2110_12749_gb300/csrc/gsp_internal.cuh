// Internal declarations of libgsp (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gsp.h"

namespace gsp {

constexpr int kMaxWidths = 32;
constexpr long long kWaitLimit = 4000000000ll;  // ~2 s of SM clock: the longest bounded wait

// DM trials per CTA of the tiled dedispersion kernel (one per consumer warp):
// 16; 15 so that the CTA (15 consumer warps + 1 producer) is 16 warps and each
// thread may hold up to 128 registers; or 7 for two 8-warp CTAs per SM at the
// same register budget.  Plans keep the DM-block tables of every size so that
// any tile variant can run on any plan.
constexpr int kNumKdm = 3;
constexpr int kKdmSizes[kNumKdm] = {16, 15, 7};
inline int kdm_index(int kdm) { return kdm == 15 ? 1 : (kdm == 7 ? 2 : 0); }

// Per-block parameters consumed by the boxcar kernel, derived in FP64 from
// exact integer block sums and rounded once to FP32:
//   m    = nearest integer to the block mean (the integer series is D - m),
//   c0   = alpha - m  (intercept of the fitted line minus m),
//   beta = slope of the fitted line,
//   good = 1 if the block is searched, 0 if it is bad (zeroed).
// 16-byte aligned, so that a kernel reads one record with a single 128-bit load
// (every array of them is a cudaMalloc block or a 256-byte aligned region).
struct alignas(16) BlockParam {
    int32_t m;
    float c0;
    float beta;
    int32_t good;
};

// Channels per shared-memory stage of the tiled kernel: 64 or 32.  Plans keep
// the per-stage tables of both widths (index cb_index(cb)).
constexpr int kNumCb = 2;
constexpr int kCbSizes[kNumCb] = {64, 32};
inline int cb_index(int cb) { return cb == 32 ? 1 : 0; }

// Tile geometry of the performance dedispersion kernel, chosen per plan.
struct DDGeom {
    int kdm = 0;       // DM trials per CTA of the plan's variant
    int t_cta = 0;     // output samples computed per CTA (t_eff stored)
    int t_eff = 0;     // output samples stored per CTA (tiles overlap)
    int cb = 0;        // channels per shared-memory stage
    int win = 0;       // bytes per channel window in shared memory (the widest stage)
    int stages = 0;    // pipeline depth
    int smem = 0;      // dynamic shared memory bytes
    int ctas_per_sm = 1;
    // per DM-block size kKdmSizes[o]:
    int nblk[kNumKdm] = {};            // DM blocks
    int grp[kNumKdm] = {1, 1, 1};      // DM blocks per launch group
    int64_t spread[kNumKdm] = {};      // largest delay spread inside a DM block
    int variant = 0;   // template variant index
};

// Launch geometry of one tile variant for a given largest in-block delay
// spread: window bytes per channel, ring depth, shared memory and CTAs per
// SM.  ok = false if fewer than two stages fit.
struct TileFit {
    bool ok = false;
    int win = 0;
    int stages = 0;
    int smem = 0;
    int ctas_per_sm = 1;
};

}  // namespace gsp

struct gsp_plan_s {
    gsp_plan_desc desc{};
    std::vector<double> dms;
    std::vector<int32_t> delays_h;  // [ndm][nchan]
    std::vector<int32_t> widths;
    int64_t max_delay = 0;
    int device = 0;
    int num_sms = 0;
    bool simple_dd = false;

    // device memory owned by the plan
    int32_t *d_delays = nullptr;     // [ndm][nchan]
    int32_t *d_blkmin[gsp::kNumKdm] = {};  // [nblk][nchan] min delay per DM block
    // per stage width kCbSizes[i]: (delay << 8) | phase-list position [ndm][nchan],
    // and the four phase-family sizes of every (DM, stage) [ndm][ceil(nchan / cb)]
    int32_t *d_dpos[gsp::kNumCb] = {};
    uint32_t *d_fcnt[gsp::kNumCb] = {};
    // largest in-block delay spread of each stage's channels, per DM-block size
    // and stage width [ceil(nchan / cb)] (sizes each stage's copy window)
    int32_t *d_stspread[gsp::kNumKdm][gsp::kNumCb] = {};
    int *d_err = nullptr;            // set by a kernel whose bounded wait gave up
    unsigned long long *d_bsum = nullptr;  // [ndm][nb_max][3] block sums (tiled path)
    double *d_sigma_b = nullptr;     // [ndm][nb_max]
    uint8_t *d_bad = nullptr;        // [ndm][nb_max]
    gsp::BlockParam *d_bparam = nullptr;  // [ndm][nb_max]
    float *d_scale = nullptr;        // [ndm][nwidths] 1/(sigma_ref sqrt(w)), 0 if sigma_ref == 0
    double *d_sref = nullptr;        // [ndm]
    gsp_cand *d_cands = nullptr;     // [max_cands]
    unsigned long long *d_ncand = nullptr;
    gsp_cand *d_slots = nullptr;     // [ndm][nwin_max] one result per (row, window)
    unsigned int *d_chunk = nullptr;  // compaction chunk counts / offsets
    int64_t nwin_max = 0;
    int32_t *d_D = nullptr;          // lazily allocated dedispersed scratch
    size_t d_D_elems = 0;
    uint8_t *d_xstage = nullptr;     // lazily allocated input staging for host calls
    size_t d_xstage_bytes = 0;
    int64_t nb_max = 0;

    gsp::DDGeom geom;

    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    // host-input pipeline (gsp_search_host): copy stream and its events, created on first use
    cudaStream_t h2d_stream = nullptr;
    cudaEvent_t h2d_ev[9] = {};  // one per chunk + one for the caller's stream
    bool timed = false;
    // bounded waits of the tiled dedispersion pipeline (gsp_plan_set_wait_limit)
    long long wait_budget = gsp::kWaitLimit;
    int wait_starve = 0;
    cudaStream_t last_stream = nullptr;
    int64_t last_nout = -1;
    int64_t last_nb = 0;
    const int32_t *last_D = nullptr;  // series of the last search and its row stride
    int64_t last_stride = 0;
    bool have_search = false;
    uint64_t search_seq = 0;          // searches run (incremented by every search)
    // block-local inclusive prefix sums of a series for the snippet kernel,
    // lazily allocated [ndm][prefix_stride]; valid for (prefix_seq, prefix_src)
    int32_t *d_prefix = nullptr;
    size_t d_prefix_elems = 0;
    int64_t prefix_stride = 0;
    uint64_t prefix_seq = 0;
    const int32_t *prefix_src = nullptr;
    int64_t prefix_src_stride = 0;
    int snippet_path = 0;             // 0 automatic, 1 direct reads, 2 prefix sums
    int32_t *d_order = nullptr;       // snippet CTAs' candidate order (by time bucket)
    size_t d_order_elems = 0;
    uint32_t *d_order_hist = nullptr;  // [1024] time-bucket counts / offsets
    float *d_sinv = nullptr;          // [ndm] 1 / sigma_ref in FP32 for the snippet kernels
    int32_t launches = 0;
};

namespace gsp {

// Kernel launchers (dedisperse.cu, search.cu).  Each returns the CUDA error
// of its launch(es) and adds the number of kernels it launched to *nlaunch.
cudaError_t launch_dedisperse_simple(const gsp_plan_s *p, const uint8_t *x, int64_t x_stride,
                                     int64_t n_out, int32_t *out, int64_t out_stride,
                                     cudaStream_t s, int32_t *nlaunch);
// One beam of a batched dedispersion launch.
struct BeamLaunch {
    const gsp_plan_s *plan;
    const uint8_t *x;
    int64_t n_in, x_stride, n_out;
    int32_t *out;
    int64_t out_stride;
    unsigned long long *bsum;  // optional block sums (zeroed by the caller)
};

// All beams (same channel count, at most 32) in one launch of the tiled kernel
// `variant`; persistent = at most num_sms CTAs striding over the work items.
cudaError_t launch_dedisperse_batch(const BeamLaunch *beams, int nbeams, int variant,
                                    bool persistent, int num_sms, int *err, cudaStream_t s,
                                    int32_t *nlaunch);
int dedisperse_num_variants();
// Variants the batch autotuner may time, in order of preference.
int dedisperse_tune_candidates(const int **list);
// Geometry of variant v for the largest in-block spreads (per DM-block size).
TileFit dedisperse_fit(int variant, const int64_t (&spread)[kNumKdm]);
// Whether variant v can run on plan p (its tables exist and its tiles fit).
bool dedisperse_variant_usable(const gsp_plan_s *p, int variant);
// Make variant v the plan's (it must be usable); updates the tile geometry.
void dedisperse_set_variant(gsp_plan_s *p, int variant);
// The preferred tiled variant for a set of plans dedispersed in one launch
// (largest spreads over the plans), or -1 if no tiled variant fits.
int dedisperse_choose_variant(const gsp_plan_s *const *plans, int nplans);

// gsp_api.cu helpers shared with the batch module.
void record_error(cudaError_t e, const char *what);

// Raise kernel fn's dynamic shared-memory limit to at least smem bytes on the
// current device, and (max_carveout) ask for the largest shared-memory
// carveout.  Kernel attributes belong to a device, so the setting is
// remembered per (device, kernel); thread-safe.  Returns the CUDA error.
cudaError_t ensure_kernel_smem(const void *fn, int smem, bool max_carveout = false);

// A kernel launched as a programmatic dependent of the previous kernel in its
// stream (launch_dependent) may start while that kernel drains; it waits here,
// before it touches that kernel's output, until the kernel has completed and
// its writes are visible.  A no-op when the kernel was launched normally.
__device__ __forceinline__ void wait_prior_grid() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Launch kern as a programmatic dependent of the previous kernel in stream s
// (its blocks may be scheduled before that kernel ends; see wait_prior_grid).
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
gsp_status plan_prepare_search(gsp_plan_s *p, int64_t n_out, int32_t **D, int64_t *stride,
                               unsigned long long **bsum);
gsp_status plan_check_input(gsp_plan_s *p, const uint8_t *x, int64_t n_in, int64_t x_stride,
                            int64_t *n_out);

// bsum (optional): int64 [ndm][nb_max][3] exact block sums {S0, S1, S2} over
// blocks of block_len samples, accumulated atomically (must be zeroed first).
cudaError_t launch_dedisperse_tiled(const gsp_plan_s *p, const uint8_t *x, int64_t n_in,
                                    int64_t x_stride, int64_t n_out, int32_t *out,
                                    int64_t out_stride, unsigned long long *bsum,
                                    cudaStream_t s, int32_t *nlaunch);
// Phase-sorted list positions of cb-channel stages (empty if the delays do
// not fit the packed form).
void plan_phase_lists(const gsp_plan_s *p, int cb, std::vector<int32_t> *dpos,
                      std::vector<uint32_t> *fcnt);
// Host tables of the tiled kernel for a plan.
struct TiledTables {
    std::vector<int32_t> blkmin[kNumKdm];
    std::vector<int32_t> dpos[kNumCb];
    std::vector<uint32_t> fcnt[kNumCb];
    std::vector<int32_t> stspread[kNumKdm][kNumCb];
};
// DM-block tables and per-stage spreads of every block size and stage width,
// then the plan's variant and geometry.  Returns false (the plan then uses
// the simple kernel) only if no tiled variant fits the plan's delay spread.
bool plan_dedisperse_tiled(gsp_plan_s *p, TiledTables *tab);

// bsum (optional): block sums left by the tiled dedispersion kernel.
cudaError_t launch_search(gsp_plan_s *p, const int32_t *D, int64_t n_out, int64_t stride,
                          int64_t t_offset, float *snr_out, const unsigned long long *bsum,
                          cudaStream_t s, int32_t *nlaunch);

// Explicit scratch and parameters of the search kernels, for callers that
// provide their own scratch (the no-allocation entry point).
struct SearchScratch {
    double *sigma_b;        // [ndm][nb_stride]
    uint8_t *bad;           // [ndm][nb_stride]
    BlockParam *bparam;     // [ndm][nb_stride]
    float *scale;           // [ndm][nwidths]
    double *sref;           // [ndm]
    int64_t nb_stride;
};

struct SearchConfig {
    int ndm;
    int block_len;
    int64_t window_len;
    float threshold;
    double bad_lo, bad_hi;
    const int32_t *widths;  // host
    int nwidths;
};

// Launch the search kernels (block statistics from the series, sigma_ref,
// boxcar) with explicit scratch; candidates go to cands / ncand (ncand is
// not zeroed here).
cudaError_t launch_search_explicit(const SearchScratch &sc, const SearchConfig &cfg,
                                   const int32_t *D, int64_t n_out, int64_t stride,
                                   int64_t t_offset, gsp_cand *cands,
                                   unsigned long long *ncand, int64_t max_cands, cudaStream_t s);

}  // namespace gsp
