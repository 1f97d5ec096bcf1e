// Internal declarations of libgsp (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "gsp.h"

namespace gsp {

constexpr int kMaxWidths = 32;

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
struct BlockParam {
    int32_t m;
    float c0;
    float beta;
    int32_t good;
};

// Tile geometry of the performance dedispersion kernel, chosen per plan.
struct DDGeom {
    int kdm = 0;       // DM trials per CTA of the plan's variant
    int t_cta = 0;     // output samples computed per CTA (t_eff stored)
    int t_eff = 0;     // output samples stored per CTA (tiles overlap)
    int cb = 0;        // channels per shared-memory stage
    int win = 0;       // bytes per channel window in shared memory
    int stages = 0;    // pipeline depth
    int smem = 0;      // dynamic shared memory bytes
    // per DM-block size kKdmSizes[o]:
    int nblk[kNumKdm] = {};            // DM blocks
    int grp[kNumKdm] = {1, 1, 1};      // DM blocks per launch group
    int64_t spread[kNumKdm] = {};      // largest delay spread inside a DM block
    int variant = 0;   // template variant index
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
    int32_t *d_dpos = nullptr;       // [ndm][nchan] (delay << 8) | phase-list position
    uint32_t *d_fcnt = nullptr;      // [ndm][ceil(nchan / 64)] phase family sizes
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
    cudaStream_t last_stream = nullptr;
    int64_t last_nout = -1;
    int64_t last_nb = 0;
    bool have_search = false;
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
int dedisperse_tune_candidates(const int **list);

// gsp_api.cu helpers shared with the batch module.
void record_error(cudaError_t e, const char *what);
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
// Phase-sorted list positions of 64-channel stages (empty if the delays do
// not fit the packed form), then the tile geometry and variant.
void plan_phase_lists(const gsp_plan_s *p, std::vector<int32_t> *dpos,
                      std::vector<uint32_t> *fcnt);
bool plan_dedisperse_tiled(gsp_plan_s *p, std::vector<int32_t> (&blkmin)[kNumKdm],
                           bool have_lists);

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
