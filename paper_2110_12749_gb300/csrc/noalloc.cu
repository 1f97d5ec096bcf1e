// gsp_search_series_static: the single-pulse search of caller-provided
// dedispersed series, for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a real-time ingest loop in
// which a device allocation (which can synchronise the device and takes a
// driver-wide lock) would break its latency budget, or a host application
// that owns every byte of device memory through its own pool and forbids
// libraries from allocating behind its back.  Such a caller can still run the
// search: it passes the series and the output buffers, and the search's
// working memory (per-block statistics and per-row normalisation) comes from
// one fixed array compiled into this library instead of from a plan.
//
// The array lives in device global memory for as long as the library is
// loaded, on every GPU that loads it.  Its address is looked up once per
// device (cudaGetSymbolAddress) on the first call made with that device
// current; with lazy module loading that first call is also the one that
// loads this library's device code on the device and with it the array, so
// it should come before any stream capture.  The address is cached for the
// life of the process: after cudaDeviceReset on a device the cached address
// is stale, so this entry point must not be used on that device again.
// Every call shares the array, so calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it; calls issued
// one after another on one stream are safe.  Nothing in the array has to
// start at zero: each call writes every entry it later reads.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "gsp_internal.cuh"

namespace {

// Limits of the static scratch: at most kMaxRows DM rows and at most
// kMaxRowBlocks (DM row, search block) pairs per call.
constexpr int kMaxRows = 4096;
constexpr int64_t kMaxRowBlocks = (int64_t)1 << 18;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffSigma = 0;
constexpr size_t kOffBad = align256(kOffSigma + kMaxRowBlocks * sizeof(double));
constexpr size_t kOffParam = align256(kOffBad + kMaxRowBlocks * sizeof(uint8_t));
constexpr size_t kOffScale = align256(kOffParam + kMaxRowBlocks * sizeof(gsp::BlockParam));
constexpr size_t kOffSref =
    align256(kOffScale + (size_t)kMaxRows * gsp::kMaxWidths * sizeof(float));
constexpr size_t kScratchBytes = align256(kOffSref + (size_t)kMaxRows * sizeof(double));

// The shared working memory (about 7 MB).  In host code this name is only a
// handle for cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_search_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

const int32_t kDefaultWidths[13] = {1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150};

}  // namespace

extern "C" gsp_status gsp_search_series_static(
    const int32_t *d_D, int32_t ndm, int64_t n_out, int64_t stride, int64_t t_offset,
    const int32_t *widths, int32_t nwidths, int32_t block_len, int32_t window_len,
    float threshold, float bad_lo, float bad_hi, gsp_cand *d_cands, int64_t max_cands,
    unsigned long long *d_ncand, void *stream) {
    if (!d_D || !d_cands || !d_ncand || ndm <= 0 || n_out <= 0 || stride < n_out ||
        max_cands <= 0 || block_len <= 0 || window_len <= 0 || !(bad_lo <= bad_hi) ||
        !std::isfinite(threshold))
        return GSP_ERR_INVALID_ARG;
    const int32_t *w = widths ? widths : kDefaultWidths;
    const int nw = widths ? nwidths : 13;
    if (nw <= 0 || nw > gsp::kMaxWidths) return GSP_ERR_INVALID_ARG;
    for (int i = 0; i < nw; i++)
        if (w[i] < 1 || (i && w[i] <= w[i - 1])) return GSP_ERR_INVALID_ARG;
    if (w[nw - 1] > block_len || w[nw - 1] > 1024) return GSP_ERR_INVALID_ARG;
    const int64_t nb = n_out / block_len;
    if (ndm > kMaxRows || (int64_t)ndm * nb > kMaxRowBlocks) return GSP_ERR_TOO_LARGE;
    // one boxcar CTA per candidate window of a row: the window count must fit a grid dimension
    if ((nb * block_len) / window_len + 2 > (int64_t)INT32_MAX) return GSP_ERR_TOO_LARGE;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSP_ERR_CUDA;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_search_scratch);
            if (e != cudaSuccess || !p) return GSP_ERR_CUDA;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    gsp::SearchScratch sc;
    sc.sigma_b = reinterpret_cast<double *>(b + kOffSigma);
    sc.bad = b + kOffBad;
    sc.bparam = reinterpret_cast<gsp::BlockParam *>(b + kOffParam);
    sc.scale = reinterpret_cast<float *>(b + kOffScale);
    sc.sref = reinterpret_cast<double *>(b + kOffSref);
    sc.nb_stride = std::max<int64_t>(nb, 1);
    gsp::SearchConfig cfg;
    cfg.ndm = ndm;
    cfg.block_len = block_len;
    cfg.window_len = window_len;
    cfg.threshold = threshold;
    cfg.bad_lo = (double)bad_lo;
    cfg.bad_hi = (double)bad_hi;
    cfg.widths = w;
    cfg.nwidths = nw;
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(d_ncand, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
        e = gsp::launch_search_explicit(sc, cfg, d_D, n_out, stride, t_offset, d_cands, d_ncand,
                                        max_cands, s);
    return e == cudaSuccess ? GSP_OK : GSP_ERR_CUDA;
}
