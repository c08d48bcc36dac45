// sr_ctx.cuh -- the context behind the opaque sr_ctx of include/sr.h, and the
// error helpers shared by the ABI translation units.  Not installed.
#pragma once
#include <cuda.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>

#include "../../include/sr.h"
#include "sr_internal.cuh"

constexpr int kStages = 4;    // stages of one sr_match with profiling events
constexpr int kProfRing = 512;   // matches whose stage events are kept

struct SrBatch;               // batched-form state, defined in sr_batch.cu
void sr_batch_free(sr_ctx *c);

struct sr_ctx {
    sr_params p{};
    cudaStream_t st = nullptr;
    int device = 0;
    double alpha0 = 0, alpha1 = 0, delta = 0;
    double f_px = 0, baseline = 0, u0 = 0, v0 = 0;
    bool camera = false;
    // scratch (owned)
    float *rw = nullptr, *mu_l = nullptr, *inv_l = nullptr, *mu_r = nullptr, *inv_r = nullptr;
    // cost volumes, element type p.vol_dtype: vol_l holds the extended
    // reference volume of sr_match (both views, row pitch W + D - 1) or the
    // reference volume of sr_match_restricted (pitch W), vol_r the target
    // volume of sr_match_restricted
    void *vol_l = nullptr, *vol_r = nullptr;
    bool vol_ext = false;            // the last match left the extended layout
    CUtensorMap tmap_x{};            // sheared view of vol_l (launch_agg_shear)
    bool tmap_x_ok = false;
    float *dsub = nullptr;
    float2 *rowsh = nullptr;         // [H] split row shifts of the last prep
    // sr_match_rows: full-disparity and label maps of the last band with its
    // halo rows (on first use, W*H each), and the sheared view of vol_l for
    // a band of band_rows image rows
    float *band_disp = nullptr;
    int16_t *band_wta = nullptr;
    CUtensorMap tmap_band{};
    int band_rows = 0;
    int16_t *lbl_l = nullptr, *lbl_r = nullptr;
    float *agg_l = nullptr, *agg_r = nullptr;
    // host-buffer staging: slot 0 for sr_match_host; slots 0 and 1 for
    // sr_match_host_async (frame k uses slot k mod 2)
    uint8_t *stage_l = nullptr, *stage_r = nullptr;
    float *stage_disp = nullptr;
    // sr_match_host_async: upload and download streams, per-slot events
    // (upload done, match done, download done), next slot, frames queued
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_up[2] = {}, ev_comp[2] = {}, ev_down[2] = {};
    int slot = 0;
    long long frames_queued = 0;
    int *h_err_async = nullptr;   // pinned [2]: the error word after each slot's frame
    int debug = 0;
    int ncc_seg = 0;                 // row segment of the NCC kernel for this frame size
    int *d_err = nullptr;            // device word set by a kernel whose bounded wait ran out
    bool matched = false, agg_valid = false;
    bool profiling = false, timed = false;
    // stage events of the last kProfRing matches while profiling: match k
    // uses ev_ring[(k % kProfRing) * (kStages + 1) ...]; prof_count matches
    // recorded since profiling was enabled
    cudaEvent_t *ev_ring = nullptr;
    long long prof_count = 0;
    char err[256] = {0};
    SrBatch *batch = nullptr;        // batched-form resources (sr_batch.cu), on first use
    // sr_grad_plane scratch, on first use: wsum and grw [H*W], FP64 partials and,
    // for 16-bit cost volumes, an FP32 reference volume [H*W*D]
    float *g_vol = nullptr, *g_wsum = nullptr, *g_rw = nullptr;
    double *g_partial = nullptr;     // block partials, then 3 results at the end
    // sr_match_restricted: per-tile bands and tensor maps of the two volumes
    int *band = nullptr;
    int2 *nrange = nullptr;          // per-tile NCC disparity ranges
    bool tmaps = false, vols_zeroed = false;
    CUtensorMap tmap_l{}, tmap_r{};
    // sr_fit_alpha / sr_fit_roll scratch, grown on demand
    int fit_cap = 0;                 // hypotheses the buffers hold
    int *f_pairs = nullptr, *f_has = nullptr, *f_counts = nullptr;
    float2 *f_model = nullptr;
    double *f_partial = nullptr;     // fit_blocks(W*H) * 9 partials, then 9 sums
};

namespace {

// Host-side diagnostics on stderr, off unless the environment sets
// SR_LOG_LEVEL: 1 = errors and device timeouts, 2 = also context creation
// and the batch autotuner's choices.  Read once per process.
inline int sr_log_level() {
    static const int level = [] {
        const char *e = getenv("SR_LOG_LEVEL");
        return e ? atoi(e) : 0;
    }();
    return level;
}
#define SR_LOG(level, ...)                                   \
    do {                                                     \
        if (sr_log_level() >= (level)) {                     \
            fprintf(stderr, "sr: " __VA_ARGS__);             \
            fputc('\n', stderr);                             \
        }                                                    \
    } while (0)

// An NVTX range on the calling thread for the lifetime of the object: the
// API calls and the stages of a match show up by name in NVTX-aware tools
// (nothing is recorded when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline sr_status fail_cuda(sr_ctx *c, cudaError_t e, const char *what) {
    if (e == sr::kOobError) {   // only a bounds-checked build's launchers return it
        if (c) snprintf(c->err, sizeof(c->err), "%s: an index outside its buffer (sr_bounds_report)", what);
        SR_LOG(1, "%s: an index outside its buffer", what);
        return SR_ERR_BOUNDS;
    }
    if (c) snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
    SR_LOG(1, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
}

#define SR_TRY(c, expr, what)                           \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return fail_cuda(c, e_, what); \
    } while (0)

// After the stream is synchronised: report (and clear) a device-side timeout.
inline sr_status take_device_error(sr_ctx *c) {
    int h = 0;
    cudaError_t e = cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(c, e, "cudaMemcpy(err)");
    if (h == 0) return SR_OK;
    cudaMemset(c->d_err, 0, sizeof(int));
    snprintf(c->err, sizeof(c->err), "a bounded device wait for a cost-row copy ran out");
    SR_LOG(1, "%s", c->err);
    return SR_ERR_TIMEOUT;
}

inline sr::AggDebug agg_debug(const sr_ctx *c) {
    sr::AggDebug d;
    d.err = c->d_err;
    if (c->debug & SR_DEBUG_WITHHOLD_ROW) {
        d.withhold_last = 1;
        d.wait_cycles = 2000000;            // ~1 ms
    }
    return d;
}

}  // namespace
