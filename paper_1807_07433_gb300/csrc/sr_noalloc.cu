// sr_noalloc.cu -- sr_match_noalloc: the disparity pipeline of sr_match for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host that hands the library a fixed
// device-memory budget and forbids allocation after start-up (real-time
// loops that must not stall on the allocator), plug-in hosts whose own
// allocator owns the device, or code that must not create a context object
// at all.  For them this file keeps every intermediate of one match (warped
// target, block statistics, both cost volumes, both label maps, subpixel
// map) in one file-scope device array of fixed size, kSrNoallocScratchBytes.
// The array exists on every GPU that loads this library, until the process
// exits.  The kernels are the ones sr_match launches; only where their
// scratch lives differs.
//
// The host only sees a stand-in for the array's name, never its device
// address, so the address is looked up with cudaGetSymbolAddress the first
// time the entry point runs on a device (with that device current) and
// cached per device.  Because that first call does the look-up, make it
// before any stream capture.
//
// Every call shares the one array and leaves its contents behind.  No part of
// it needs to start at zero: each stage writes every element that a later
// stage reads.  Calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on the array.
#include <cuda.h>
#include <math.h>

#include <mutex>

#include "../../include/sr.h"
#include "sr_internal.cuh"

namespace {

constexpr size_t kSrNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kSrNoallocScratchBytes];

std::mutex g_lookup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool pos_finite(float x) { return isfinite(x) && x > 0.0f; }

}  // namespace

extern "C" sr_status sr_match_noalloc(const sr_params *params, double alpha0, double alpha1,
                                      double delta, const uint8_t *d_left,
                                      const uint8_t *d_right, int pitch_bytes, float *d_disp,
                                      int16_t *d_wta_or_null, void *cuda_stream) {
    if (!params || !d_left || !d_right || !d_disp) return SR_ERR_INVALID_ARG;
    const sr_params &p = *params;
    if (p.width < 1 || p.height < 1 || p.width > 16384 || p.height > 16384 || p.max_disp < 1 ||
        p.ncc_radius < 0 || p.agg_radius < 0 || !pos_finite(p.gamma_d) ||
        !pos_finite(p.gamma_r) || !(p.lr_thresh >= 0.0f) || !isfinite(p.lr_thresh) ||
        pitch_bytes < p.width || !isfinite(alpha0) || !isfinite(alpha1) || !isfinite(delta))
        return SR_ERR_INVALID_ARG;
    if (!sr::ncc_supported(p.max_disp, p.ncc_radius) ||
        !sr::agg_supported(p.max_disp, p.agg_radius) ||
        (p.vol_dtype != SR_VOL_F32 && p.vol_dtype != SR_VOL_F16 && p.vol_dtype != SR_VOL_BF16))
        return SR_ERR_UNSUPPORTED;

    // Carve the scratch: the same arrays sr_create allocates, 256-byte aligned.
    const size_t W = p.width, H = p.height, D = p.max_disp, npx = W * H, WE = W + D - 1;
    const size_t b_img = align256(npx * sizeof(float));
    const size_t b_ext = align256(H * WE * sizeof(float));
    const size_t b_vol = align256(H * WE * D * sr::vol_elem_bytes(p.vol_dtype));   // extended
    const size_t b_lbl = align256(npx * sizeof(int16_t));
    const size_t need = 2 * b_img + 4 * b_ext + b_vol + 2 * b_lbl;
    if (need > kSrNoallocScratchBytes) return SR_ERR_UNSUPPORTED;   // frame too large

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return SR_ERR_CUDA;
    unsigned char *q = static_cast<unsigned char *>(base);
    auto take = [&q](size_t b) { unsigned char *r = q; q += b; return r; };
    float *rw = reinterpret_cast<float *>(take(b_img));
    float *dsub = reinterpret_cast<float *>(take(b_img));
    float *mu_l = reinterpret_cast<float *>(take(b_ext));
    float *inv_l = reinterpret_cast<float *>(take(b_ext));
    float *mu_r = reinterpret_cast<float *>(take(b_ext));
    float *inv_r = reinterpret_cast<float *>(take(b_ext));
    void *volx = take(b_vol);
    int16_t *lbl_l = reinterpret_cast<int16_t *>(take(b_lbl));
    int16_t *lbl_r = reinterpret_cast<int16_t *>(take(b_lbl));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const sr::AggDebug dbg;   // default bounded waits; no error word to report through
    const int Wi = p.width, Hi = p.height, Di = p.max_disp, WEi = Wi + Di - 1;
    // the sheared view of the extended volume (a host-side descriptor)
    CUtensorMap tmap;
    if (!sr::encode_shear_map(&tmap, volx, p.vol_dtype, Wi, Hi, Di, p.agg_radius))
        return SR_ERR_CUDA;
    if (sr::launch_prep(d_left, d_right, pitch_bytes, Wi, Hi, Di, p.ncc_radius, alpha0, alpha1,
                        delta, rw, mu_l, inv_l, mu_r, inv_r, st) != cudaSuccess ||
        sr::launch_ncc(false, d_left, pitch_bytes, rw, mu_l, inv_l, mu_r, inv_r, Wi, Hi, Di,
                       p.ncc_radius, volx, p.vol_dtype, st, nullptr, WEi) != cudaSuccess ||
        sr::launch_agg_shear(&tmap, p.vol_dtype, rw, Wi, Hi, Di, p.agg_radius, p.gamma_d,
                             p.gamma_r, lbl_r, nullptr, dbg, st) != cudaSuccess)
        return SR_ERR_CUDA;
    // the reference view last, with the L-R check and post-processing in its
    // epilogue (as in sr_match)
    sr::AggWin post;
    post.post.lbl_r = lbl_r;
    post.post.disp = d_disp;
    post.post.wta = d_wta_or_null;
    post.post.alpha0 = alpha0;
    post.post.alpha1 = alpha1;
    post.post.delta = delta;
    post.post.lr_thresh = p.lr_thresh;
    if (sr::launch_agg(volx, p.vol_dtype, d_left, pitch_bytes, nullptr, Wi, Hi, Di, p.agg_radius,
                       p.gamma_d, p.gamma_r, lbl_l, dsub, nullptr, dbg, st, post, WEi) != cudaSuccess)
        return SR_ERR_CUDA;
    return SR_OK;
}
