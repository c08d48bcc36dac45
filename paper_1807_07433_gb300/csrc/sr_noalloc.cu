// sr_noalloc.cu -- sr_match_noalloc: the disparity pipeline of sr_match for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host that hands the library a fixed
// device-memory budget and forbids allocation after start-up (real-time
// loops that must not stall on the allocator), plug-in hosts whose own
// allocator owns the device, or code that must not create a context object
// at all.  For them this file keeps every intermediate of one match (warped
// target, block statistics, the cost volume, both label maps, subpixel map)
// in one file-scope device array of fixed size, kSrNoallocScratchBytes, and
// the timeout flag of the bounded waits in a file-scope device word.  Both
// exist on every GPU that loads this library, until the process exits.  The
// kernels are the ones sr_match launches; only where their scratch lives
// differs.
//
// The host only sees stand-ins for those names, never their device
// addresses, so the addresses are looked up with cudaGetSymbolAddress the
// first time the entry point runs in a CUDA context (with that context
// current) and cached under the context's unique ID (cuCtxGetId): a
// context created later -- after a device reset, or a driver-API context
// other than the device's primary one -- gets its own look-up, since the
// module, and with it the arrays, is loaded anew there.  Because that first
// call in a context does the look-up, make it before any stream capture.
//
// Every call shares the one array and leaves its contents behind.  No part of
// it needs to start at zero: each stage writes every element that a later
// stage reads.  Calls whose work overlaps on the GPU (different streams, or
// different host threads without ordering) race on the array.  The timeout
// word is sticky: a bounded wait that runs out sets it, and only
// sr_noalloc_status reads and clears it.
#include <cuda.h>
#include <math.h>

#include <mutex>

#include "../../include/sr.h"
#include "sr_internal.cuh"

namespace {

constexpr size_t kSrNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kCacheSlots = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kSrNoallocScratchBytes];
static __device__ int g_noalloc_err;

// Device addresses of the two arrays in one CUDA context.
struct Addrs {
    unsigned long long ctx_id;
    void *scratch;
    int *err;
};

std::mutex g_lookup_mutex;
Addrs g_cache[kCacheSlots] = {};
int g_cache_used = 0, g_cache_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

template <typename Fn>
Fn driver_fn(const char *name) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<Fn>(p);
}

// Unique ID of the context current on this thread; false if none is current
// or the driver cannot tell.
bool current_context_id(unsigned long long *id) {
    static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device addresses of the scratch array and the timeout word in the current
// context (looked up once per context; without a context ID, on every call).
cudaError_t noalloc_addrs(Addrs *out) {
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (have_id)
        for (int i = 0; i < g_cache_used; ++i)
            if (g_cache[i].ctx_id == id) {
                *out = g_cache[i];
                return cudaSuccess;
            }
    Addrs a{};
    cudaError_t e = cudaGetSymbolAddress(&a.scratch, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&a.err, g_noalloc_err);
    if (e != cudaSuccess) return e;
    // the look-up makes the device's primary context current if none was
    if (!have_id) have_id = current_context_id(&id);
    if (have_id) {
        a.ctx_id = id;
        const int slot = g_cache_used < kCacheSlots ? g_cache_used++ : g_cache_next++ % kCacheSlots;
        g_cache[slot] = a;
    }
    *out = a;
    return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

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
    const size_t b_row = align256(H * sizeof(float2));
    const size_t need = 2 * b_img + 4 * b_ext + b_vol + 2 * b_lbl + b_row;
    if (need > kSrNoallocScratchBytes) return SR_ERR_UNSUPPORTED;   // frame too large

    Addrs addrs;
    if (noalloc_addrs(&addrs) != cudaSuccess) return SR_ERR_CUDA;
    unsigned char *q = static_cast<unsigned char *>(addrs.scratch);
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
    float2 *rowsh = reinterpret_cast<float2 *>(take(b_row));

    cudaStream_t st = (cudaStream_t)cuda_stream;
    sr::AggDebug dbg;   // default bounded waits, reporting to the sticky timeout word
    dbg.err = addrs.err;
    const int Wi = p.width, Hi = p.height, Di = p.max_disp, WEi = Wi + Di - 1;
    // the sheared view of the extended volume (a host-side descriptor)
    CUtensorMap tmap;
    if (!sr::encode_shear_map(&tmap, volx, p.vol_dtype, Wi, Hi, Di, p.agg_radius))
        return SR_ERR_CUDA;
    if (sr::launch_prep(d_left, d_right, pitch_bytes, Wi, Hi, Di, p.ncc_radius, alpha0, alpha1,
                        delta, 0, rw, mu_l, inv_l, mu_r, inv_r, rowsh, st) != cudaSuccess ||
        sr::launch_ncc_sl(d_left, d_right, pitch_bytes, Wi, Hi, Di, p.ncc_radius, 0, alpha0,
                          alpha1, delta, inv_l, inv_r, volx, p.vol_dtype, WEi,
                          sr::ncc_segment(Wi, Hi, Di, p.ncc_radius, p.vol_dtype), st) != cudaSuccess ||
        sr::launch_agg_shear(&tmap, p.vol_dtype, rw, Wi, Hi, Di, p.agg_radius, p.gamma_d,
                             p.gamma_r, lbl_r, nullptr, dbg, st) != cudaSuccess)
        return SR_ERR_CUDA;
    // the reference view last, with the L-R check and post-processing in its
    // epilogue (as in sr_match)
    sr::AggWin post;
    post.post.lbl_r = lbl_r;
    post.post.disp = d_disp;
    post.post.wta = d_wta_or_null;
    post.post.rowsh = rowsh;
    post.post.lr_thresh = p.lr_thresh;
    if (sr::launch_agg(volx, p.vol_dtype, d_left, pitch_bytes, nullptr, Wi, Hi, Di, p.agg_radius,
                       p.gamma_d, p.gamma_r, lbl_l, dsub, nullptr, dbg, st, post, WEi) != cudaSuccess)
        return SR_ERR_CUDA;
    return SR_OK;
}

extern "C" sr_status sr_noalloc_status(void *cuda_stream) {
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return SR_ERR_CUDA;
    Addrs addrs;
    if (noalloc_addrs(&addrs) != cudaSuccess) return SR_ERR_CUDA;
    int flag = 0;
    if (cudaMemcpy(&flag, addrs.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SR_ERR_CUDA;
    if (!flag) return SR_OK;
    const int zero = 0;
    if (cudaMemcpy(addrs.err, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return SR_ERR_CUDA;
    return SR_ERR_TIMEOUT;
}
