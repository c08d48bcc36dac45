// sr_internal.cuh -- launchers shared by the kernel translation units and the
// C ABI layer (sr_api.cu).  Not installed; the public interface is sr.h.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sr {

// ---- bounds-checked build (-DSR_BOUNDS_CHECK) ------------------------------
// SR_CHECK(i, n, site) is true when 0 <= i < n.  Otherwise it records the
// first offender of this translation unit -- site number and index -- in the
// device word g_sr_oob and is false, and the caller skips the access (a
// skipped load reads 0).  After each launch the unit's launcher calls
// SR_OOB_COLLECT, which (outside stream capture) synchronises the stream,
// moves a recorded offence to the host record (oob_record, sr_api.cu) and
// returns kOobError, which the C ABI reports as SR_ERR_BOUNDS.  In release
// builds SR_CHECK is the constant true and SR_OOB_COLLECT does nothing.
// Site numbers: 1xx NCC, 2xx aggregation, 3xx per-pixel kernels.
constexpr cudaError_t kOobError = cudaErrorAssert;   // no kernel here asserts
#ifdef SR_BOUNDS_CHECK
static __device__ unsigned long long g_sr_oob;
__device__ __forceinline__ bool sr_check(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_sr_oob, 0ull,
              (1ull << 63) | ((unsigned long long)(site & 0x7fff) << 48) |
                  ((unsigned long long)i & 0xffffffffffffull));
    return false;
}
// host record of an offence (the word above, the unit's source file)
void oob_record(unsigned long long word, const char *unit);
static inline cudaError_t sr_oob_collect(cudaStream_t st, const char *unit) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return cudaSuccess;   // a captured launch is checked by the next plain one
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    unsigned long long w = 0;
    e = cudaMemcpyFromSymbol(&w, g_sr_oob, sizeof(w));
    if (e != cudaSuccess) return e;
    if (!w) return cudaSuccess;
    oob_record(w, unit);
    const unsigned long long z = 0;
    e = cudaMemcpyToSymbol(g_sr_oob, &z, sizeof(z));
    return e != cudaSuccess ? e : kOobError;
}
#define SR_CHECK(i, n, site) ::sr::sr_check((long long)(i), (long long)(n), (site))
#define SR_OOB_COLLECT(e, st)                                                   \
    do {                                                                        \
        if ((e) == cudaSuccess) (e) = ::sr::sr_oob_collect((st), __BASE_FILE__); \
    } while (0)
#else
#define SR_CHECK(i, n, site) true
#define SR_OOB_COLLECT(e, st) \
    do {                      \
    } while (0)
#endif

// Offset subtracted from the sliding block in the NCC dot product.  Any
// constant leaves Eq. 3 unchanged (the fixed block is centred, so the sum of
// its centred values is zero); 128 keeps the products small for 0..255 data.
constexpr float kNccOffset = 128.0f;

// Variance below which a block counts as flat (NCC = 0).
constexpr float kFlatVar = 1e-6f;

// Storage type of the cost volumes (values of sr_vol_dtype).
enum VolType { kVolF32 = 0, kVolF16 = 1, kVolBF16 = 2 };
inline size_t vol_elem_bytes(int vt) { return vt == kVolF32 ? 4 : 2; }

// Loads of two adjacent stored costs, widened to FP32, and stores of eight.
__device__ __forceinline__ float2 load_pair(const float *p) {
    return *reinterpret_cast<const float2 *>(p);
}
__device__ __forceinline__ float2 load_pair(const __half *p) {
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
// (a bfloat16 is the upper half of the FP32 word of equal value)
__device__ __forceinline__ float2 load_pair(const __nv_bfloat16 *p) {
    const unsigned w = *reinterpret_cast<const unsigned *>(p);
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
// One stored cost, widened to FP32.
__device__ __forceinline__ float load_one(const float *p) { return *p; }
__device__ __forceinline__ float load_one(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float load_one(const __nv_bfloat16 *p) {
    return __uint_as_float((unsigned)*reinterpret_cast<const unsigned short *>(p) << 16);
}
__device__ __forceinline__ void store8(float *p, const float *v) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store8(__half *p, const float *v) {
    __half2 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(h);
}
__device__ __forceinline__ void store8(__nv_bfloat16 *p, const float *v) {
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(h);
}

// Stores of four costs: one 16-byte (FP32) or 8-byte (16-bit) store.
__device__ __forceinline__ void store4(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(__half *p, const float *v) {
    __half2 h[2] = {__floats2half2_rn(v[0], v[1]), __floats2half2_rn(v[2], v[3])};
    *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(h);
}
__device__ __forceinline__ void store4(__nv_bfloat16 *p, const float *v) {
    __nv_bfloat162 h[2] = {__floats2bfloat162_rn(v[0], v[1]), __floats2bfloat162_rn(v[2], v[3])};
    *reinterpret_cast<uint2 *>(p) = *reinterpret_cast<const uint2 *>(h);
}

// Sec. II-A row shift of image row v, s(v) = alpha0 + alpha1 v - delta: the
// plane of Eq. 2, evaluated once per image row in FP64 (a row's shift enters
// the warp as its integer part and fraction, and the post-processing of Sec.
// II-C adds it back).
__host__ __device__ __forceinline__ double row_shift(double alpha0, double alpha1, double delta,
                                                     int v) {
    return alpha0 + alpha1 * (double)v - delta;
}
// s split into two floats, hi = s rounded to float and lo = the rest rounded
// to float, so that the per-pixel post-processing runs in FP32.
__device__ __forceinline__ float2 split_shift(double s) {
    const float hi = __double2float_rn(s);
    return make_float2(hi, __double2float_rn(s - (double)hi));
}
// Sec. II-C: full disparity = subpixel residual disparity + s(v), from the
// split shift of the pixel's row.
__device__ __forceinline__ float post_disp(float ds, float2 sh) { return (ds + sh.x) + sh.y; }

// Supported compile-time parameter sets.
bool ncc_supported(int D, int ncc_r);
bool agg_supported(int D, int agg_r);

// Sec. II-A perspective transformation: rw[v][x] = i_r(x - s(v), v),
// s(v) = alpha0 + alpha1*v - delta, linear in x, clamp-to-edge.
cudaError_t launch_warp(const uint8_t *right, int pitch, int W, int H, double alpha0,
                        double alpha1, double delta, float *rw, cudaStream_t st);

// Eqs. 4-5 block statistics, for block centres on an extended range (the
// sliding block of the target volume is centred up to u+D-1, that of the
// reference volume down to u-(D-1)).  mu_l, inv_l: [H][W+D-1] for centres x in
// [0, W+D-1); mu_r, inv_r: [H][W+D-1] for centres x in [-(D-1), W) stored at
// x+D-1.  inv = 1/(n*sigma), 0 for a flat block.
cudaError_t launch_stats(const uint8_t *left, int pitch, const float *rw, int W, int H, int D,
                         int ncc_r, float *mu_l, float *inv_l, float *mu_r, float *inv_r,
                         cudaStream_t st);

// launch_warp and launch_stats in one kernel (the same values): the warped
// image rw and the four statistics arrays, and the split row shift
// rowsh[v] = split_shift(s(v + row0)) of every row (for the post-processing).
// row0: image row of the first row of left/right; the rows of a band of a
// larger frame take the plane of their rows in that frame.
cudaError_t launch_prep(const uint8_t *left, const uint8_t *right, int pitch, int W, int H, int D,
                        int ncc_r, double alpha0, double alpha1, double delta, int row0,
                        float *rw, float *mu_l, float *inv_l, float *mu_r, float *inv_r,
                        float2 *rowsh, cudaStream_t st);

// Eq. 3 cost volume [H][Wo][D], stored as vt (VolType; FP32 arithmetic,
// rounded to nearest on store).  target = false: reference volume
// c(u,v,d) = NCC(left block u, warped-target block u-d); target = true:
// target volume c(u,v,d) = NCC(left block u+d, warped-target block u).
//   range (nullable): per 32 x 4 tile, the disparities {lo, hi} that some
//   reader of the tile needs; chunks of disparities outside are not computed
//   Wo: output columns, W (0) or, for the reference volume only, the
//   extended W + D - 1, which holds the target volume too: target
//   c(u,v,d) = extended c(u+d,v,d) (entries with u - d >= W are not used)
cudaError_t launch_ncc(bool target, const uint8_t *left, int pitch, const float *rw,
                       const float *mu_l, const float *inv_l, const float *mu_r,
                       const float *inv_r, int W, int H, int D, int ncc_r, void *vol, int vt,
                       cudaStream_t st, const int2 *range = nullptr, int Wo = 0);

constexpr int kNslMaxSeg = 128;   // longest row segment of launch_ncc_sl
constexpr int kNslResident = 3;   // its CTAs per SM (launch bound)
constexpr int kNslThreads = 128;  // its threads per CTA
constexpr int kNslU = 4, kNslDB = 8;   // columns and disparities per thread

// Eq. 3 reference volume [H][Wo][D] (Wo = W or the extended W + D - 1)
// from exact integer window sums (k_ncc_sl.cuh): the left and right images
// and the plane, not the warped image; inv_l, inv_r are launch_prep's
// statistics (rows of W + D - 1).  A CTA walks a segment of seg image rows;
// segments start at the frame's rows that are multiples of seg, row0 being
// the frame row of the image's first row (a band's), and the costs' last
// bits depend on seg (ncc_segment gives the one every call on a frame
// size uses).  seg in 1..128.
cudaError_t launch_ncc_sl(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int D, int ncc_r, int row0, double alpha0, double alpha1, double delta,
                          const float *inv_l, const float *inv_r, void *vol, int vt, int Wo,
                          int seg, cudaStream_t st);
// Segment length of launch_ncc_sl for a W x H frame (a function of the frame
// size, D, the NCC radius, the volume type and the device only, so that a
// frame, its bands and a batch pair of that size use the same segments);
// the environment variable SR_NCC_SEG (1..128) overrides it.
int ncc_segment(int W, int H, int D, int ncc_r, int vt);

// Overlap of sr_match's kernels by programmatic dependent launch: the two
// aggregations are launched as programmatic dependents, so each starts
// while its predecessor drains (once every CTA of the predecessor has
// triggered).  The NCC kernel triggers at its start.  The target-view
// aggregation's first cost-row copy waits for the NCC grid (thread 0,
// griddepcontrol.wait) and its CTAs trigger only after that wait, so the
// reference view starts only once the NCC volume is complete; the reference
// view then runs its main loop and waits for the target-view grid (its
// labels) only before the L-R check of its epilogue.
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Bounded-wait settings of the aggregation kernel.  err (nullable) receives 1
// when a wait for a cost-row copy runs out after wait_cycles SM clocks;
// withhold_last = 1 withholds the copy of the last source row of every tile
// (a test of the timeout path), 0 in normal use.
struct AggDebug {
    int *err = nullptr;
    long long wait_cycles = 2000000000LL;   // ~1 s at 2 GHz
    int withhold_last = 0;
    int pdl = 0;   // launch as a programmatic dependent (see pdl_trigger)
};


// Restricted search (the paper's Sec. IV plan): pixel p searches only
// [max(0, c - radius), min(dfull - 1, c + radius)] around its centre c
// (centre[v*W+u], or centre_const when centre is null), clamped to 0..dfull-1.
// radius < 0: the full search 0..D-1.  band (nullable): per 32 x 4 tile, the
// first disparity of the band kernel's 16-wide slice (-1: the tile needs the
// full-D kernel); the full-D kernel skips tiles with band >= 0.
// Eq. 11 L-R check and Sec. II-C post-processing fused into the epilogue of
// the reference-view aggregation (disp != nullptr): the target labels lbl_r
// must be complete before that kernel starts.  The arithmetic is that of
// launch_lrc_post.
struct AggPost {
    const int16_t *lbl_r = nullptr;
    float *disp = nullptr;           // full disparity, NaN where rejected
    int16_t *wta = nullptr;          // optional copy of the reference labels
    const float2 *rowsh = nullptr;   // split row shift per row (launch_prep)
    float lr_thresh = 0.0f;
};
struct AggWin {
    const int16_t *centre = nullptr;
    int centre_const = 0;
    int radius = -1;
    int dfull = 0;
    const int *band = nullptr;
    AggPost post;                    // fused L-R check (full search only)
};
constexpr int kBandD = 16;        // disparities per band-kernel slice
constexpr int kAggTileX = 32, kAggTileY = 4;   // aggregation tile (pixels)

// Eqs. 8-10 bilateral aggregation fused with WTA (Sec. II-B-3) and, for the
// reference view, the Eq. 12 parabola.  Guide: the left image (uint8, when
// guide_u8 != nullptr) or the warped target (float).  Writes lbl [H][W]
// int16, dsub [H][W] float (nullable) and, for inspection, the normalised
// aggregated volume agg [H][W][D] (nullable).  vpitch: pixels per row of
// the volume (0: W; W + D - 1 for the extended reference volume).
// dbg.pdl: launch as a programmatic dependent of the target view; the fused
// L-R check waits for it (see pdl_trigger).
cudaError_t launch_agg(const void *vol, int vt, const uint8_t *guide_u8, int pitch,
                       const float *guide_f32, int W, int H, int D, int agg_r, float gamma_d,
                       float gamma_r, int16_t *lbl, float *dsub, float *agg,
                       const AggDebug &dbg, cudaStream_t st, const AggWin &win = AggWin(),
                       int vpitch = 0);

// The target view's aggregation read from the extended reference volume
// (launch_ncc with Wo = W + D - 1): pixel u at disparity d takes column
// u + d, through the 2-D tensor map tmap of encode_shear_map.  Guide: the
// warped target.  Writes lbl [H][W] and, for inspection, agg (nullable).
// dbg.pdl: launch as a programmatic dependent of the NCC kernel (see
// pdl_trigger).
cudaError_t launch_agg_shear(const void *tmap, int vt, const float *guide_f32, int W, int H,
                             int D, int agg_r, float gamma_d, float gamma_r, int16_t *lbl,
                             float *agg, const AggDebug &dbg, cudaStream_t st);
// The tensor map launch_agg_shear reads: the extended volume volx
// [H][W+D-1][D] viewed as [H*(W+D-1)][D], box of the sheared kernel's chunk
// (16 or 32 disparities x the pixels a row needs), zeros outside.  tmap:
// 64-byte aligned storage of a CUtensorMap (128 bytes).  False when the
// driver refuses the map or the parameters have no sheared kernel.
bool encode_shear_map(void *tmap, const void *volx, int vt, int W, int H, int D, int agg_r);

// The band kernel of the restricted search: tiles with band >= 0 aggregate
// the kBandD disparities [band, band + kBandD) of their pixels, read through
// the 2-D tensor map tmap (a CUtensorMap over the volume viewed as
// [H*W][D], box kBandD x (32 + 2 agg_r)); other tiles return at once.
cudaError_t launch_agg_band(const void *tmap, int vt, const uint8_t *guide_u8, int pitch,
                            const float *guide_f32, int W, int H, int agg_r, float gamma_d,
                            float gamma_r, int16_t *lbl, float *dsub, const AggDebug &dbg,
                            const AggWin &win, cudaStream_t st);
// Per-tile bands of the restricted search (32 x 4 tiles, see AggWin):
// band[t] = the aligned start of a kBandD slice holding every window of the
// tile (align: 16 bytes of the stored type), or -1.
cudaError_t launch_tile_bands(const AggWin &win, int W, int H, int align, int *band,
                              cudaStream_t st);
// The NCC range of every 32 x 4 tile under the restricted search: the union
// of the disparity slices of the aggregation tiles whose windows (radius
// agg_r) reach it, [0, D-1] when one of them needs all D.
cudaError_t launch_ncc_ranges(const int *band, int W, int H, int D, int agg_r, int2 *range,
                              cudaStream_t st);

// Eq. 11 check with tolerance, then Sec. II-C post-processing with the split
// row shifts rowsh [H] of launch_prep.
cudaError_t launch_lrc_post(const int16_t *lbl_l, const int16_t *lbl_r, const float *dsub, int W,
                            int H, const float2 *rowsh, float lr_thresh, float *disp,
                            int16_t *wta_out, cudaStream_t st);

// Sec. II-D reconstruction, three planes X, Y, Z of [H][W].
// selftest (bounds-checked builds): one thread evaluates a failing check
// (site 399) with no memory access.
cudaError_t launch_xyz(const float *disp, int W, int H, double f_px, double baseline, double u0,
                       double v0, float *xyz, cudaStream_t st, bool selftest = false);

// Adjoint of L = sum_{dstar >= 0} c_agg(p, dstar[p]) (Eq. 8 over Eq. 3 on the
// Sec. II-A warp) with respect to alpha and the images; rw, the block
// statistics and cost (the FP32 reference volume [H][W][D]) must hold the
// warp, Eqs. 4-5 and Eq. 3 at (alpha0, alpha1, delta).
//   wsum [H*W], partial [grad_partial_count(W, H) * 3] doubles: scratch
//   grw, gl, gr: [H*W] FP32 or null (gr needs grw); out3 = {L, dL/dalpha0, dL/dalpha1}
size_t grad_partial_count(int W, int H);
cudaError_t launch_grad(const uint8_t *left, const uint8_t *right, int pitch, int W, int H, int D,
                        int ncc_r, int agg_r, float gamma_d, float gamma_r, double alpha0,
                        double alpha1, double delta, const float *rw, const float *mu_l,
                        const float *inv_l, const float *mu_r, const float *inv_r,
                        const float *cost, const int16_t *dstar, float *wsum, float *grw,
                        float *gl, float *gr, double *partial, double *out3, cudaStream_t st);

// Sec. II-A road-plane fitting from a full-disparity map [H][W] (NaN =
// rejected).  launch_fit_count: per hypothesis h, the line through pixels
// pairs[2h], pairs[2h+1] (model[h], has_model[h]) and its inlier count
// counts[h] (|d - (a0 + a1 v)| <= tau, single precision).  launch_fit_ls:
// out5 = FP64 {n, sum v, sum v^2, sum d, sum v d} over the inliers of (a0, a1).
// launch_roll_sums: out9 = FP64 normal-equation sums {n, su, sv, suu, suv,
// svv, sd, sud, svd} over the valid pixels of [u_lo, u_hi) x [v_lo, v_hi).
// partial: scratch of fit_blocks(items) * 9 doubles.
int fit_blocks(long long items);
cudaError_t launch_fit_count(const float *disp, int W, int H, const int *pairs, int n, float tau,
                             float2 *model, int *has_model, int *counts, cudaStream_t st);
cudaError_t launch_fit_ls(const float *disp, int W, int H, float a0, float a1, float tau,
                          double *partial, double *out5, cudaStream_t st);
cudaError_t launch_roll_sums(const float *disp, int W, int u_lo, int v_lo, int u_hi, int v_hi,
                             double *partial, double *out9, cudaStream_t st);

__host__ __device__ inline int clampi(int x, int lo, int hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

// One stereo pair of a batch: its inputs, outputs and scratch (device
// pointers) and plane.  Batched kernels read an array of these and walk a flat
// list of (pair, tile) work items; tiles of pair p occupy
// [start[p], start[p+1]) of that list.
struct PairDesc {
    int W, H, pitch;
    const uint8_t *left, *right;
    double alpha0, alpha1, delta;
    float *disp;
    int16_t *wta;                 // nullable
    float *rw, *mu_l, *inv_l, *mu_r, *inv_r, *dsub;
    float2 *rowsh;                // [H] split row shifts
    void *vol_l, *vol_r;
    int16_t *lbl_l, *lbl_r;
};

// Pair owning flat work item t (start[] ascending, start[0] = 0), searched
// forward from a previous answer p0 <= the result (a persistent CTA's items
// only grow, so this is usually zero or one step).
__device__ __forceinline__ int find_pair(const int *start, int n, int t, int p0 = 0) {
    int p = p0;
    while (p + 1 < n && start[p + 1] <= t) ++p;
    return p;
}

// Copies start[0..n] into shared memory when it fits (kStartSmem ints), for
// the persistent kernels' pair search; returns the array to search.
constexpr int kStartSmem = 256;
__device__ __forceinline__ const int *stage_start(int *s_start, const int *start, int n) {
    if (n + 1 > kStartSmem) return start;
    for (int i = threadIdx.x + threadIdx.y * blockDim.x; i <= n; i += blockDim.x * blockDim.y)
        s_start[i] = start[i];
    __syncthreads();
    return s_start;
}

// Tiles of each batched stage (tile sizes of the kernels below).
constexpr int kPixTX = 32, kPixTY = 8;    // per-pixel stages (warp, stats, L-R + post)
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Batched stages: one persistent launch each over all pairs' tiles.
//   starts: device [n+1] prefix arrays per stage (see sr_batch.cu)
cudaError_t launch_warp_batch(const PairDesc *pairs, const int *start, int n, int grid,
                              cudaStream_t st);
cudaError_t launch_stats_batch(const PairDesc *pairs, const int *start, int n, int D, int ncc_r,
                               int grid, cudaStream_t st);
//   next: nullable device counter (zeroed before the launch); when given,
//   CTAs take work items in order from it instead of striding
cudaError_t launch_ncc_batch(bool target, const PairDesc *pairs, const int *start, int n, int D,
                             int ncc_r, int vt, int grid, int *next, cudaStream_t st);
cudaError_t launch_agg_batch(bool target, const PairDesc *pairs, const int *start, int n, int D,
                             int agg_r, int vt, float gamma_d, float gamma_r, const AggDebug &dbg,
                             int grid, int *next, cudaStream_t st);
cudaError_t launch_lrc_post_batch(const PairDesc *pairs, const int *start, int n, float lr_thresh,
                                  int grid, cudaStream_t st);
// Resident CTAs per SM of the batched NCC / aggregation kernels (for grid sizing).
int ncc_batch_occupancy(int D, int ncc_r, int vt);
int agg_batch_occupancy(int D, int agg_r, int vt);

}  // namespace sr
