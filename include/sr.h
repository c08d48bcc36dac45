/*
 * sr.h -- C ABI of the GB300 road-surface stereo library (libsr.so).
 *
 * Method: Fan et al., "Real-Time Stereo Vision for Road Surface 3-D
 * Reconstruction" (arXiv 1807.07433), Fig. 1 pipeline:
 *   perspective transformation of the target image (Sec. II-A, Eq. 2)
 *   -> block NCC costs in a reference and a target cost volume (Eqs. 3-5,
 *      Sec. II-B-1)
 *   -> bilateral cost aggregation (Eqs. 8-10)
 *   -> winner-take-all on both volumes (Sec. II-B-3)
 *   -> left-right consistency check (Eq. 11) and parabola subpixel
 *      refinement (Eq. 12)
 *   -> post-processing back to full disparity (Sec. II-C)
 *   -> 3-D reconstruction (Sec. II-D).
 *
 * Conventions shared by every entry point:
 *   - Images are 8-bit grayscale, row-major, W columns by H rows.  The left
 *     image is the reference view, the right image the target view.
 *   - Pointers named d_* are CUDA device pointers owned by the caller; h_*
 *     are host pointers owned by the caller.  The library never frees or
 *     retains a caller pointer beyond the call (or, for asynchronous calls,
 *     beyond the completion of the work queued on the context's stream).
 *   - All GPU work is queued asynchronously on the stream given to
 *     sr_create (a cudaStream_t passed as void*; NULL = legacy default
 *     stream).  Functions that write host memory synchronise that stream.
 *   - No function aborts or throws.  Every function returns an sr_status;
 *     sr_status_str() names it.  A CUDA error is reported as SR_ERR_CUDA;
 *     the text of the last CUDA error of a context is kept and returned by
 *     sr_last_error().  Nothing is printed unless the environment sets
 *     SR_LOG_LEVEL (1: errors and device timeouts on stderr; 2: also
 *     context creation and the batch autotuner's choices).
 *   - The API calls and the four stages of sr_match push NVTX ranges named
 *     after them (visible in NVTX-aware profilers; no cost without one).
 *   - Disparities: the search covers residual disparities 0..D-1 in the
 *     transformed (warped) domain; full disparity = residual + alpha0 +
 *     alpha1*v - delta (Sec. II-C).
 *   - The library is single-GPU: a context lives on the device that was
 *     current when it was created, and every call must be made with that
 *     device current.
 */
#ifndef SR_H
#define SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SR_OK = 0,
    SR_ERR_INVALID_ARG = 1,   /* null pointer, bad size or pitch, ... */
    SR_ERR_UNSUPPORTED = 2,   /* parameter outside the compiled kernel set */
    SR_ERR_OOM = 3,           /* device or host allocation failed */
    SR_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    SR_ERR_STATE = 5,         /* call out of order (e.g. no camera set) */
    SR_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    SR_ERR_BOUNDS = 7         /* bounds-checked build: an index fell outside its
                                 buffer (see sr_bounds_report) */
} sr_status;

/* Storage type of the staged cost volumes.  All arithmetic is FP32: NCC
 * costs are computed in FP32 and rounded to nearest when stored; the
 * aggregation widens them back to FP32 and accumulates in FP32. */
typedef enum { SR_VOL_F32 = 0, SR_VOL_F16 = 1, SR_VOL_BF16 = 2 } sr_vol_dtype;

/* Method parameters, fixed for the lifetime of a context.
 *   width, height  image size W x H, 1..16384 each.
 *   max_disp       D, residual disparities searched, 0..D-1 (Sec. II-B-3);
 *                  supported: 16, 32, 64.
 *   ncc_radius     NCC block radius (the rho-script of Eq. 3), block
 *                  (2r+1)^2; supported 1..5.
 *   agg_radius     bilateral window radius (rho of Eq. 8); supported 1..7.
 *   gamma_d        Eq. 9 spatial constant, > 0 (exp(-r^2/gamma_d^2)).
 *   gamma_r        Eq. 10 intensity constant on the 0..255 scale, > 0.
 *   lr_thresh      tolerance of the Eq. 11 consistency check in pixels,
 *                  >= 0 (Eq. 11 itself is 0).
 *   vol_dtype      storage of the staged cost volumes (see sr_vol_dtype).
 */
typedef struct {
    int width, height;
    int max_disp;
    int ncc_radius;
    int agg_radius;
    float gamma_d, gamma_r;
    float lr_thresh;
    sr_vol_dtype vol_dtype;
} sr_params;

typedef struct sr_ctx sr_ctx;   /* opaque; owns only its device scratch */

/* Create a context on the current device.  cuda_stream is the cudaStream_t
 * all work is queued on (NULL = legacy default stream).  Allocates the
 * context's scratch: warped image, block statistics, the two cost volumes
 * and the per-pixel maps (about ((2*W + D)*H*D*e + 40*W*H) bytes, e = 4 bytes per
 * stored cost for SR_VOL_F32 and 2 for SR_VOL_F16 / SR_VOL_BF16).
 * Errors: SR_ERR_INVALID_ARG (null out, non-positive sizes or constants),
 * SR_ERR_UNSUPPORTED (D, radii outside the supported set), SR_ERR_OOM,
 * SR_ERR_CUDA.  On error *out is set to NULL. */
sr_status sr_create(const sr_params *params, void *cuda_stream, sr_ctx **out);

/* Release the context and its scratch (synchronises its stream first).
 * NULL is accepted and ignored. */
sr_status sr_destroy(sr_ctx *ctx);

/* Road-plane model of Eq. 2 and the offset of Sec. II-A: target row v is
 * shifted alpha0 + alpha1*v - delta pixels to the right before matching.
 * Units: alpha0 and delta in pixels, alpha1 in pixels per row.  All
 * finite values are accepted; the default is (0, 0, 0). */
sr_status sr_set_plane(sr_ctx *ctx, double alpha0, double alpha1, double delta);

/* Camera of Sec. II-D: focal length f_px (pixels), baseline (any length
 * unit, XYZ comes out in that unit) and principal point (u0, v0) in pixels.
 * Required before sr_reconstruct. */
sr_status sr_set_camera(sr_ctx *ctx, double f_px, double baseline, double u0, double v0);

/* Disparity estimation, Secs. II-A..II-C (the hot path).
 *   d_left, d_right  W x H uint8 images, row pitch pitch_bytes (>= W).
 *   d_disp           W x H float (dense, pitch W): full disparity of each
 *                    left pixel, NaN where the L-R check (Eq. 11) fails.
 *   d_wta_or_null    optional W x H int16 (dense): the integer WTA residual
 *                    disparity l_ref of the reference view.
 * The NCC cost (Eq. 3) is computed once, as the reference volume over
 * W + D - 1 columns; the target view of Sec. II-B-1 reads it at column
 * u + d.  Its numerator is split into an exact integer part and the part
 * the row shifts' fractions carry (only the latter is rounded), with window
 * sums kept per segment of image rows, so the costs' last bits depend on
 * the segment length, a function of the frame size (SR_NCC_SEG overrides
 * it).  Four kernels: prep, ncc, agg_tgt, agg_ref; the last one also
 * runs the L-R check and the post-processing on its WTA labels.  The first
 * call builds the tensor map of that read.  Asynchronous on the context's
 * stream.  Errors: SR_ERR_INVALID_ARG for null images/output or pitch < W,
 * SR_ERR_CUDA for a failed launch or a driver that refuses the tensor map. */
sr_status sr_match(sr_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right, int pitch_bytes,
                   float *d_disp, int16_t *d_wta_or_null);

/* One band of rows of sr_match's result: the disparities of image rows
 * [y0, y1) of the W x H frame the context was created for, equal bit for bit
 * to those rows of sr_match on the whole frame.  Every step of the path is
 * row-local up to a window: an NCC block (Eq. 3) reaches ncc_radius rows and
 * a bilateral window (Eq. 8) agg_radius rows, so a band needs only halo rows
 * of both images, r0 .. r1 - 1 as sr_band_rows gives them: r1 = min(H, y1 +
 * h), h = ncc_radius + agg_radius, and r0 <= y0 - h (or 0), back to the first
 * row of the NCC kernel's row segment that holds row y0 - agg_radius, less
 * ncc_radius (the NCC kernel keeps window sums per segment of image rows, and
 * their rounding starts at the segment's first row).  The band takes the
 * plane of its rows in the frame (row v shifted by alpha0 + alpha1*v - delta,
 * v counted from the frame's first row).  This is the row partition of a
 * frame over several GPUs: each holds its band and halo rows, and the bands
 * need no exchange.
 *   d_left_rows, d_right_rows  image rows r0..r1-1 (pointers to row r0),
 *                              row pitch pitch_bytes (>= W)
 *   y0, y1                     0 <= y0 < y1 <= H
 *   d_disp_rows                (y1 - y0) x W floats, dense: rows y0..y1-1
 *                              of sr_match's d_disp
 *   d_wta_rows_or_null         optional (y1 - y0) x W int16: the same rows
 *                              of sr_match's d_wta_or_null
 * The halo rows are matched too (and discarded), so a band costs its rows
 * plus up to 2h rows and one NCC row segment (sr_band_rows).  Uses the
 * context's scratch (sr_get_buffer reports SR_ERR_STATE afterwards); the first call allocates 6*W*H bytes of band
 * output and builds a tensor map for bands of r1 - r0 rows (rebuilt when
 * that count changes).  Asynchronous.  Errors: SR_ERR_INVALID_ARG,
 * SR_ERR_OOM, SR_ERR_CUDA. */
sr_status sr_match_rows(sr_ctx *ctx, const uint8_t *d_left_rows, const uint8_t *d_right_rows,
                        int pitch_bytes, int y0, int y1, float *d_disp_rows,
                        int16_t *d_wta_rows_or_null);

/* The image rows [*r0, *r1) that sr_match_rows reads for output rows
 * [y0, y1) (see there).  Host only, no GPU work.  Errors: SR_ERR_INVALID_ARG
 * for null arguments or rows outside 0 <= y0 < y1 <= H. */
sr_status sr_band_rows(const sr_ctx *ctx, int y0, int y1, int *r0, int *r1);

/* Restricted search: sr_match with every pixel of both views searching only
 * the window [c - radius, c + radius] (clamped to 0..D-1) around its centre
 * c, the plan of the paper's Sec. IV (filter only the space around previously
 * calculated disparities).  WTA (Sec. II-B-3) and Eq. 12 run over the window,
 * with its ends in the role of 0 and D-1 (no parabola at an end); the
 * aggregated costs themselves are those of sr_match, which this call equals
 * when radius >= D-1.
 *   d_centre   W x H int16 residual disparities (e.g. the WTA map of the
 *              previous frame, d_wta_or_null of sr_match), or NULL for the
 *              plane hypothesis: every pixel centred at round(delta)
 *   radius     0 <= radius < D
 * The aggregation runs only where needed: each 32 x 4 tile whose windows fit
 * one 16-disparity slice aggregates just that slice (read through a TMA
 * tensor map), the others aggregate all D; NCC costs are computed only in
 * the 32-disparity chunks some tile reads.  sr_get_buffer's cost volumes are
 * therefore partial after this call.  Asynchronous; the first call
 * allocates three ints per tile, zeroes the cost volumes and builds the
 * tensor maps.  Errors: SR_ERR_INVALID_ARG, SR_ERR_CUDA. */
sr_status sr_match_restricted(sr_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                              int pitch_bytes, const int16_t *d_centre, int radius,
                              float *d_disp, int16_t *d_wta_or_null);

/* sr_match with host buffers: copies h_left/h_right (W x H, dense) to the
 * device, runs sr_match, copies the disparity map back into h_disp (W x H
 * float) and synchronises the stream.  Pinned host memory makes the copies
 * asynchronous; pageable memory works but is slower.  Uses staging buffers
 * owned by the context (allocated on first use). */
sr_status sr_match_host(sr_ctx *ctx, const uint8_t *h_left, const uint8_t *h_right,
                        float *h_disp);

/* Streaming form of sr_match_host for a sequence of frames (video): queues
 * the upload of h_left/h_right, the match and the download of the disparity
 * map into h_disp, and returns without waiting for them.  Uploads and
 * downloads run on two copy streams the context creates on first use, so
 * that the next frame's upload and the previous frame's download overlap
 * this frame's kernels (which run on the context's stream, in call order).
 * At most two frames are in flight: when the call returns, every frame
 * queued two or more calls earlier has finished (its disparity map is in its
 * h_disp and its host images may be reused); sr_synchronize finishes all of
 * them.  Host buffers should be pinned (cudaHostAlloc / cudaHostRegister)
 * for the copies to overlap.  Results are those of sr_match_host.  Errors as
 * sr_match_host; a device-side timeout of an earlier frame is reported by
 * the call that waits for it. */
sr_status sr_match_host_async(sr_ctx *ctx, const uint8_t *h_left, const uint8_t *h_right,
                              float *h_disp);

/* sr_match for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this entry point concerns only memory ownership.)
 * Some callers cannot call cudaMalloc -- a host that fixes the library's
 * device-memory budget at start-up and forbids allocation afterwards, a
 * plug-in whose host owns the device allocator, a real-time loop that must
 * never wait on the allocator.  This call needs no context and allocates
 * nothing: the intermediates of the match live in one fixed device array of
 * 32 MiB inside libsr.so, which every GPU that loads the library holds until
 * the process exits.  Inputs, outputs and parameters have the meaning they
 * have for sr_create + sr_set_plane + sr_match; d_disp receives the same
 * values sr_match writes.
 *   Size limit: with A(b) = b rounded up to a multiple of 256 and e the
 *   bytes of one stored cost (4 for SR_VOL_F32, 2 for SR_VOL_F16/BF16),
 *     2*A(4*W*H) + 4*A(4*H*(W+D-1)) + A(e*H*(W+D-1)*D) + 2*A(2*W*H) + A(8*H)
 *       <= 32 MiB
 *   (e.g. 640x480 at D = 16, 400x225 at D = 64 with FP32 volumes); larger
 *   frames are rejected with SR_ERR_UNSUPPORTED before any GPU work.
 *   The first call in a CUDA context (the device's primary context, or a
 *   driver-API context made current by the caller) looks up the array's
 *   device address with cudaGetSymbolAddress, with that context current,
 *   and keeps it under the context's unique ID; a context created later
 *   (e.g. after cudaDeviceReset) gets its own look-up.  Make the first call
 *   in each context before any stream capture.
 *   Every call reuses the same array and leaves its contents behind; nothing
 *   in it needs to start at zero.  Calls whose GPU work overlaps (other
 *   streams, or other threads without ordering) race on the array.
 *   Bounded device-side waits that run out set a sticky timeout word (also
 *   a fixed device variable, not an allocation); the call itself returns
 *   before the GPU work ends, so a timeout is reported by
 *   sr_noalloc_status, not by this call.
 * Asynchronous on cuda_stream (NULL = legacy default stream).  Errors:
 * SR_ERR_INVALID_ARG, SR_ERR_UNSUPPORTED (parameters or size), SR_ERR_CUDA. */
sr_status sr_match_noalloc(const sr_params *params, double alpha0, double alpha1, double delta,
                           const uint8_t *d_left, const uint8_t *d_right, int pitch_bytes,
                           float *d_disp, int16_t *d_wta_or_null, void *cuda_stream);

/* Status of the sr_match_noalloc calls made in the current CUDA context:
 * synchronises cuda_stream, then returns SR_ERR_TIMEOUT if a bounded wait of
 * any such call ran out since the last sr_noalloc_status (the results of
 * that call are undefined), clearing the condition, else SR_OK.  Allocates
 * nothing (two 4-byte copies between a host variable and the device word).
 * Errors: SR_ERR_CUDA. */
sr_status sr_noalloc_status(void *cuda_stream);

/* Bounds-checked builds (libsr_check.so, compiled with SR_BOUNDS_CHECK).
 * Every checked index of the match-path kernels -- warp and block statistics
 * (Sec. II-A, Eqs. 4-5), NCC (Eq. 3), aggregation (Eqs. 8-12, including its
 * cost-row copies and shared-memory tiles), L-R check and post-processing
 * (Eq. 11, Sec. II-C), reconstruction (Sec. II-D) -- that falls outside its
 * buffer is recorded, the first per launch (site number, index, source
 * file), and its access is skipped; the call that launched the kernel then
 * returns SR_ERR_BOUNDS.  Launches inside stream capture are checked at the
 * next plain launch of the same kernel file.  The arithmetic is that of the
 * release build, so results are bit-identical where no index is out of range.
 *
 * sr_bounds_report copies the first offence recorded since the last report
 * into *site, *index and unit (unit_len bytes, NUL-terminated), the number
 * of offences into *count, and clears the record; any pointer may be NULL.
 * Returns SR_OK when none was recorded, SR_ERR_BOUNDS when one was, and
 * SR_ERR_UNSUPPORTED in a release build.  Site numbers: 1xx NCC, 2xx
 * aggregation, 3xx per-pixel kernels.  Thread-safe; process-wide. */
sr_status sr_bounds_report(int *site, long long *index, char *unit, int unit_len,
                           long long *count);

/* One stereo pair of a batch (all pointers device pointers owned by the
 * caller; layouts as for sr_match). */
typedef struct {
    int width, height;          /* 1..16384 each */
    int pitch_bytes;            /* row pitch of both images, >= width */
    const uint8_t *d_left, *d_right;
    double alpha0, alpha1, delta;   /* Eq. 2 plane and offset of this pair */
    float *d_disp;              /* width x height, dense */
    int16_t *d_wta_or_null;     /* optional, width x height */
} sr_pair_desc;

/* The pipeline of sr_match for n pairs of any sizes in one call, captured
 * into a CUDA graph that later calls replay.  By default each stage is one
 * persistent launch over the flat list of (pair, tile) work items of the
 * whole batch; sr_set_batch_schedule and sr_set_autotune select among
 * other schedules.  The context supplies D, the radii, gamma_d, gamma_r,
 * lr_thresh, vol_dtype and the stream; its width and height are not used.
 * Scratch is held by the context and sized for the schedule that runs:
 * the per-pair schedules (4-7) run the pairs of one stream in order and give
 * each stream one slot sized for its largest pair (schedules 6-7: about
 * (W + D)*H*D*e + 40*W*H bytes, e as for sr_create; 4-5 add W*H*D*e for the
 * target volume), so scratch is bounded by the streams, not by n; the
 * persistent schedules (0-3) run all pairs at once and need one slot per
 * pair.  The autotuner skips a schedule whose scratch would not fit the free
 * device memory, and after its choice the pool shrinks to that schedule's
 * need.  Results are identical to n sr_match calls.  Asynchronous.
 * Errors: SR_ERR_INVALID_ARG (n < 1, a bad pair), SR_ERR_OOM, SR_ERR_CUDA. */
sr_status sr_match_batch(sr_ctx *ctx, int n, const sr_pair_desc *pairs);

/* Autotuning of sr_match_batch.  With enable != 0, the first batch of each
 * shape (multiset of image sizes, D, radii, volume type, GPU) times the
 * eight candidate schedules of sr_set_batch_schedule on the caller's data
 * and keeps the fastest.  cache_path (nullable) names a file of
 * one JSON object per line that stores the choices across processes (when
 * NULL, the path in the environment variable SR_TUNE_CACHE, if set);
 * unreadable lines are skipped (defaults used) and reported by
 * sr_last_error.  Disabled: grid factor 1, caller's order. */
sr_status sr_set_autotune(sr_ctx *ctx, int enable, const char *cache_path);

/* Fix the schedule of sr_match_batch instead of tuning it: 0-3 one
 * persistent launch per stage (bit 0: two waves of CTAs instead of one;
 * bit 1: largest pair first); 4 / 5 per-pair launches of the
 * descriptor-driven kernels on 4 / 8 streams of the graph, largest pair
 * first; 6 / 7 per-pair launches of the kernels of sr_match on 1 / 4 streams,
 * largest pair first (the graph holds the pairs' pointers and planes, and is
 * re-captured and updated in place when they change); -1 restores the
 * automatic choice.  SR_ERR_INVALID_ARG for other values. */
sr_status sr_set_batch_schedule(sr_ctx *ctx, int variant);

/* One-line JSON description of the schedule of the last sr_match_batch. */
sr_status sr_batch_info(sr_ctx *ctx, char *buf, size_t size);

/* 3-D reconstruction, Sec. II-D, for the left pixels of a full-disparity
 * map d_disp (W x H float, as written by sr_match).  d_xyz receives three
 * planes of W x H floats (X, then Y, then Z) in the camera frame of the
 * left camera: Z = f*B/d, X = (u-u0)*Z/f, Y = (v-v0)*Z/f; NaN where d is
 * NaN or not positive.  Asynchronous.  SR_ERR_STATE if no camera is set. */
sr_status sr_reconstruct(sr_ctx *ctx, const float *d_disp, float *d_xyz);

/* Road-plane fitting from a disparity map, Sec. II-A: the paper fits alpha
 * of Eq. 2 by least squares with RANSAC on reliable correspondences, and the
 * roll angle by fitting a plane to a near-field patch of the disparity map.
 * Here the correspondences are the valid pixels of a full-disparity map
 * (d_disp, W x H float as written by sr_match, NaN = rejected), so that the
 * plane of the next frame can come from this frame's result.
 *
 * sr_fit_alpha: RANSAC over n_hyp caller-drawn point pairs
 *   h_pairs[2h], h_pairs[2h+1] (pixel indices v*W+u, host memory;
 *   1 <= n_hyp <= 65536).  Hypothesis h is the line d = a0 + a1 v through its
 *   two points, computed in double and rounded to float; it has no model
 *   if a point is out of range or NaN, or both lie on one row.  Its inliers
 *   are the valid pixels with |d - (a0 + a1 v)| <= tau_px, decided in single
 *   precision (one fused multiply-add, then one subtraction).  The hypothesis
 *   with the most inliers wins (ties: the smallest h).  h_alpha (host
 *   double[2]) receives the least-squares line through its inliers
 *   (normal equations, FP64 sums).  Optional outputs: h_counts (int32[n_hyp],
 *   -1 for no model), h_best, h_n_inliers.  Synchronises the stream.
 *   SR_ERR_STATE if no hypothesis has a model or the inliers span one row.
 * sr_fit_roll: least-squares plane d = g0 + g1 u + g2 v over the valid
 *   pixels of the patch [u_lo, u_hi) x [v_lo, v_hi) (clipped to the image),
 *   h_gamma = (g0, g1, g2), *h_roll = atan(-g1 / g2) in radians, *h_n (nullable)
 *   the pixels used.  Synchronises the stream.  SR_ERR_INVALID_ARG for an
 *   empty patch, SR_ERR_STATE if the normal equations are singular. */
sr_status sr_fit_alpha(sr_ctx *ctx, const float *d_disp, int n_hyp, const int32_t *h_pairs,
                       float tau_px, double *h_alpha, int32_t *h_counts, int *h_best,
                       int *h_n_inliers);
sr_status sr_fit_roll(sr_ctx *ctx, const float *d_disp, int u_lo, int v_lo, int u_hi, int v_hi,
                      double *h_gamma, double *h_roll, int *h_n);

/* Gradient of the aggregated matching cost with respect to the road plane,
 * for refining alpha (Sec. II-A, Eq. 2) by gradient ascent.  The paper fits
 * alpha once from a disparity map (Sec. II-A) and has no gradient; this is
 * the adjoint of its own cost, by the chain rule through the warp (Sec.
 * II-A), the NCC (Eqs. 3-5) and the bilateral aggregation of the reference
 * volume (Eqs. 8-10, guide = left image):
 *   L(alpha) = sum over pixels p with d_dstar[p] >= 0 of c_agg(p, d_dstar[p]),
 * with the disparities d_dstar held fixed (the plane hypothesis is every
 * pixel at residual delta; the winning labels of sr_match are another set).
 * The warp and block statistics are recomputed at the context's current
 * plane (sr_set_plane), so the call does not depend on an earlier sr_match.
 *   d_left, d_right   8-bit images, pitch_bytes >= W, as for sr_match
 *   d_dstar           int16 [H][W] dense residual disparities; a value
 *                     outside 0..D-1 (e.g. -1) leaves the pixel out of L
 *   h_out3            host double[3]: L, dL/dalpha0, dL/dalpha1
 *   d_grad_left, d_grad_right
 *                     float [H][W] dense or NULL: dL/di_l and dL/di_r, the
 *                     images read as real values (FP32 atomics: the last
 *                     bits vary from run to run; L and dL/dalpha are summed
 *                     in FP64 in a fixed order and do not)
 * Arithmetic is FP32 per term with FP64 sums.  The objective is piecewise
 * smooth in alpha: it has kinks where a row shift alpha0 + alpha1 v - delta
 * crosses an integer.  Synchronises the context's stream (h_out3 is host
 * memory).  The context's scratch is reused (the buffers of the last
 * sr_match are no longer available to sr_get_buffer afterwards); the first
 * call allocates about 12*W*H bytes more, plus 4*W*H*D bytes for an FP32
 * cost volume when the context stores 16-bit volumes. */
sr_status sr_grad_plane(sr_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                        int pitch_bytes, const int16_t *d_dstar, double *h_out3,
                        float *d_grad_left, float *d_grad_right);

/* Intermediate arrays of the last sr_match, for inspection and tests.
 * which selects the array; its device layout and element type are fixed:
 *   SR_BUF_WARPED     float [H][W]        warped target i_r' (Sec. II-A)
 *   SR_BUF_MU_L       float [H][W]        block mean of i_l (Eq. 4)
 *   SR_BUF_INV_L      float [H][W]        1/(n*sigma_l), 0 for a flat block
 *   SR_BUF_MU_R       float [H][W]        block mean of i_r'
 *   SR_BUF_INV_R      float [H][W]        1/(n*sigma_r), 0 for a flat block
 *   SR_BUF_COST_L     float [H][W][D]     reference NCC volume (Eq. 3)
 *   SR_BUF_COST_R     float [H][W][D]     target NCC volume (after sr_match
 *                                          rebuilt on the host from the
 *                                          extended reference volume
 *                                          sr_match computes: target cost
 *                                          (u,v,d) = its column u + d)
 *   SR_BUF_AGG_L      float [H][W][D]     aggregated reference volume (Eq. 8),
 *   SR_BUF_AGG_R      float [H][W][D]     ... and target volume; these two are
 *                                          only written while the debug flag
 *                                          SR_DEBUG_KEEP_AGG is set
 *   SR_BUF_WTA_L      int16 [H][W]        l_ref
 *   SR_BUF_WTA_R      int16 [H][W]        l_tar
 *   SR_BUF_DSUB       float [H][W]        subpixel residual d^s (Eq. 12)
 * The array is copied (synchronously) into dst, a host or device pointer of
 * at least the array's size, which *bytes_inout gives on input and receives
 * on output.  Volumes stored in FP16/BF16 are widened to float.
 * Errors: SR_ERR_INVALID_ARG (unknown which, dst too small),
 * SR_ERR_STATE (array not produced, e.g. AGG without the debug flag). */
typedef enum {
    SR_BUF_WARPED = 0, SR_BUF_MU_L, SR_BUF_INV_L, SR_BUF_MU_R, SR_BUF_INV_R,
    SR_BUF_COST_L, SR_BUF_COST_R, SR_BUF_AGG_L, SR_BUF_AGG_R,
    SR_BUF_WTA_L, SR_BUF_WTA_R, SR_BUF_DSUB
} sr_buffer;
sr_status sr_get_buffer(sr_ctx *ctx, sr_buffer which, void *dst, size_t *bytes_inout);

/* Debug flags (bit set).  SR_DEBUG_KEEP_AGG makes sr_match also store both
 * aggregated volumes (allocated on first use, 2*W*H*D floats).
 * SR_DEBUG_WITHHOLD_ROW is fault injection for the timeout path: the
 * aggregation kernel withholds the copy of one cost row of every tile and
 * shortens its bounded wait to ~1 ms, so the wait runs out, the results are
 * garbage and the next synchronising call returns SR_ERR_TIMEOUT.  The GPU
 * stays usable. */
#define SR_DEBUG_KEEP_AGG 1
#define SR_DEBUG_WITHHOLD_ROW 2
#define SR_DEBUG_NO_BAND 4       /* sr_match_restricted: every tile runs the full-D kernel */
/* SR_DEBUG_BOUNDS_SELFTEST: in a bounds-checked build, each sr_reconstruct
 * records one offence at site 399 (index -1) without any memory access, so
 * that the call returns SR_ERR_BOUNDS and sr_bounds_report reports it; no
 * effect in a release build. */
#define SR_DEBUG_BOUNDS_SELFTEST 8
sr_status sr_set_debug(sr_ctx *ctx, int flags);

/* Wait for the context's queued work.  Device-side waits are bounded; when
 * one ran out since the last check this returns SR_ERR_TIMEOUT (and clears
 * the condition).  sr_match_host, sr_get_buffer and sr_stage_times check the
 * same condition after they synchronise. */
sr_status sr_synchronize(sr_ctx *ctx);

/* Per-stage timing.  While enabled, sr_match records a CUDA event before
 * and after each stage on the context's stream, in a ring that keeps the
 * events of the last 512 matches (created on the first enable; enabling
 * restarts the count).  Recording does not synchronise anything.
 * sr_stage_times synchronises the stream and writes, for the most recent
 * sr_match, the duration in milliseconds of each stage into ms[0..n) in the
 * order of sr_stage_names(); it returns the number of stages in *count.
 * sr_stage_times_history writes the stage durations of the most recent
 * min(max_matches, matches recorded, 512) matches, oldest first, stage s of
 * match k at ms[k * stages + s]; *count receives the number of matches.
 * Both return SR_ERR_STATE when no match has been recorded. */
sr_status sr_set_profiling(sr_ctx *ctx, int enable);
sr_status sr_stage_times(sr_ctx *ctx, float *ms, int n, int *count);
sr_status sr_stage_times_history(sr_ctx *ctx, float *ms, int max_matches, int *count);
const char *sr_stage_names(void);   /* comma-separated stage names */

/* Number of kernel launches one sr_match queues (for launch accounting). */
int sr_kernels_per_match(const sr_ctx *ctx);

const char *sr_status_str(sr_status s);
const char *sr_last_error(const sr_ctx *ctx);
const char *sr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SR_H */
