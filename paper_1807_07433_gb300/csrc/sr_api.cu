// sr_api.cu -- the C ABI of include/sr.h: context, argument checks, scratch
// ownership, stage sequencing on the caller's stream, timing and errors.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/sr.h"
#include "sr_ctx.cuh"

namespace sr {
cudaError_t launch_ncc_d16_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d16_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d16_f16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d16_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d16_bf16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d16_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d32_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d32_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d32_f16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d32_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d32_bf16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d32_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d64_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d64_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d64_f16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d64_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_ncc_d64_bf16(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range);
cudaError_t launch_agg_d64_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);

cudaError_t launch_aggw_d16_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d16_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d16_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d32_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d32_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d32_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d64_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d64_f16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggw_d64_bf16(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch);
cudaError_t launch_aggs_d16_f32(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d16_f16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d16_bf16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d32_f32(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d32_f16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d32_bf16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d64_f32(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d64_f16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
cudaError_t launch_aggs_d64_bf16(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st);
bool aggs_box_d16_f32(int agg_r, int *cw, int *bh);
bool aggs_box_d16_f16(int agg_r, int *cw, int *bh);
bool aggs_box_d16_bf16(int agg_r, int *cw, int *bh);
bool aggs_box_d32_f32(int agg_r, int *cw, int *bh);
bool aggs_box_d32_f16(int agg_r, int *cw, int *bh);
bool aggs_box_d32_bf16(int agg_r, int *cw, int *bh);
bool aggs_box_d64_f32(int agg_r, int *cw, int *bh);
bool aggs_box_d64_f16(int agg_r, int *cw, int *bh);
bool aggs_box_d64_bf16(int agg_r, int *cw, int *bh);
cudaError_t launch_agg_band_f32(const void *tmap, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, const AggDebug &dbg, const AggWin &win, cudaStream_t st);
cudaError_t launch_agg_band_f16(const void *tmap, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, const AggDebug &dbg, const AggWin &win, cudaStream_t st);
cudaError_t launch_agg_band_bf16(const void *tmap, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, const AggDebug &dbg, const AggWin &win, cudaStream_t st);

cudaError_t launch_ncc_batch_d16_f32(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d16_f32(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d16_f32(int);
int agg_occ_d16_f32(int);
cudaError_t launch_ncc_batch_d16_f16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d16_f16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d16_f16(int);
int agg_occ_d16_f16(int);
cudaError_t launch_ncc_batch_d16_bf16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d16_bf16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d16_bf16(int);
int agg_occ_d16_bf16(int);
cudaError_t launch_ncc_batch_d32_f32(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d32_f32(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d32_f32(int);
int agg_occ_d32_f32(int);
cudaError_t launch_ncc_batch_d32_f16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d32_f16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d32_f16(int);
int agg_occ_d32_f16(int);
cudaError_t launch_ncc_batch_d32_bf16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d32_bf16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d32_bf16(int);
int agg_occ_d32_bf16(int);
cudaError_t launch_ncc_batch_d64_f32(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d64_f32(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d64_f32(int);
int agg_occ_d64_f32(int);
cudaError_t launch_ncc_batch_d64_f16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d64_f16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d64_f16(int);
int agg_occ_d64_f16(int);
cudaError_t launch_ncc_batch_d64_bf16(bool, const PairDesc *, const int *, int, int, int, int *, cudaStream_t);
cudaError_t launch_agg_batch_d64_bf16(bool, const PairDesc *, const int *, int, int, float, float, const AggDebug &, int, int *, cudaStream_t);
int ncc_occ_d64_bf16(int);
int agg_occ_d64_bf16(int);

cudaError_t launch_ncc_sl_d16_f32(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d16_f32(int);
cudaError_t launch_ncc_sl_d16_f16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d16_f16(int);
cudaError_t launch_ncc_sl_d16_bf16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d16_bf16(int);
cudaError_t launch_ncc_sl_d32_f32(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d32_f32(int);
cudaError_t launch_ncc_sl_d32_f16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d32_f16(int);
cudaError_t launch_ncc_sl_d32_bf16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d32_bf16(int);
cudaError_t launch_ncc_sl_d64_f32(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d64_f32(int);
cudaError_t launch_ncc_sl_d64_f16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d64_f16(int);
cudaError_t launch_ncc_sl_d64_bf16(const uint8_t *, const uint8_t *, int, int, int, int, int, double, double, double, const float *, const float *, void *, int, int, cudaStream_t);
int ncc_sl_occ_d64_bf16(int);

bool ncc_supported(int D, int ncc_r) {
    return (D == 16 || D == 32 || D == 64) && ncc_r >= 1 && ncc_r <= 5;
}
bool agg_supported(int D, int agg_r) {
    return (D == 16 || D == 32 || D == 64) && agg_r >= 1 && agg_r <= 7;
}

#define SR_VT_DISPATCH(FN, D, vt, ...)                              \
    switch (vt) {                                                   \
        case kVolF32: return FN##_d##D##_f32(__VA_ARGS__);          \
        case kVolF16: return FN##_d##D##_f16(__VA_ARGS__);          \
        case kVolBF16: return FN##_d##D##_bf16(__VA_ARGS__);        \
        default: return cudaErrorInvalidValue;                      \
    }

cudaError_t launch_ncc(bool target, const uint8_t *left, int pitch, const float *rw,
                       const float *mu_l, const float *inv_l, const float *mu_r,
                       const float *inv_r, int W, int H, int D, int ncc_r, void *vol, int vt,
                       cudaStream_t st, const int2 *range, int Wo) {
    if (Wo <= 0) Wo = W;
    if (target && Wo != W) return cudaErrorInvalidValue;
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_ncc, 16, vt, target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r, vol, Wo, st, range)
        case 32: SR_VT_DISPATCH(launch_ncc, 32, vt, target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r, vol, Wo, st, range)
        case 64: SR_VT_DISPATCH(launch_ncc, 64, vt, target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r, vol, Wo, st, range)
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ncc_sl(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                          int D, int ncc_r, int row0, double alpha0, double alpha1, double delta,
                          const float *inv_l, const float *inv_r, void *vol, int vt, int Wo,
                          int seg, cudaStream_t st) {
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_ncc_sl, 16, vt, left, right, pitch, W, H, ncc_r, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st)
        case 32: SR_VT_DISPATCH(launch_ncc_sl, 32, vt, left, right, pitch, W, H, ncc_r, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st)
        case 64: SR_VT_DISPATCH(launch_ncc_sl, 64, vt, left, right, pitch, W, H, ncc_r, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st)
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_agg(const void *vol, int vt, const uint8_t *guide_u8, int pitch,
                       const float *guide_f32, int W, int H, int D, int agg_r, float gamma_d,
                       float gamma_r, int16_t *lbl, float *dsub, float *agg,
                       const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch) {
    const float log2e = 1.4426950408889634f;
    const float kd = log2e / (gamma_d * gamma_d), kr = log2e / (gamma_r * gamma_r);
    if (vpitch <= 0) vpitch = W;
    if (win.radius >= 0) {   // restricted search: the windowed kernels
        switch (D) {
            case 16: SR_VT_DISPATCH(launch_aggw, 16, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
            case 32: SR_VT_DISPATCH(launch_aggw, 32, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
            case 64: SR_VT_DISPATCH(launch_aggw, 64, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
            default: return cudaErrorInvalidValue;
        }
    }
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_agg, 16, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
        case 32: SR_VT_DISPATCH(launch_agg, 32, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
        case 64: SR_VT_DISPATCH(launch_agg, 64, vt, vol, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, agg, dbg, st, win, vpitch)
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_agg_shear(const void *tmap, int vt, const float *guide_f32, int W, int H,
                             int D, int agg_r, float gamma_d, float gamma_r, int16_t *lbl,
                             float *agg, const AggDebug &dbg, cudaStream_t st) {
    const float log2e = 1.4426950408889634f;
    const float kd = log2e / (gamma_d * gamma_d), kr = log2e / (gamma_r * gamma_r);
    const int vpitch = W + D - 1;
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_aggs, 16, vt, tmap, vpitch, guide_f32, W, H, agg_r, kd, kr, lbl, agg, dbg, st)
        case 32: SR_VT_DISPATCH(launch_aggs, 32, vt, tmap, vpitch, guide_f32, W, H, agg_r, kd, kr, lbl, agg, dbg, st)
        case 64: SR_VT_DISPATCH(launch_aggs, 64, vt, tmap, vpitch, guide_f32, W, H, agg_r, kd, kr, lbl, agg, dbg, st)
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_agg_band(const void *tmap, int vt, const uint8_t *guide_u8, int pitch,
                            const float *guide_f32, int W, int H, int agg_r, float gamma_d,
                            float gamma_r, int16_t *lbl, float *dsub, const AggDebug &dbg,
                            const AggWin &win, cudaStream_t st) {
    const float log2e = 1.4426950408889634f;
    const float kd = log2e / (gamma_d * gamma_d), kr = log2e / (gamma_r * gamma_r);
    switch (vt) {
        case kVolF32: return launch_agg_band_f32(tmap, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, dbg, win, st);
        case kVolF16: return launch_agg_band_f16(tmap, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, dbg, win, st);
        case kVolBF16: return launch_agg_band_bf16(tmap, guide_u8, pitch, guide_f32, W, H, agg_r, kd, kr, lbl, dsub, dbg, win, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ncc_batch(bool target, const PairDesc *pairs, const int *start, int n, int D,
                             int ncc_r, int vt, int grid, int *next, cudaStream_t st) {
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_ncc_batch, 16, vt, target, pairs, start, n, ncc_r, grid, next, st)
        case 32: SR_VT_DISPATCH(launch_ncc_batch, 32, vt, target, pairs, start, n, ncc_r, grid, next, st)
        case 64: SR_VT_DISPATCH(launch_ncc_batch, 64, vt, target, pairs, start, n, ncc_r, grid, next, st)
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_agg_batch(bool target, const PairDesc *pairs, const int *start, int n, int D,
                             int agg_r, int vt, float gamma_d, float gamma_r, const AggDebug &dbg,
                             int grid, int *next, cudaStream_t st) {
    const float log2e = 1.4426950408889634f;
    const float kd = log2e / (gamma_d * gamma_d), kr = log2e / (gamma_r * gamma_r);
    switch (D) {
        case 16: SR_VT_DISPATCH(launch_agg_batch, 16, vt, target, pairs, start, n, agg_r, kd, kr, dbg, grid, next, st)
        case 32: SR_VT_DISPATCH(launch_agg_batch, 32, vt, target, pairs, start, n, agg_r, kd, kr, dbg, grid, next, st)
        case 64: SR_VT_DISPATCH(launch_agg_batch, 64, vt, target, pairs, start, n, agg_r, kd, kr, dbg, grid, next, st)
        default: return cudaErrorInvalidValue;
    }
}

#define SR_OCC_DISPATCH(FN, D, vt, r)                     \
    switch (vt) {                                         \
        case kVolF32: return FN##_d##D##_f32(r);          \
        case kVolF16: return FN##_d##D##_f16(r);          \
        case kVolBF16: return FN##_d##D##_bf16(r);        \
        default: return 0;                                \
    }

int ncc_batch_occupancy(int D, int ncc_r, int vt) {
    switch (D) {
        case 16: SR_OCC_DISPATCH(ncc_occ, 16, vt, ncc_r)
        case 32: SR_OCC_DISPATCH(ncc_occ, 32, vt, ncc_r)
        case 64: SR_OCC_DISPATCH(ncc_occ, 64, vt, ncc_r)
        default: return 0;
    }
}

int agg_batch_occupancy(int D, int agg_r, int vt) {
    switch (D) {
        case 16: SR_OCC_DISPATCH(agg_occ, 16, vt, agg_r)
        case 32: SR_OCC_DISPATCH(agg_occ, 32, vt, agg_r)
        case 64: SR_OCC_DISPATCH(agg_occ, 64, vt, agg_r)
        default: return 0;
    }
}

int ncc_sl_occupancy(int D, int ncc_r, int vt) {
    switch (D) {
        case 16: SR_OCC_DISPATCH(ncc_sl_occ, 16, vt, ncc_r)
        case 32: SR_OCC_DISPATCH(ncc_sl_occ, 32, vt, ncc_r)
        case 64: SR_OCC_DISPATCH(ncc_sl_occ, 64, vt, ncc_r)
        default: return 0;
    }
}

// Segment length: a CTA of launch_ncc_sl owns 4096/D columns and seg rows,
// and spends about seg + ncc_r + 2 row steps (the window's first 2 ncc_r + 1
// rows are only added).  Model: an SM holding L CTAs of a launch takes
// L * (seg + ncc_r + 2) / min(L, resident, 3) steps (its throughput saturates
// at three resident CTAs); the shortest model time wins, the longer segment
// on ties.  Deterministic per (frame size, D, radius, device): the resident
// count is the kernel's launch bound, not a measured occupancy, which a
// bounds-checked build would change.
int ncc_segment(int W, int H, int D, int ncc_r, int vt) {
    static int env = -1;
    if (env < 0) {
        const char *e = getenv("SR_NCC_SEG");
        const int v = e ? atoi(e) : 0;
        env = (v >= 1 && v <= kNslMaxSeg) ? v : 0;
    }
    if (env > 0) return env;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    (void)vt;
    const int occ = kNslResident;   // a constant, so that every build picks the same segments
    const int tx = kNslThreads / (D / kNslDB) * kNslU;   // columns of a CTA
    const long long nx = (W + D - 1 + tx - 1) / tx;
    const int hi = std::min(std::max(H, 1), kNslMaxSeg), lo = std::min(hi, 8);
    int best = hi;
    double best_t = 1e300;
    for (int seg = hi; seg >= lo; --seg) {
        const long long nseg = (H + seg - 1) / seg;
        const long long L = (nx * nseg + sms - 1) / sms;
        const long long conc = std::min<long long>(std::min<long long>(L, occ), 3);
        const double t = (double)L * (seg + ncc_r + 2) / (double)conc;
        if (t < best_t) { best_t = t; best = seg; }
    }
    return best;
}

}  // namespace sr

namespace {

const char *const kStageNames = "prep,ncc,agg_tgt,agg_ref";

}  // namespace


namespace {

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc((void **)p, n * sizeof(T));
}

void free_all(sr_ctx *c) {
    void *ptrs[] = {c->rw, c->mu_l, c->inv_l, c->mu_r, c->inv_r, c->vol_l, c->vol_r, c->dsub,
                    c->rowsh, c->band_disp, c->band_wta,
                    c->lbl_l, c->lbl_r, c->agg_l, c->agg_r, c->stage_l, c->stage_r,
                    c->stage_disp, c->d_err, c->g_vol, c->g_wsum, c->g_rw, c->g_partial,
                    c->f_pairs, c->f_has, c->f_counts, c->f_model, c->f_partial, c->band,
                    c->nrange};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (c->ev_ring) {
        for (int i = 0; i < kProfRing * (kStages + 1); ++i)
            if (c->ev_ring[i]) cudaEventDestroy(c->ev_ring[i]);
        delete[] c->ev_ring;
    }
    for (int i = 0; i < 2; ++i) {
        if (c->ev_up[i]) cudaEventDestroy(c->ev_up[i]);
        if (c->ev_comp[i]) cudaEventDestroy(c->ev_comp[i]);
        if (c->ev_down[i]) cudaEventDestroy(c->ev_down[i]);
    }
    if (c->up) cudaStreamDestroy(c->up);
    if (c->down) cudaStreamDestroy(c->down);
    if (c->h_err_async) cudaFreeHost(c->h_err_async);
    sr_batch_free(c);
}

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tensor map of a cost volume [H][W][D] viewed as [H*W][D], box kBandD
// disparities plus 16 bytes (the band kernel's padded cost columns) x
// (32 + 2 agg_r) pixels, zeros outside.
bool encode_volume_map(CUtensorMap *m, void *vol, int vt, int W, int H, int D, int agg_r) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const CUtensorMapDataType dt = vt == sr::kVolF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : vt == sr::kVolF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)W * H};
    const cuuint64_t strides[1] = {(cuuint64_t)D * sr::vol_elem_bytes(vt)};
    const cuuint32_t box[2] = {(cuuint32_t)(sr::kBandD + 16 / sr::vol_elem_bytes(vt)),
                               (cuuint32_t)(32 + 2 * agg_r)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, dt, 2, vol, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// Tensor map of the extended reference volume [H][W+D-1][D] viewed as
// [H*(W+D-1)][D], box CW disparities x BH pixels of the sheared kernel's
// configuration, zeros outside (see launch_agg_shear).
bool sr::encode_shear_map(void *tmap, const void *volx, int vt, int W, int H, int D, int agg_r) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    int cw = 0, bh = 0;
    bool ok = false;
#define SR_BOX(DD)                                                                    \
    ok = vt == kVolF32 ? sr::aggs_box_d##DD##_f32(agg_r, &cw, &bh)                    \
       : vt == kVolF16 ? sr::aggs_box_d##DD##_f16(agg_r, &cw, &bh)                    \
                       : sr::aggs_box_d##DD##_bf16(agg_r, &cw, &bh)
    switch (D) {
        case 16: SR_BOX(16); break;
        case 32: SR_BOX(32); break;
        case 64: SR_BOX(64); break;
        default: break;
    }
#undef SR_BOX
    if (!ok) return false;
    const CUtensorMapDataType dt = vt == sr::kVolF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : vt == sr::kVolF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)(W + D - 1) * H};
    const cuuint64_t strides[1] = {(cuuint64_t)D * sr::vol_elem_bytes(vt)};
    const cuuint32_t box[2] = {(cuuint32_t)cw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    return fn(static_cast<CUtensorMap *>(tmap), dt, 2, const_cast<void *>(volx), dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// IEEE 754 binary16 bit pattern -> float (sign, 5-bit exponent, 10-bit fraction).
float half_bits_to_float(uint16_t h) {
    const int s = h >> 15, e = (h >> 10) & 0x1f, m = h & 0x3ff;
    float v;
    if (e == 0) v = ldexpf((float)m, -24);                      // subnormal: m * 2^-24
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexpf((float)(m | 0x400), e - 25);                // (1024 + m) * 2^(e-25)
    return s ? -v : v;
}
// bfloat16 is the upper half of a binary32 pattern.
float bf16_bits_to_float(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float v;
    memcpy(&v, &u, sizeof(v));
    return v;
}

}  // namespace

extern "C" {

const char *sr_version(void) { return "sr 0.1 (sm_103a, staged fp32)"; }

const char *sr_status_str(sr_status s) {
    switch (s) {
        case SR_OK: return "SR_OK";
        case SR_ERR_INVALID_ARG: return "SR_ERR_INVALID_ARG";
        case SR_ERR_UNSUPPORTED: return "SR_ERR_UNSUPPORTED";
        case SR_ERR_OOM: return "SR_ERR_OOM";
        case SR_ERR_CUDA: return "SR_ERR_CUDA";
        case SR_ERR_STATE: return "SR_ERR_STATE";
        case SR_ERR_TIMEOUT: return "SR_ERR_TIMEOUT";
        case SR_ERR_BOUNDS: return "SR_ERR_BOUNDS";
    }
    return "SR_ERR_UNKNOWN";
}

const char *sr_last_error(const sr_ctx *c) { return c ? c->err : ""; }

const char *sr_stage_names(void) { return kStageNames; }

int sr_kernels_per_match(const sr_ctx *c) {
    (void)c;
    return 4;   // prep (warp + statistics), ncc (extended volume), agg_tgt, agg_ref (+ L-R check)
}

sr_status sr_create(const sr_params *params, void *cuda_stream, sr_ctx **out) {
    if (!out) return SR_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params) return SR_ERR_INVALID_ARG;
    const sr_params &p = *params;
    if (p.width < 1 || p.height < 1 || p.width > 16384 || p.height > 16384 || p.max_disp < 1 ||
        p.ncc_radius < 0 || p.agg_radius < 0 || !finite_pos(p.gamma_d) ||
        !finite_pos(p.gamma_r) || !(p.lr_thresh >= 0.0f) || !isfinite(p.lr_thresh))
        return SR_ERR_INVALID_ARG;
    if (p.vol_dtype != SR_VOL_F32 && p.vol_dtype != SR_VOL_F16 && p.vol_dtype != SR_VOL_BF16)
        return SR_ERR_INVALID_ARG;
    if (!sr::ncc_supported(p.max_disp, p.ncc_radius) || !sr::agg_supported(p.max_disp, p.agg_radius))
        return SR_ERR_UNSUPPORTED;

    sr_ctx *c = new (std::nothrow) sr_ctx();
    if (!c) return SR_ERR_OOM;
    c->p = p;
    c->st = (cudaStream_t)cuda_stream;
    cudaGetDevice(&c->device);
    const size_t W = p.width, H = p.height, D = p.max_disp, npx = W * H;
    const size_t WE = W + D - 1;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&c->rw, npx);
    if (e == cudaSuccess) e = dalloc(&c->mu_l, H * WE);
    if (e == cudaSuccess) e = dalloc(&c->mu_r, H * WE);
    if (e == cudaSuccess) e = dalloc(&c->inv_l, H * WE);
    if (e == cudaSuccess) e = dalloc(&c->inv_r, H * WE);
    // vol_l: the extended reference volume [H][W+D-1][D] of sr_match, or the
    // reference volume [H][W][D] of sr_match_restricted (a prefix of it)
    const size_t vbytes = npx * D * sr::vol_elem_bytes(p.vol_dtype);
    if (e == cudaSuccess) e = cudaMalloc(&c->vol_l, H * WE * D * sr::vol_elem_bytes(p.vol_dtype));
    if (e == cudaSuccess) e = cudaMalloc(&c->vol_r, vbytes);
    if (e == cudaSuccess) e = dalloc(&c->dsub, npx);
    if (e == cudaSuccess) e = dalloc(&c->rowsh, H);
    if (e == cudaSuccess) e = dalloc(&c->lbl_l, npx);
    if (e == cudaSuccess) e = dalloc(&c->lbl_r, npx);
    if (e == cudaSuccess) e = dalloc(&c->d_err, 1);
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear a sticky allocation error
        free_all(c);
        delete c;
        return e == cudaErrorMemoryAllocation ? SR_ERR_OOM : SR_ERR_CUDA;
    }
    c->ncc_seg = sr::ncc_segment(p.width, p.height, p.max_disp, p.ncc_radius, (int)p.vol_dtype);
    *out = c;
    SR_LOG(2, "context %dx%d, D %d, NCC %dx%d, bilateral %dx%d, volume type %d on device %d",
           p.width, p.height, p.max_disp, 2 * p.ncc_radius + 1, 2 * p.ncc_radius + 1,
           2 * p.agg_radius + 1, 2 * p.agg_radius + 1, (int)p.vol_dtype, c->device);
    return SR_OK;
}

sr_status sr_destroy(sr_ctx *c) {
    if (!c) return SR_OK;
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
    return SR_OK;
}

sr_status sr_set_plane(sr_ctx *c, double alpha0, double alpha1, double delta) {
    if (!c || !isfinite(alpha0) || !isfinite(alpha1) || !isfinite(delta)) return SR_ERR_INVALID_ARG;
    c->alpha0 = alpha0;
    c->alpha1 = alpha1;
    c->delta = delta;
    return SR_OK;
}

sr_status sr_set_camera(sr_ctx *c, double f_px, double baseline, double u0, double v0) {
    if (!c || !(f_px > 0) || !isfinite(f_px) || !(baseline > 0) || !isfinite(baseline) ||
        !isfinite(u0) || !isfinite(v0))
        return SR_ERR_INVALID_ARG;
    c->f_px = f_px;
    c->baseline = baseline;
    c->u0 = u0;
    c->v0 = v0;
    c->camera = true;
    return SR_OK;
}

sr_status sr_set_debug(sr_ctx *c, int flags) {
    if (!c || (flags & ~(SR_DEBUG_KEEP_AGG | SR_DEBUG_WITHHOLD_ROW | SR_DEBUG_NO_BAND |
                   SR_DEBUG_BOUNDS_SELFTEST)))
        return SR_ERR_INVALID_ARG;
    if ((flags & SR_DEBUG_KEEP_AGG) && !c->agg_l) {
        const size_t n = (size_t)c->p.width * c->p.height * c->p.max_disp;
        SR_TRY(c, dalloc(&c->agg_l, n), "cudaMalloc(agg_l)");
        SR_TRY(c, dalloc(&c->agg_r, n), "cudaMalloc(agg_r)");
    }
    c->debug = flags;
    return SR_OK;
}

sr_status sr_set_profiling(sr_ctx *c, int enable) {
    if (!c) return SR_ERR_INVALID_ARG;
    if (enable && !c->ev_ring) {
        c->ev_ring = new (std::nothrow) cudaEvent_t[kProfRing * (kStages + 1)]();
        if (!c->ev_ring) return SR_ERR_OOM;
        for (int i = 0; i < kProfRing * (kStages + 1); ++i)
            SR_TRY(c, cudaEventCreate(&c->ev_ring[i]), "cudaEventCreate");
    }
    c->profiling = enable != 0;
    c->timed = false;
    c->prof_count = 0;
    return SR_OK;
}

sr_status sr_stage_times(sr_ctx *c, float *ms, int n, int *count) {
    if (!c || (n > 0 && !ms)) return SR_ERR_INVALID_ARG;
    if (count) *count = kStages;
    if (!c->timed || c->prof_count < 1) return SR_ERR_STATE;
    const cudaEvent_t *e = c->ev_ring + ((c->prof_count - 1) % kProfRing) * (kStages + 1);
    SR_TRY(c, cudaEventSynchronize(e[kStages]), "cudaEventSynchronize");
    for (int i = 0; i < kStages && i < n; ++i)
        SR_TRY(c, cudaEventElapsedTime(&ms[i], e[i], e[i + 1]), "cudaEventElapsedTime");
    return take_device_error(c);
}

sr_status sr_stage_times_history(sr_ctx *c, float *ms, int max_matches, int *count) {
    if (!c || !ms || max_matches < 1 || !count) return SR_ERR_INVALID_ARG;
    *count = 0;
    if (!c->ev_ring || c->prof_count < 1) return SR_ERR_STATE;
    long long m = c->prof_count < kProfRing ? c->prof_count : kProfRing;
    if (m > max_matches) m = max_matches;
    const long long first = c->prof_count - m;
    SR_TRY(c, cudaEventSynchronize(c->ev_ring[((c->prof_count - 1) % kProfRing) * (kStages + 1) +
                                              kStages]),
           "cudaEventSynchronize");
    for (long long k = 0; k < m; ++k) {
        const cudaEvent_t *e = c->ev_ring + ((first + k) % kProfRing) * (kStages + 1);
        for (int i = 0; i < kStages; ++i)
            SR_TRY(c, cudaEventElapsedTime(&ms[k * kStages + i], e[i], e[i + 1]),
                   "cudaEventElapsedTime");
    }
    *count = (int)m;
    return take_device_error(c);
}

sr_status sr_synchronize(sr_ctx *c) {
    if (!c) return SR_ERR_INVALID_ARG;
    SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
    if (c->up) SR_TRY(c, cudaStreamSynchronize(c->up), "cudaStreamSynchronize(upload)");
    if (c->down) SR_TRY(c, cudaStreamSynchronize(c->down), "cudaStreamSynchronize(download)");
    return take_device_error(c);
}

sr_status sr_match(sr_ctx *c, const uint8_t *d_left, const uint8_t *d_right, int pitch_bytes,
                   float *d_disp, int16_t *d_wta_or_null) {
    NvtxRange nvtx_call("sr_match");
    if (!c || !d_left || !d_right || !d_disp || pitch_bytes < c->p.width) return SR_ERR_INVALID_ARG;
    const sr_params &p = c->p;
    const int W = p.width, H = p.height, D = p.max_disp;
    cudaStream_t st = c->st;
    const bool prof = c->profiling;
    const bool keep = (c->debug & SR_DEBUG_KEEP_AGG) != 0;
    int stage = 0;
    cudaEvent_t *evs = prof ? c->ev_ring + (c->prof_count % kProfRing) * (kStages + 1) : nullptr;
    auto mark = [&]() -> cudaError_t {
        return prof ? cudaEventRecord(evs[stage++], st) : cudaSuccess;
    };
    c->matched = false;
    c->timed = false;
    if (!c->tmap_x_ok) {
        if (!sr::encode_shear_map(&c->tmap_x, c->vol_l, p.vol_dtype, W, H, D, p.agg_radius)) {
            snprintf(c->err, sizeof(c->err), "cuTensorMapEncodeTiled failed or is unavailable");
            return SR_ERR_CUDA;
        }
        c->tmap_x_ok = true;
    }
    const int WE = W + D - 1;
    SR_TRY(c, mark(), "cudaEventRecord");
    {
        NvtxRange r("prep");
        SR_TRY(c, sr::launch_prep(d_left, d_right, pitch_bytes, W, H, D, p.ncc_radius, c->alpha0,
                                  c->alpha1, c->delta, 0, c->rw, c->mu_l, c->inv_l, c->mu_r,
                                  c->inv_r, c->rowsh, st),
               "prep");
    }
    SR_TRY(c, mark(), "cudaEventRecord");
    {
        // one extended reference volume holds both views (target c(u,d) =
        // extended reference c(u+d,d))
        NvtxRange r("ncc");
        SR_TRY(c, sr::launch_ncc_sl(d_left, d_right, pitch_bytes, W, H, D, p.ncc_radius, 0,
                                    c->alpha0, c->alpha1, c->delta, c->inv_l, c->inv_r, c->vol_l,
                                    p.vol_dtype, WE, c->ncc_seg, st),
               "ncc");
    }
    SR_TRY(c, mark(), "cudaEventRecord");
    sr::AggDebug dbg = agg_debug(c);
    // each aggregation starts while its predecessor drains (programmatic
    // dependent launch, see sr::pdl_trigger); not while stage events sit
    // between the kernels
    dbg.pdl = !prof;
    // target view first: the reference-view kernel runs the L-R check and
    // the post-processing in its epilogue, on the finished target labels
    {
        NvtxRange r("agg_tgt");
        SR_TRY(c, sr::launch_agg_shear(&c->tmap_x, p.vol_dtype, c->rw, W, H, D, p.agg_radius,
                                       p.gamma_d, p.gamma_r, c->lbl_r, keep ? c->agg_r : nullptr,
                                       dbg, st),
               "agg_tgt");
    }
    SR_TRY(c, mark(), "cudaEventRecord");
    sr::AggWin post;
    post.post.lbl_r = c->lbl_r;
    post.post.disp = d_disp;
    post.post.wta = d_wta_or_null;
    post.post.rowsh = c->rowsh;
    post.post.lr_thresh = p.lr_thresh;
    {
        NvtxRange r("agg_ref");
        SR_TRY(c, sr::launch_agg(c->vol_l, p.vol_dtype, d_left, pitch_bytes, nullptr, W, H, D,
                                 p.agg_radius, p.gamma_d, p.gamma_r, c->lbl_l, c->dsub,
                                 keep ? c->agg_l : nullptr, dbg, st, post, WE),
               "agg_ref");
    }
    SR_TRY(c, mark(), "cudaEventRecord");
    c->matched = true;
    c->vol_ext = true;
    c->agg_valid = keep;
    c->timed = prof;
    if (prof) ++c->prof_count;
    return SR_OK;
}

// Image rows [r0, r1) that the band of output rows [y0, y1) reads: the rows
// its bilateral windows (agg_radius) and NCC blocks (ncc_radius) reach, and
// above them back to the first row of the NCC segment of its first cost row
// minus ncc_radius, where that segment's window sums start in the whole
// frame too (see launch_ncc_sl).
static void band_read_rows(const sr_ctx *c, int y0, int y1, int *r0, int *r1) {
    const sr_params &p = c->p;
    const int first_cost = std::max(0, y0 - p.agg_radius);
    const int seg_start = first_cost / c->ncc_seg * c->ncc_seg;
    *r0 = std::max(0, seg_start - p.ncc_radius);
    *r1 = std::min(p.height, y1 + p.ncc_radius + p.agg_radius);
}

sr_status sr_band_rows(const sr_ctx *c, int y0, int y1, int *r0, int *r1) {
    if (!c || !r0 || !r1 || y0 < 0 || y1 > c->p.height || y0 >= y1) return SR_ERR_INVALID_ARG;
    band_read_rows(c, y0, y1, r0, r1);
    return SR_OK;
}

sr_status sr_match_rows(sr_ctx *c, const uint8_t *d_left_rows, const uint8_t *d_right_rows,
                        int pitch_bytes, int y0, int y1, float *d_disp_rows,
                        int16_t *d_wta_rows_or_null) {
    NvtxRange nvtx_call("sr_match_rows");
    if (!c || !d_left_rows || !d_right_rows || !d_disp_rows || pitch_bytes < c->p.width)
        return SR_ERR_INVALID_ARG;
    const sr_params &p = c->p;
    const int W = p.width, H = p.height, D = p.max_disp;
    if (y0 < 0 || y1 > H || y0 >= y1) return SR_ERR_INVALID_ARG;
    // the band and the halo rows its NCC blocks and bilateral windows reach
    int r0 = 0, r1 = 0;
    band_read_rows(c, y0, y1, &r0, &r1);
    const int Hs = r1 - r0;
    const size_t npx = (size_t)W * H;
    cudaStream_t st = c->st;
    if (!c->band_disp) {
        SR_TRY(c, dalloc(&c->band_disp, npx), "cudaMalloc(band disparity)");
        SR_TRY(c, dalloc(&c->band_wta, npx), "cudaMalloc(band labels)");
    }
    if (c->band_rows != Hs) {
        // the sheared view of a volume of Hs rows: copies past its last row
        // read zeros, as for a whole frame
        if (!sr::encode_shear_map(&c->tmap_band, c->vol_l, p.vol_dtype, W, Hs, D, p.agg_radius)) {
            snprintf(c->err, sizeof(c->err), "cuTensorMapEncodeTiled failed or is unavailable");
            c->band_rows = 0;
            return SR_ERR_CUDA;
        }
        c->band_rows = Hs;
    }
    c->matched = false;   // the scratch holds a band, not a frame
    c->timed = false;
    const int WE = W + D - 1;
    SR_TRY(c, sr::launch_prep(d_left_rows, d_right_rows, pitch_bytes, W, Hs, D, p.ncc_radius,
                              c->alpha0, c->alpha1, c->delta, r0, c->rw, c->mu_l, c->inv_l,
                              c->mu_r, c->inv_r, c->rowsh, st),
           "prep");
    SR_TRY(c, sr::launch_ncc_sl(d_left_rows, d_right_rows, pitch_bytes, W, Hs, D, p.ncc_radius,
                                r0, c->alpha0, c->alpha1, c->delta, c->inv_l, c->inv_r, c->vol_l,
                                p.vol_dtype, WE, c->ncc_seg, st),
           "ncc");
    const sr::AggDebug dbg = agg_debug(c);
    SR_TRY(c, sr::launch_agg_shear(&c->tmap_band, p.vol_dtype, c->rw, W, Hs, D, p.agg_radius,
                                   p.gamma_d, p.gamma_r, c->lbl_r, nullptr, dbg, st),
           "agg_tgt");
    sr::AggWin post;
    post.post.lbl_r = c->lbl_r;
    post.post.disp = c->band_disp;
    post.post.wta = c->band_wta;
    post.post.rowsh = c->rowsh;
    post.post.lr_thresh = p.lr_thresh;
    SR_TRY(c, sr::launch_agg(c->vol_l, p.vol_dtype, d_left_rows, pitch_bytes, nullptr, W, Hs, D,
                             p.agg_radius, p.gamma_d, p.gamma_r, c->lbl_l, c->dsub, nullptr, dbg,
                             st, post, WE),
           "agg_ref");
    const size_t off = (size_t)(y0 - r0) * W, n = (size_t)(y1 - y0) * W;
    SR_TRY(c, cudaMemcpyAsync(d_disp_rows, c->band_disp + off, n * sizeof(float),
                              cudaMemcpyDeviceToDevice, st),
           "band rows");
    if (d_wta_rows_or_null)
        SR_TRY(c, cudaMemcpyAsync(d_wta_rows_or_null, c->band_wta + off, n * sizeof(int16_t),
                                  cudaMemcpyDeviceToDevice, st),
               "band rows");
    return SR_OK;
}

sr_status sr_match_restricted(sr_ctx *c, const uint8_t *d_left, const uint8_t *d_right,
                              int pitch_bytes, const int16_t *d_centre, int radius, float *d_disp,
                              int16_t *d_wta_or_null) {
    NvtxRange nvtx_call("sr_match_restricted");
    if (!c || !d_left || !d_right || !d_disp || pitch_bytes < c->p.width) return SR_ERR_INVALID_ARG;
    const sr_params &p = c->p;
    const int W = p.width, H = p.height, D = p.max_disp;
    if (radius < 0 || radius >= D) return SR_ERR_INVALID_ARG;
    cudaStream_t st = c->st;
    sr::AggWin win;
    win.centre = d_centre;
    win.centre_const = (int)lround(c->delta);
    win.radius = radius;
    win.dfull = D;
    const bool banded = D > sr::kBandD && !(c->debug & SR_DEBUG_NO_BAND);
    if (banded) {
        if (!c->tmaps) {
            if (!encode_volume_map(&c->tmap_l, c->vol_l, p.vol_dtype, W, H, D, p.agg_radius) ||
                !encode_volume_map(&c->tmap_r, c->vol_r, p.vol_dtype, W, H, D, p.agg_radius)) {
                snprintf(c->err, sizeof(c->err), "cuTensorMapEncodeTiled failed or is unavailable");
                return SR_ERR_CUDA;
            }
            c->tmaps = true;
        }
        if (!c->band) {
            const size_t tiles = (size_t)sr::ceil_div(W, sr::kAggTileX) * sr::ceil_div(H, sr::kAggTileY);
            SR_TRY(c, dalloc(&c->band, tiles), "cudaMalloc(bands)");
            SR_TRY(c, dalloc(&c->nrange, tiles), "cudaMalloc(ranges)");
        }
        if (!c->vols_zeroed) {
            // costs outside a tile's NCC range are not written; the band boxes
            // may read such entries next to the image's ends (with zero weight),
            // so they must hold finite values
            const size_t vb = (size_t)W * H * D * sr::vol_elem_bytes(p.vol_dtype);
            SR_TRY(c, cudaMemsetAsync(c->vol_l, 0, vb, st), "cudaMemset(volume)");
            SR_TRY(c, cudaMemsetAsync(c->vol_r, 0, vb, st), "cudaMemset(volume)");
            c->vols_zeroed = true;
        }
        win.band = c->band;
        const int align = (int)(16 / sr::vol_elem_bytes(p.vol_dtype));
        SR_TRY(c, sr::launch_tile_bands(win, W, H, align, c->band, st), "tile bands");
        SR_TRY(c, sr::launch_ncc_ranges(c->band, W, H, D, p.agg_radius, c->nrange, st), "ncc ranges");
    }
    c->matched = false;
    c->timed = false;
    const sr::AggDebug dbg = agg_debug(c);
    SR_TRY(c, sr::launch_prep(d_left, d_right, pitch_bytes, W, H, D, p.ncc_radius, c->alpha0,
                              c->alpha1, c->delta, 0, c->rw, c->mu_l, c->inv_l, c->mu_r,
                              c->inv_r, c->rowsh, st),
           "prep");
    const int2 *nrange = banded ? c->nrange : nullptr;
    SR_TRY(c, sr::launch_ncc(false, d_left, pitch_bytes, c->rw, c->mu_l, c->inv_l, c->mu_r,
                             c->inv_r, W, H, D, p.ncc_radius, c->vol_l, p.vol_dtype, st, nrange),
           "ncc_ref");
    SR_TRY(c, sr::launch_ncc(true, d_left, pitch_bytes, c->rw, c->mu_l, c->inv_l, c->mu_r,
                             c->inv_r, W, H, D, p.ncc_radius, c->vol_r, p.vol_dtype, st, nrange),
           "ncc_tgt");
    if (banded) {
        SR_TRY(c, sr::launch_agg_band(&c->tmap_l, p.vol_dtype, d_left, pitch_bytes, nullptr, W, H,
                                      p.agg_radius, p.gamma_d, p.gamma_r, c->lbl_l, c->dsub, dbg,
                                      win, st),
               "agg_ref band");
        SR_TRY(c, sr::launch_agg_band(&c->tmap_r, p.vol_dtype, nullptr, 0, c->rw, W, H,
                                      p.agg_radius, p.gamma_d, p.gamma_r, c->lbl_r, nullptr, dbg,
                                      win, st),
               "agg_tgt band");
    }
    SR_TRY(c, sr::launch_agg(c->vol_l, p.vol_dtype, d_left, pitch_bytes, nullptr, W, H, D,
                             p.agg_radius, p.gamma_d, p.gamma_r, c->lbl_l, c->dsub, nullptr, dbg,
                             st, win),
           "agg_ref");
    SR_TRY(c, sr::launch_agg(c->vol_r, p.vol_dtype, nullptr, 0, c->rw, W, H, D, p.agg_radius,
                             p.gamma_d, p.gamma_r, c->lbl_r, nullptr, nullptr, dbg, st, win),
           "agg_tgt");
    SR_TRY(c, sr::launch_lrc_post(c->lbl_l, c->lbl_r, c->dsub, W, H, c->rowsh, p.lr_thresh,
                                  d_disp, d_wta_or_null, st),
           "lrc_post");
    c->matched = true;
    c->vol_ext = false;
    c->agg_valid = false;
    return SR_OK;
}

// Two slots of host-buffer staging (allocated on first use).
static sr_status ensure_staging(sr_ctx *c) {
    if (c->stage_l) return SR_OK;
    const size_t npx = (size_t)c->p.width * c->p.height;
    SR_TRY(c, dalloc(&c->stage_l, 2 * npx), "cudaMalloc(stage)");
    SR_TRY(c, dalloc(&c->stage_r, 2 * npx), "cudaMalloc(stage)");
    SR_TRY(c, dalloc(&c->stage_disp, 2 * npx), "cudaMalloc(stage)");
    return SR_OK;
}

sr_status sr_match_host(sr_ctx *c, const uint8_t *h_left, const uint8_t *h_right, float *h_disp) {
    NvtxRange nvtx_call("sr_match_host");
    if (!c || !h_left || !h_right || !h_disp) return SR_ERR_INVALID_ARG;
    const size_t npx = (size_t)c->p.width * c->p.height;
    sr_status s0 = ensure_staging(c);
    if (s0 != SR_OK) return s0;
    // frames still queued by sr_match_host_async use the staging too
    if (c->up) SR_TRY(c, cudaStreamSynchronize(c->up), "cudaStreamSynchronize(upload)");
    if (c->down) SR_TRY(c, cudaStreamSynchronize(c->down), "cudaStreamSynchronize(download)");
    SR_TRY(c, cudaMemcpyAsync(c->stage_l, h_left, npx, cudaMemcpyHostToDevice, c->st), "H2D left");
    SR_TRY(c, cudaMemcpyAsync(c->stage_r, h_right, npx, cudaMemcpyHostToDevice, c->st), "H2D right");
    sr_status s = sr_match(c, c->stage_l, c->stage_r, c->p.width, c->stage_disp, nullptr);
    if (s != SR_OK) return s;
    SR_TRY(c, cudaMemcpyAsync(h_disp, c->stage_disp, npx * sizeof(float), cudaMemcpyDeviceToHost,
                              c->st),
           "D2H disp");
    SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
    return take_device_error(c);
}

sr_status sr_match_host_async(sr_ctx *c, const uint8_t *h_left, const uint8_t *h_right,
                              float *h_disp) {
    NvtxRange nvtx_call("sr_match_host_async");
    if (!c || !h_left || !h_right || !h_disp) return SR_ERR_INVALID_ARG;
    const size_t npx = (size_t)c->p.width * c->p.height;
    sr_status s0 = ensure_staging(c);
    if (s0 != SR_OK) return s0;
    if (!c->up) {
        SR_TRY(c, cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking), "cudaStreamCreate");
        SR_TRY(c, cudaStreamCreateWithFlags(&c->down, cudaStreamNonBlocking), "cudaStreamCreate");
        SR_TRY(c, cudaMallocHost(&c->h_err_async, 2 * sizeof(int)), "cudaMallocHost(err)");
        c->h_err_async[0] = c->h_err_async[1] = 0;
        for (int i = 0; i < 2; ++i) {
            SR_TRY(c, cudaEventCreateWithFlags(&c->ev_up[i], cudaEventDisableTiming), "cudaEventCreate");
            SR_TRY(c, cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming), "cudaEventCreate");
            SR_TRY(c, cudaEventCreateWithFlags(&c->ev_down[i], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    const int k = c->slot;
    uint8_t *dl = c->stage_l + k * npx, *dr = c->stage_r + k * npx;
    float *dd = c->stage_disp + k * npx;
    if (c->frames_queued >= 2) {
        // the frame queued two calls ago used this slot: let it finish, so
        // that its result is in its host buffer and its inputs are free
        SR_TRY(c, cudaEventSynchronize(c->ev_down[k]), "cudaEventSynchronize");
        // the error word as that frame's download left it (copied behind it on
        // the download stream): no blocking read that would wait for the
        // frame queued since
        if (c->h_err_async[k]) {
            c->h_err_async[k] = 0;
            SR_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st), "cudaMemsetAsync(err)");
            snprintf(c->err, sizeof(c->err), "a bounded device wait for a cost-row copy ran out");
            SR_LOG(1, "%s", c->err);
            return SR_ERR_TIMEOUT;
        }
        // upload after that frame's kernels have read the slot's images
        SR_TRY(c, cudaStreamWaitEvent(c->up, c->ev_comp[k], 0), "cudaStreamWaitEvent");
    }
    SR_TRY(c, cudaMemcpyAsync(dl, h_left, npx, cudaMemcpyHostToDevice, c->up), "H2D left");
    SR_TRY(c, cudaMemcpyAsync(dr, h_right, npx, cudaMemcpyHostToDevice, c->up), "H2D right");
    SR_TRY(c, cudaEventRecord(c->ev_up[k], c->up), "cudaEventRecord");
    SR_TRY(c, cudaStreamWaitEvent(c->st, c->ev_up[k], 0), "cudaStreamWaitEvent");
    sr_status s = sr_match(c, dl, dr, c->p.width, dd, nullptr);
    if (s != SR_OK) return s;
    SR_TRY(c, cudaEventRecord(c->ev_comp[k], c->st), "cudaEventRecord");
    SR_TRY(c, cudaStreamWaitEvent(c->down, c->ev_comp[k], 0), "cudaStreamWaitEvent");
    SR_TRY(c, cudaMemcpyAsync(h_disp, dd, npx * sizeof(float), cudaMemcpyDeviceToHost, c->down),
           "D2H disp");
    SR_TRY(c, cudaMemcpyAsync(&c->h_err_async[k], c->d_err, sizeof(int), cudaMemcpyDeviceToHost,
                              c->down),
           "D2H err");
    SR_TRY(c, cudaEventRecord(c->ev_down[k], c->down), "cudaEventRecord");
    // the next match on this slot writes dd: after this download
    c->slot = k ^ 1;
    ++c->frames_queued;
    return SR_OK;
}

sr_status sr_reconstruct(sr_ctx *c, const float *d_disp, float *d_xyz) {
    NvtxRange nvtx_call("sr_reconstruct");
    if (!c || !d_disp || !d_xyz) return SR_ERR_INVALID_ARG;
    if (!c->camera) return SR_ERR_STATE;
    SR_TRY(c, sr::launch_xyz(d_disp, c->p.width, c->p.height, c->f_px, c->baseline, c->u0, c->v0,
                             d_xyz, c->st, (c->debug & SR_DEBUG_BOUNDS_SELFTEST) != 0),
           "xyz");
    return SR_OK;
}

sr_status sr_grad_plane(sr_ctx *c, const uint8_t *d_left, const uint8_t *d_right, int pitch_bytes,
                        const int16_t *d_dstar, double *h_out3, float *d_grad_left,
                        float *d_grad_right) {
    NvtxRange nvtx_call("sr_grad_plane");
    if (!c || !d_left || !d_right || !d_dstar || !h_out3 || pitch_bytes < c->p.width)
        return SR_ERR_INVALID_ARG;
    const sr_params &p = c->p;
    const int W = p.width, H = p.height, D = p.max_disp;
    const size_t npx = (size_t)W * H;
    const size_t nparts = sr::grad_partial_count(W, H) * 3;
    if (!c->g_wsum) {
        SR_TRY(c, dalloc(&c->g_wsum, npx), "cudaMalloc(grad wsum)");
        SR_TRY(c, dalloc(&c->g_rw, npx), "cudaMalloc(grad rw)");
        SR_TRY(c, dalloc(&c->g_partial, nparts + 3), "cudaMalloc(grad partial)");
    }
    // FP32 reference volume: the context's own when it stores FP32, else an
    // FP32 volume of its own (allocated once)
    float *cost = (float *)c->vol_l;
    if (p.vol_dtype != SR_VOL_F32) {
        if (!c->g_vol) SR_TRY(c, dalloc(&c->g_vol, npx * D), "cudaMalloc(grad volume)");
        cost = c->g_vol;
    }
    cudaStream_t st = c->st;
    c->matched = false;   // the context's scratch no longer holds the last sr_match
    SR_TRY(c, sr::launch_prep(d_left, d_right, pitch_bytes, W, H, D, p.ncc_radius, c->alpha0,
                              c->alpha1, c->delta, 0, c->rw, c->mu_l, c->inv_l, c->mu_r,
                              c->inv_r, c->rowsh, st),
           "prep");
    SR_TRY(c, sr::launch_ncc(false, d_left, pitch_bytes, c->rw, c->mu_l, c->inv_l, c->mu_r,
                             c->inv_r, W, H, D, p.ncc_radius, cost, sr::kVolF32, st),
           "ncc_ref");
    double *out3 = c->g_partial + nparts;
    SR_TRY(c, sr::launch_grad(d_left, d_right, pitch_bytes, W, H, D, p.ncc_radius, p.agg_radius,
                              p.gamma_d, p.gamma_r, c->alpha0, c->alpha1, c->delta, c->rw, c->mu_l,
                              c->inv_l, c->mu_r, c->inv_r, cost, d_dstar, c->g_wsum,
                              d_grad_right ? c->g_rw : nullptr, d_grad_left, d_grad_right,
                              c->g_partial, out3, st),
           "grad");
    SR_TRY(c, cudaMemcpyAsync(h_out3, out3, 3 * sizeof(double), cudaMemcpyDeviceToHost, st),
           "D2H grad");
    SR_TRY(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return take_device_error(c);
}

sr_status sr_fit_alpha(sr_ctx *c, const float *d_disp, int n_hyp, const int32_t *h_pairs,
                       float tau_px, double *h_alpha, int32_t *h_counts, int *h_best,
                       int *h_n_inliers) {
    NvtxRange nvtx_call("sr_fit_alpha");
    if (!c || !d_disp || !h_pairs || !h_alpha || n_hyp < 1 || n_hyp > (1 << 16) ||
        !(tau_px >= 0.0f) || !isfinite(tau_px))
        return SR_ERR_INVALID_ARG;
    const int W = c->p.width, H = c->p.height;
    const int nb = sr::fit_blocks((long long)W * H);
    if (!c->f_partial) SR_TRY(c, dalloc(&c->f_partial, (size_t)nb * 9 + 9), "cudaMalloc(fit partials)");
    if (n_hyp > c->fit_cap) {
        cudaFree(c->f_pairs); cudaFree(c->f_has); cudaFree(c->f_counts); cudaFree(c->f_model);
        c->f_pairs = c->f_has = c->f_counts = nullptr;
        c->f_model = nullptr;
        c->fit_cap = 0;
        SR_TRY(c, dalloc(&c->f_pairs, 2 * (size_t)n_hyp), "cudaMalloc(fit pairs)");
        SR_TRY(c, dalloc(&c->f_has, n_hyp), "cudaMalloc(fit)");
        SR_TRY(c, dalloc(&c->f_counts, n_hyp), "cudaMalloc(fit)");
        SR_TRY(c, dalloc(&c->f_model, n_hyp), "cudaMalloc(fit)");
        c->fit_cap = n_hyp;
    }
    cudaStream_t st = c->st;
    SR_TRY(c, cudaMemcpyAsync(c->f_pairs, h_pairs, 2 * (size_t)n_hyp * sizeof(int32_t),
                              cudaMemcpyHostToDevice, st), "H2D pairs");
    SR_TRY(c, sr::launch_fit_count(d_disp, W, H, c->f_pairs, n_hyp, tau_px, c->f_model, c->f_has,
                                   c->f_counts, st), "fit count");
    std::vector<int> counts(n_hyp), has(n_hyp);
    SR_TRY(c, cudaMemcpyAsync(counts.data(), c->f_counts, n_hyp * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
    SR_TRY(c, cudaMemcpyAsync(has.data(), c->f_has, n_hyp * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
    SR_TRY(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    int best = -1, best_n = -1;
    for (int h = 0; h < n_hyp; ++h) {
        if (!has[h]) { counts[h] = -1; continue; }
        if (counts[h] > best_n) { best_n = counts[h]; best = h; }
    }
    if (h_counts) memcpy(h_counts, counts.data(), n_hyp * sizeof(int32_t));
    if (h_best) *h_best = best;
    if (h_n_inliers) *h_n_inliers = best_n < 0 ? 0 : best_n;
    if (best < 0) {
        snprintf(c->err, sizeof(c->err), "sr_fit_alpha: no hypothesis has a model");
        return SR_ERR_STATE;
    }
    float2 m;
    SR_TRY(c, cudaMemcpy(&m, c->f_model + best, sizeof(float2), cudaMemcpyDeviceToHost), "D2H model");
    double *sums = c->f_partial + (size_t)nb * 9;
    SR_TRY(c, sr::launch_fit_ls(d_disp, W, H, m.x, m.y, tau_px, c->f_partial, sums, st), "fit ls");
    double s[5];
    SR_TRY(c, cudaMemcpyAsync(s, sums, sizeof(s), cudaMemcpyDeviceToHost, st), "D2H sums");
    SR_TRY(c, cudaStreamSynchronize(st), "cudaStreamSynchronize");
    // normal equations of d = a0 + a1 v: [n sv; sv svv] a = [sd; svd]
    const double det = s[0] * s[2] - s[1] * s[1];
    if (det == 0.0) {
        snprintf(c->err, sizeof(c->err), "sr_fit_alpha: inliers span fewer than two rows");
        return SR_ERR_STATE;
    }
    h_alpha[1] = (s[0] * s[4] - s[1] * s[3]) / det;
    h_alpha[0] = (s[3] - h_alpha[1] * s[1]) / s[0];
    return take_device_error(c);
}

sr_status sr_fit_roll(sr_ctx *c, const float *d_disp, int u_lo, int v_lo, int u_hi, int v_hi,
                      double *h_gamma, double *h_roll, int *h_n) {
    NvtxRange nvtx_call("sr_fit_roll");
    if (!c || !d_disp || !h_gamma || !h_roll) return SR_ERR_INVALID_ARG;
    const int W = c->p.width, H = c->p.height;
    u_lo = std::max(u_lo, 0); v_lo = std::max(v_lo, 0);
    u_hi = std::min(u_hi, W); v_hi = std::min(v_hi, H);
    if (u_lo >= u_hi || v_lo >= v_hi) return SR_ERR_INVALID_ARG;
    const int nb = sr::fit_blocks((long long)W * H);
    if (!c->f_partial) SR_TRY(c, dalloc(&c->f_partial, (size_t)nb * 9 + 9), "cudaMalloc(fit partials)");
    double *sums = c->f_partial + (size_t)nb * 9;
    SR_TRY(c, sr::launch_roll_sums(d_disp, W, u_lo, v_lo, u_hi, v_hi, c->f_partial, sums, c->st),
           "roll sums");
    double s[9];
    SR_TRY(c, cudaMemcpyAsync(s, sums, sizeof(s), cudaMemcpyDeviceToHost, c->st), "D2H sums");
    SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
    if (h_n) *h_n = (int)s[0];
    // normal equations of d = g0 + g1 u + g2 v, Gaussian elimination with
    // partial pivoting
    double A[3][4] = {{s[0], s[1], s[2], s[6]}, {s[1], s[3], s[4], s[7]}, {s[2], s[4], s[5], s[8]}};
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) {
            snprintf(c->err, sizeof(c->err), "sr_fit_roll: singular patch (too few rows or columns)");
            return SR_ERR_STATE;
        }
        if (piv != col)
            for (int k = 0; k < 4; ++k) std::swap(A[col][k], A[piv][k]);
        for (int r = col + 1; r < 3; ++r) {
            const double f = A[r][col] / A[col][col];
            for (int k = col; k < 4; ++k) A[r][k] -= f * A[col][k];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double t = A[r][3];
        for (int k = r + 1; k < 3; ++k) t -= A[r][k] * h_gamma[k];
        h_gamma[r] = t / A[r][r];
    }
    *h_roll = atan(-h_gamma[1] / h_gamma[2]);
    return take_device_error(c);
}

sr_status sr_get_buffer(sr_ctx *c, sr_buffer which, void *dst, size_t *bytes_inout) {
    if (!c || !dst || !bytes_inout) return SR_ERR_INVALID_ARG;
    const size_t npx = (size_t)c->p.width * c->p.height, D = c->p.max_disp;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (which) {
        case SR_BUF_WARPED: src = c->rw; bytes = npx * 4; break;
        case SR_BUF_MU_L: case SR_BUF_MU_R: case SR_BUF_INV_L: case SR_BUF_INV_R: {
            // stored with D-1 extra block centres per row; copy the in-image ones
            if (*bytes_inout < npx * 4) { *bytes_inout = npx * 4; return SR_ERR_INVALID_ARG; }
            if (!c->matched) return SR_ERR_STATE;
            const size_t WE = c->p.width + D - 1;
            const float *base = which == SR_BUF_INV_L ? c->inv_l
                              : which == SR_BUF_MU_L  ? c->mu_l
                              : which == SR_BUF_INV_R ? c->inv_r + (D - 1)
                                                      : c->mu_r + (D - 1);
            SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
            SR_TRY(c, cudaMemcpy2D(dst, c->p.width * 4, base, WE * 4, c->p.width * 4, c->p.height,
                                   cudaMemcpyDefault),
                   "cudaMemcpy2D");
            *bytes_inout = npx * 4;
            return SR_OK;
        }
        case SR_BUF_COST_L: case SR_BUF_COST_R: {
            const size_t n = npx * D;
            if (*bytes_inout < n * 4) { *bytes_inout = n * 4; return SR_ERR_INVALID_ARG; }
            if (!c->matched) return SR_ERR_STATE;
            // After sr_match both views live in the extended reference volume
            // (row pitch W + D - 1; the target cost (u, d) is its column
            // u + d); after sr_match_restricted each view has its own volume.
            const bool ext = c->vol_ext;
            const size_t W = c->p.width, H = c->p.height, pitch = ext ? W + D - 1 : W;
            const bool tgt = which == SR_BUF_COST_R;
            const void *v = (ext || !tgt) ? c->vol_l : c->vol_r;
            const size_t m = H * pitch * D;   // elements of the source volume
            SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
            // the source widened to float on the host, then the view's elements
            float *wide = (float *)malloc(m * 4);
            float *view = ext ? (float *)malloc(n * 4) : wide;
            uint16_t *raw = c->p.vol_dtype == SR_VOL_F32 ? nullptr : (uint16_t *)malloc(m * 2);
            if (!wide || !view || (c->p.vol_dtype != SR_VOL_F32 && !raw)) {
                free(wide); if (ext) free(view); free(raw);
                return SR_ERR_OOM;
            }
            cudaError_t e;
            if (raw) {
                e = cudaMemcpy(raw, v, m * 2, cudaMemcpyDeviceToHost);
                for (size_t i = 0; e == cudaSuccess && i < m; ++i)
                    wide[i] = c->p.vol_dtype == SR_VOL_F16 ? half_bits_to_float(raw[i])
                                                           : bf16_bits_to_float(raw[i]);
            } else {
                e = cudaMemcpy(wide, v, m * 4, cudaMemcpyDeviceToHost);
            }
            if (e == cudaSuccess && ext)
                for (size_t y = 0; y < H; ++y)
                    for (size_t u = 0; u < W; ++u)
                        for (size_t d = 0; d < (size_t)D; ++d)
                            view[(y * W + u) * D + d] = wide[(y * pitch + u + (tgt ? d : 0)) * D + d];
            if (e == cudaSuccess) e = cudaMemcpy(dst, view, n * 4, cudaMemcpyDefault);
            free(wide);
            if (ext) free(view);
            free(raw);
            if (e != cudaSuccess) return fail_cuda(c, e, "cudaMemcpy(volume)");
            *bytes_inout = n * 4;
            return take_device_error(c);
        }
        case SR_BUF_AGG_L: src = c->agg_valid ? c->agg_l : nullptr; bytes = npx * D * 4; break;
        case SR_BUF_AGG_R: src = c->agg_valid ? c->agg_r : nullptr; bytes = npx * D * 4; break;
        case SR_BUF_WTA_L: src = c->lbl_l; bytes = npx * 2; break;
        case SR_BUF_WTA_R: src = c->lbl_r; bytes = npx * 2; break;
        case SR_BUF_DSUB: src = c->dsub; bytes = npx * 4; break;
        default: return SR_ERR_INVALID_ARG;
    }
    if (*bytes_inout < bytes) { *bytes_inout = bytes; return SR_ERR_INVALID_ARG; }
    if (!c->matched || !src) return SR_ERR_STATE;
    SR_TRY(c, cudaStreamSynchronize(c->st), "cudaStreamSynchronize");
    SR_TRY(c, cudaMemcpy(dst, src, bytes, cudaMemcpyDefault), "cudaMemcpy");
    *bytes_inout = bytes;
    return take_device_error(c);
}

}  // extern "C"

// ---- bounds-checked build: host record of offences (see sr_internal.cuh) ----
#ifdef SR_BOUNDS_CHECK
#include <mutex>
namespace sr {
namespace {
std::mutex g_oob_mu;
unsigned long long g_oob_word = 0;   // first offence since the last report
long long g_oob_count = 0;
char g_oob_unit[160] = {0};
}  // namespace
void oob_record(unsigned long long word, const char *unit) {
    std::lock_guard<std::mutex> lk(g_oob_mu);
    if (g_oob_word == 0) {
        g_oob_word = word;
        snprintf(g_oob_unit, sizeof(g_oob_unit), "%s", unit ? unit : "");
    }
    ++g_oob_count;
    SR_LOG(1, "bounds check: site %d, index %lld (%s)", (int)((word >> 48) & 0x7fff),
           (long long)(word & 0xffffffffffffull), unit ? unit : "");
}
}  // namespace sr
#endif

extern "C" sr_status sr_bounds_report(int *site, long long *index, char *unit, int unit_len,
                                      long long *count) {
#ifndef SR_BOUNDS_CHECK
    (void)site; (void)index; (void)unit; (void)unit_len; (void)count;
    return SR_ERR_UNSUPPORTED;
#else
    std::lock_guard<std::mutex> lk(sr::g_oob_mu);
    const unsigned long long w = sr::g_oob_word;
    if (site) *site = w ? (int)((w >> 48) & 0x7fff) : -1;
    if (index) {
        // the 48-bit index field, sign-extended
        long long i = (long long)(w & 0xffffffffffffull);
        if (i & (1ll << 47)) i -= (1ll << 48);
        *index = w ? i : 0;
    }
    if (unit && unit_len > 0) snprintf(unit, (size_t)unit_len, "%s", w ? sr::g_oob_unit : "");
    if (count) *count = sr::g_oob_count;
    sr::g_oob_word = 0;
    sr::g_oob_count = 0;
    sr::g_oob_unit[0] = 0;
    return w ? SR_ERR_BOUNDS : SR_OK;
#endif
}
