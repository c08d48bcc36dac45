// Band kernels of the restricted search (Eqs. 8-12 on a __nv_bfloat16 volume, 16-disparity slices).
#include "k_agg.cuh"

namespace sr {
cudaError_t launch_agg_band_bf16(const void *tmap, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, const AggDebug &dbg, const AggWin &win, cudaStream_t st) {
    return agg_band_launch_d<__nv_bfloat16>(*static_cast<const CUtensorMap *>(tmap), gl, pitch, gf, W, H,
                                   agg_r, kd, kr, lbl, dsub, dbg, win, st);
}
}  // namespace sr
