// Eqs. 8-12 aggregation/WTA kernels with the restricted search's windowed WTA,
// instantiated for D = 64, volumes stored as float.
#include "k_agg.cuh"

namespace sr {
cudaError_t launch_aggw_d64_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch) {
    return agg_launch_d<64, float, true>(static_cast<const float *>(vol), gl, pitch, gf, W, H, agg_r,
                                         kd, kr, lbl, dsub, agg, dbg, st, win, vpitch);
}
}  // namespace sr
