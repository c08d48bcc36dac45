// Eqs. 8-12 aggregation/WTA of the target view, read sheared from the
// extended reference volume, instantiated for D = 16, volumes stored as float.
#include "k_agg.cuh"

namespace sr {
cudaError_t launch_aggs_d16_f32(const void *tmap, int vpitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *agg, const AggDebug &dbg, cudaStream_t st) {
    return agg_shear_launch_d<16, float>(*static_cast<const CUtensorMap *>(tmap), vpitch, gf, W, H,
                                       agg_r, kd, kr, lbl, agg, dbg, st);
}
bool aggs_box_d16_f32(int agg_r, int *cw, int *bh) {
    return agg_shear_box_d<16, float>(agg_r, cw, bh);
}
}  // namespace sr
