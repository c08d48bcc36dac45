// Eqs. 8-12 aggregation/WTA kernels instantiated for D = 32, volumes stored as float.
#include "k_agg.cuh"

namespace sr {
cudaError_t launch_agg_d32_f32(const void *vol, const uint8_t *gl, int pitch, const float *gf, int W, int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub, float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch) {
    return agg_launch_d<32, float, false>(static_cast<const float *>(vol), gl, pitch, gf, W, H, agg_r, kd, kr,
                                   lbl, dsub, agg, dbg, st, win, vpitch);
}
cudaError_t launch_agg_batch_d32_f32(bool target, const PairDesc *pairs, const int *start, int n,
                                  int agg_r, float kd, float kr, const AggDebug &dbg, int grid,
                                  int *next, cudaStream_t st) {
    return agg_batch_d<32, float>(target, pairs, start, n, agg_r, kd, kr, dbg, grid, next, st);
}
int agg_occ_d32_f32(int agg_r) { return agg_occ_d<32, float>(agg_r); }
}  // namespace sr
