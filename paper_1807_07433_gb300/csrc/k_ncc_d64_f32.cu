// Eq. 3 cost-volume kernels instantiated for D = 64, volumes stored as float.
#include "k_ncc.cuh"

namespace sr {
cudaError_t launch_ncc_d64_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range) {
    return ncc_launch_d<64, float>(target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r,
                                   static_cast<float *>(vol), Wo, st, range);
}
cudaError_t launch_ncc_batch_d64_f32(bool target, const PairDesc *pairs, const int *start, int n,
                                  int ncc_r, int grid, int *next, cudaStream_t st) {
    return ncc_batch_d<64, float>(target, pairs, start, n, ncc_r, grid, next, st);
}
int ncc_occ_d64_f32(int ncc_r) { return ncc_occ_d<64, float>(ncc_r); }
}  // namespace sr
