// Eq. 3 cost-volume kernels instantiated for D = 64, volumes stored as float.
#include "k_ncc.cuh"

namespace sr {
cudaError_t launch_ncc_d64_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, cudaStream_t st) {
    return ncc_launch_d<64, float>(target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r,
                                   static_cast<float *>(vol), st);
}
}  // namespace sr
