// Eq. 3 cost-volume kernels instantiated for D = 16, volumes stored as float.
#include "k_ncc.cuh"
#include "k_ncc_sl.cuh"

namespace sr {
cudaError_t launch_ncc_d16_f32(bool target, const uint8_t *left, int pitch, const float *rw, const float *mu_l, const float *inv_l, const float *mu_r, const float *inv_r, int W, int H, int ncc_r, void *vol, int Wo, cudaStream_t st, const int2 *range) {
    return ncc_launch_d<16, float>(target, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, ncc_r,
                                   static_cast<float *>(vol), Wo, st, range);
}
cudaError_t launch_ncc_batch_d16_f32(bool target, const PairDesc *pairs, const int *start, int n,
                                  int ncc_r, int grid, int *next, cudaStream_t st) {
    return ncc_batch_d<16, float>(target, pairs, start, n, ncc_r, grid, next, st);
}
int ncc_occ_d16_f32(int ncc_r) { return ncc_occ_d<16, float>(ncc_r); }
cudaError_t launch_ncc_sl_d16_f32(const uint8_t *left, const uint8_t *right, int pitch, int W,
                                  int H, int ncc_r, int row0, double alpha0, double alpha1,
                                  double delta, const float *inv_l, const float *inv_r, void *vol,
                                  int Wo, int seg, cudaStream_t st) {
    return ncc_sl_launch_d<16, float>(left, right, pitch, W, H, ncc_r, row0, alpha0, alpha1, delta,
                                     inv_l, inv_r, static_cast<float *>(vol), Wo, seg, st);
}
int ncc_sl_occ_d16_f32(int ncc_r) { return ncc_sl_occ_d<16, float>(ncc_r); }
}  // namespace sr
