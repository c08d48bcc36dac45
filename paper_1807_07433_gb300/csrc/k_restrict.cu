// k_restrict.cu -- tile bands of the restricted search (the paper's Sec. IV
// plan: aggregate only around previously calculated disparities).
//
// Each 32 x 4 aggregation tile gets the start of one kBandD-disparity slice
// that holds the search window of every pixel of the tile, or -1 when the
// windows span more than the slice (those tiles run the full-D kernel).  The
// start is aligned to 16 bytes of the stored cost type, as the tensor-map
// copies of the band kernel need.
#include "sr_internal.cuh"

namespace sr {
namespace {

constexpr int kTileTX = 32, kTileTY = 4;   // the aggregation tile

__global__ void __launch_bounds__(kTileTX * kTileTY)
k_tile_bands(AggWin win, int W, int H, int align, int *__restrict__ band) {
    __shared__ int s_lo[kTileTX * kTileTY / 32], s_hi[kTileTX * kTileTY / 32];
    const int u = blockIdx.x * kTileTX + threadIdx.x % kTileTX;
    const int v = blockIdx.y * kTileTY + threadIdx.x / kTileTX;
    int lo = 1 << 30, hi = -1;
    if (u < W && v < H) {
        int c = win.centre ? win.centre[(size_t)v * W + u] : win.centre_const;
        c = min(max(c, 0), win.dfull - 1);
        lo = max(c - win.radius, 0);
        hi = min(c + win.radius, win.dfull - 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { s_lo[threadIdx.x >> 5] = lo; s_hi[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kTileTX * kTileTY / 32; ++w) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
        }
        int b = lo / align * align;
        b = min(b, win.dfull - kBandD);          // dfull - kBandD is a multiple of align
        band[blockIdx.y * gridDim.x + blockIdx.x] =
            (win.dfull > kBandD && b >= 0 && hi <= b + kBandD - 1) ? b : -1;
    }
}

__global__ void k_ncc_ranges(const int *__restrict__ band, int tx, int ty, int D, int reach_y,
                             int2 *__restrict__ range) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tx * ty) return;
    const int bx = t % tx, by = t / tx;
    int lo = D, hi = -1;
    // aggregation tiles within one tile column (agg_r < 32) and reach_y tile
    // rows read this tile's costs
    for (int y = max(by - reach_y, 0); y <= min(by + reach_y, ty - 1); ++y)
        for (int x = max(bx - 1, 0); x <= min(bx + 1, tx - 1); ++x) {
            const int b = band[y * tx + x];
            if (b < 0) { lo = 0; hi = D - 1; }
            else { lo = min(lo, b); hi = max(hi, b + kBandD - 1); }
        }
    range[t] = make_int2(lo, hi);
}

}  // namespace

cudaError_t launch_ncc_ranges(const int *band, int W, int H, int D, int agg_r, int2 *range,
                              cudaStream_t st) {
    const int tx = (W + kTileTX - 1) / kTileTX, ty = (H + kTileTY - 1) / kTileTY;
    const int reach_y = (agg_r + kTileTY - 1) / kTileTY;
    k_ncc_ranges<<<(tx * ty + 255) / 256, 256, 0, st>>>(band, tx, ty, D, reach_y, range);
    return cudaGetLastError();
}

cudaError_t launch_tile_bands(const AggWin &win, int W, int H, int align, int *band,
                              cudaStream_t st) {
    const dim3 grid((W + kTileTX - 1) / kTileTX, (H + kTileTY - 1) / kTileTY);
    k_tile_bands<<<grid, kTileTX * kTileTY, 0, st>>>(win, W, H, align, band);
    return cudaGetLastError();
}

}  // namespace sr
