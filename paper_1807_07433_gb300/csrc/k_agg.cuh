// k_agg.cuh -- Eqs. 8-10 bilateral cost aggregation fused with WTA
// (Sec. II-B-3) and the Eq. 12 parabola.
//
// c_agg(u,v,d) = sum_k w_k(u,v) c(u+dx_k, v+dy_k, d) / sum_k w_k(u,v),
// w_k = exp(-(dx^2+dy^2)/gamma_d^2) * exp(-(g(u+dx,v+dy)-g(u,v))^2/gamma_r^2),
// neighbours outside the image excluded.  The weights do not depend on d.
//
// Work decomposition (FP32 FMA-bound: 2*(2R+1)^2 flop per (u,v,d)):
//   * a CTA owns a 32 x 4 pixel tile and ALL D disparities, so WTA and the
//     parabola finish in the CTA and the aggregated volume never reaches HBM;
//   * the weights of the tile's 128 pixels are computed once into shared
//     memory (rows padded to a multiple of 4 for 128-bit loads);
//   * the cost rows of the tile (+R halo columns) stream through a
//     double-buffered shared-memory ring, one image row at a time, with
//     asynchronous 16-byte copies (cp.async, zero-filled outside the image);
//   * lane = pair of disparities (float2), D/2 lanes share one 8 x 4 pixel
//     block, so the weights a lane needs are the same for all those lanes
//     (shared-memory broadcast);
//   * each thread accumulates 8 x 4 pixels x 2 disparities = 64 sums.  For
//     every streamed source row it loads the (8+2R) cost pairs of the row
//     into registers once and reuses each for up to (2R+1) pixels x up to
//     4 output rows: ~10 FMAs per shared-memory cost load;
//   * epilogue: the sums are transposed through shared memory so that each
//     lane scans the D costs of one pixel: argmax (ties to the smallest d),
//     then Eq. 12 on the neighbours of the winner.  The normalisation by
//     sum_k w_k is a positive per-pixel scale, which changes neither the
//     argmax nor the parabola vertex, so it is applied only when the
//     aggregated volume is exported.
#pragma once
#include "sr_internal.cuh"

namespace sr {

constexpr int kAggTX = 32, kAggTY = 4, kAggPX = 8, kAggPix = kAggTX * kAggTY;

template <int R, int D>
struct AggCfg {
    static constexpr int SLOTS = D / 2;            // lanes per pixel group
    static constexpr int G = 32 / SLOTS;           // pixel groups per warp
    static constexpr int NW = 4 / G;               // warps per CTA
    static constexpr int NT = 32 * NW;
    static constexpr int WS = 2 * R + 1;           // window side
    static constexpr int WP = (WS + 3) / 4 * 4;    // padded weight row
    static constexpr int PS = WS * WP;             // weight floats per pixel
    static constexpr int TXE = kAggTX + 2 * R;     // ring row width (pixels)
    static constexpr int TYE = kAggTY + 2 * R;     // source rows per tile
    static constexpr int RING = TXE * D;           // floats per ring slot
    static constexpr int WTS = kAggTY * (kAggTX * PS + 16);  // + bank skew
    static constexpr int EPI = kAggPix * (D + 1);  // epilogue transpose
    static constexpr int UNION = WTS > EPI ? WTS : EPI;
    static constexpr int GUIDE = TYE * TXE;
    static constexpr size_t SMEM =
        sizeof(float) * (2 * RING + UNION + ((GUIDE + 3) / 4 * 4) + kAggPix);
    static_assert(D == 16 || D == 32 || D == 64, "D must be 16, 32 or 64");
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;   // 0 source bytes => 16 zero bytes written
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Weight offset (floats) of pixel (py, px) of the tile.  Block column
// px/8 adds a 16-byte skew so that pixel groups of one warp that read the
// weights of different blocks hit different shared-memory banks; each pixel
// row gets 16 spare floats so that the skew never runs into the next row.
__device__ __forceinline__ int wts_index(int py, int px, int PS) {
    return py * (kAggTX * PS + 16) + px * PS + 4 * (px >> 3);
}

template <int R, int D, bool GU8>
__global__ void __launch_bounds__(AggCfg<R, D>::NT)
k_agg_wta(const float *__restrict__ vol, const uint8_t *__restrict__ gl, int pitch,
          const float *__restrict__ gf, int W, int H, float kd, float kr,
          int16_t *__restrict__ lbl, float *__restrict__ dsub, float *__restrict__ agg) {
    using C = AggCfg<R, D>;
    extern __shared__ __align__(16) float smem[];
    float *ring = smem;                          // [2][TXE][D]
    float *wts = ring + 2 * C::RING;             // [128][PS] (+skew); reused by epilogue
    float *guide = wts + C::UNION;               // [TYE][TXE]
    float *wsum = guide + (C::GUIDE + 3) / 4 * 4;  // [128]

    const int x0 = blockIdx.x * kAggTX, y0 = blockIdx.y * kAggTY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    auto load_row = [&](int j) {   // source row j of the tile -> ring slot j&1
        const int y = y0 - R + j;
        if (y < 0 || y >= H) return;
        float *dst = ring + (j & 1) * C::RING;
        const float *src_row = vol + (size_t)y * W * D;
        constexpr int CH = C::RING / 4;
        for (int i = tid; i < CH; i += C::NT) {
            const int c = (i * 4) / D;            // tile column of this chunk
            const int x = x0 - R + c;
            const bool ok = (x >= 0) && (x < W);
            const int xc = clampi(x, 0, W - 1);
            cp_async16(dst + i * 4, src_row + (size_t)xc * D + (i * 4) % D, ok);
        }
    };

    // ---- prologue: guide tile, first cost row, weights ---------------------
    for (int i = tid; i < C::GUIDE; i += C::NT) {
        const int r = i / C::TXE, c = i % C::TXE;
        const int y = y0 - R + r, x = x0 - R + c;
        float g = 0.0f;
        if (y >= 0 && y < H && x >= 0 && x < W)
            g = GU8 ? (float)gl[(size_t)y * pitch + x] : gf[(size_t)y * W + x];
        guide[i] = g;
    }
    load_row(0);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    __syncthreads();

    for (int p = tid; p < kAggPix; p += C::NT) {
        const int py = p / kAggTX, px = p % kAggTX;
        const int u = x0 + px, v = y0 + py;
        const bool pin = (u < W) && (v < H);
        const float gc = guide[(py + R) * C::TXE + px + R];
        float *wp = wts + wts_index(py, px, C::PS);
        float s = 0.0f;
        for (int dyi = 0; dyi < C::WS; ++dyi) {
            const int y = v + dyi - R;
            const bool yin = pin && (y >= 0) && (y < H);
            const float *grow = guide + (py + dyi) * C::TXE + px;
#pragma unroll
            for (int dxi = 0; dxi < C::WP; ++dxi) {
                float w = 0.0f;
                const int x = u + dxi - R;
                if (dxi < C::WS && yin && x >= 0 && x < W) {
                    const float dg = grow[dxi] - gc;
                    const float r2 = (float)((dxi - R) * (dxi - R) + (dyi - R) * (dyi - R));
                    w = exp2f(-fmaf(r2, kd, dg * dg * kr));   // Eq. 9 x Eq. 10
                }
                wp[dyi * C::WP + dxi] = w;
                s += w;
            }
        }
        wsum[p] = s > 0.0f ? s : 1.0f;
    }
    cp_async_wait_all();
    __syncthreads();

    // ---- main loop: stream the tile's source rows --------------------------
    const int sl = lane % C::SLOTS, grp = lane / C::SLOTS;
    const int bcol = warp * C::G + grp;          // 8-pixel block column, 0..3
    const int bx = bcol * kAggPX;                // first tile column of the block

    float2 acc[kAggTY][kAggPX];
#pragma unroll
    for (int py = 0; py < kAggTY; ++py)
#pragma unroll
        for (int px = 0; px < kAggPX; ++px) acc[py][px] = make_float2(0.0f, 0.0f);

#pragma unroll 1
    for (int j = 0; j < C::TYE; ++j) {
        if (j + 1 < C::TYE) load_row(j + 1);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        const int y = y0 - R + j;
        if (y >= 0 && y < H) {
            const float *rs = ring + (j & 1) * C::RING + bx * D + 2 * sl;
            float2 cst[kAggPX + 2 * R];
#pragma unroll
            for (int i = 0; i < kAggPX + 2 * R; ++i)
                cst[i] = *reinterpret_cast<const float2 *>(rs + i * D);
#pragma unroll
            for (int py = 0; py < kAggTY; ++py) {
                const int dyi = j - py;
                if (dyi >= 0 && dyi < C::WS) {
                    const float *wrow = wts + wts_index(py, bx, C::PS) + dyi * C::WP;
#pragma unroll
                    for (int px = 0; px < kAggPX; ++px) {
                        float w[C::WP];
#pragma unroll
                        for (int q = 0; q < C::WP; q += 4) {
                            const float4 t = *reinterpret_cast<const float4 *>(wrow + px * C::PS + q);
                            w[q] = t.x; w[q + 1] = t.y; w[q + 2] = t.z; w[q + 3] = t.w;
                        }
                        float2 a = acc[py][px];
#pragma unroll
                        for (int dx = 0; dx < C::WS; ++dx) {
                            a.x = fmaf(w[dx], cst[px + dx].x, a.x);
                            a.y = fmaf(w[dx], cst[px + dx].y, a.y);
                        }
                        acc[py][px] = a;
                    }
                }
            }
        }
        cp_async_wait_all();
        __syncthreads();
    }

    // ---- epilogue: transpose, WTA, parabola ---------------------------------
    float *E = wts + warp * (32 * C::G) * (D + 1);     // this warp's pixels x D
#pragma unroll
    for (int py = 0; py < kAggTY; ++py)
#pragma unroll
        for (int px = 0; px < kAggPX; ++px) {
            float *e = E + (grp * 32 + py * kAggPX + px) * (D + 1) + 2 * sl;
            e[0] = acc[py][px].x;
            e[1] = acc[py][px].y;
        }
    __syncwarp();
    for (int pw = lane; pw < 32 * C::G; pw += 32) {
        const int g = pw >> 5, py = (pw & 31) / kAggPX, px = pw % kAggPX;
        const int tpx = (warp * C::G + g) * kAggPX + px;
        const int u = x0 + tpx, v = y0 + py;
        if (u >= W || v >= H) continue;
        const float *e = E + pw * (D + 1);
        int best = 0;
        float cb = e[0];
#pragma unroll 8
        for (int d = 1; d < D; ++d) {
            const float c = e[d];
            if (c > cb) { cb = c; best = d; }
        }
        const size_t o = (size_t)v * W + u;
        lbl[o] = (int16_t)best;
        if (dsub) {
            float ds = (float)best;
            if (best > 0 && best < D - 1) {
                const float cm = e[best - 1], cp = e[best + 1];
                const float den = 2.0f * cm + 2.0f * cp - 4.0f * cb;
                if (den < 0.0f) ds += (cm - cp) / den;
            }
            dsub[o] = ds;
        }
    }
    if (agg) {
        for (int pw = 0; pw < 32 * C::G; ++pw) {
            const int g = pw >> 5, py = (pw & 31) / kAggPX, px = pw % kAggPX;
            const int tpx = (warp * C::G + g) * kAggPX + px;
            const int u = x0 + tpx, v = y0 + py;
            if (u >= W || v >= H) continue;
            const float sc = 1.0f / wsum[py * kAggTX + tpx];
            for (int d = lane; d < D; d += 32)
                agg[((size_t)v * W + u) * D + d] = E[pw * (D + 1) + d] * sc;
        }
    }
}

template <int R, int D>
cudaError_t agg_launch_t(const float *vol, const uint8_t *gl, int pitch, const float *gf, int W,
                         int H, float kd, float kr, int16_t *lbl, float *dsub, float *agg,
                         cudaStream_t st) {
    using C = AggCfg<R, D>;
    const dim3 grid((W + kAggTX - 1) / kAggTX, (H + kAggTY - 1) / kAggTY);
    if (gl) {
        auto k = k_agg_wta<R, D, true>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        k<<<grid, C::NT, C::SMEM, st>>>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg);
    } else {
        auto k = k_agg_wta<R, D, false>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        k<<<grid, C::NT, C::SMEM, st>>>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg);
    }
    return cudaGetLastError();
}

template <int D>
cudaError_t agg_launch_d(const float *vol, const uint8_t *gl, int pitch, const float *gf, int W,
                         int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub,
                         float *agg, cudaStream_t st) {
    switch (agg_r) {
        case 1: return agg_launch_t<1, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 2: return agg_launch_t<2, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 3: return agg_launch_t<3, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 4: return agg_launch_t<4, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 5: return agg_launch_t<5, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 6: return agg_launch_t<6, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        case 7: return agg_launch_t<7, D>(vol, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sr
