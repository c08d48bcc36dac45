// k_ncc.cuh -- Eq. 3 NCC cost volumes.
//
// One thread per output pixel (u,v) computes all D costs of that pixel.
//   reference volume: c(u,v,d) = NCC(left block at u, warped-target block at u-d)
//   target volume:    c(u,v,d) = NCC(left block at u+d, warped-target block at u)
// (the two volumes of Sec. II-B-1; c of the reference volume at (u,v,d) equals
// c of the target volume at (u-d,v,d)).  The reference kernel also runs on
// an extended output width Wo = W + D - 1: block centres u in [W, W + D - 1)
// are clamp-to-edge blocks like any other, and that one extended volume
// holds both (target c(u,v,d) = extended reference c(u+d,v,d)); entries with
// u - d >= W are computed from clamped statistics and never read.
//
// Numerics.  The numerator of Eq. 3, sum(i_l i_r) - n mu_l mu_r, equals
// sum((f - mu_f) * (s - K)) for ANY constant K when f is the block that stays
// fixed while d varies and s the block that slides.  The fixed block is
// centred once per pixel (49 registers for a 7x7 block), the sliding block is
// offset by K = 128, so no large terms cancel.  The centred values a_i carry
// the rounding error e of the FP32 mean; to first order it adds
// -e * sum(s - K) = (sum a_i) * n(mu_s - K) / n, so the kernel subtracts
// (sum a_i) * (mu_s - K) using the sliding block's mean.  The result keeps
// ~1e-7 relative accuracy even on near-flat blocks, where the textbook form
// loses ~1e-5 and the uncorrected centred form ~1e-3.
//
// Work per pixel: the dot products of all D disparities are organised by
// sliding-image COLUMN: column c contributes sum_oy a[oy][ox] * s(c, v+oy) to
// disparity d = (u - c) + ox - r (reference) or (c - u) - ox + r (target) for
// each block column ox.  Each column of the sliding block is read from shared
// memory once (2r+1 loads) and feeds up to (2r+1)^2 FMAs, so the kernel is
// FMA-bound rather than shared-memory-bound.  Disparities are processed in
// chunks of DC (16 or 32, see NccOcc) so that the accumulators stay in
// registers.
//
// Tiles: 32 x 4 output pixels per CTA (128 threads); the fixed image tile and
// the sliding image tile (widened by D-1 columns) are staged in shared memory
// with clamp-to-edge reads, as the block definition of Eqs. 3-5 requires.
// The per-tile work is one device function, used by the single-image kernel
// (one tile per CTA) and by the batched kernel (a persistent CTA walks the
// flat (pair, tile) list of a batch).
#pragma once
#include "sr_internal.cuh"

namespace sr {

constexpr int kNccTX = 32, kNccTY = 4, kNccThreads = kNccTX * kNccTY;

// Register budget by block radius.  At 5 x 5 and 7 x 7 blocks a
// 16-disparity chunk of accumulators leaves room for seven CTAs per SM (at
// most 72 registers; 7 x 7 measured 13 % faster than 32-disparity chunks at
// five CTAs).  3 x 3 blocks fit many CTAs anyway, and 9 x 9 and 11 x 11
// blocks (81 and 121 centred values in registers) keep 32-disparity chunks
// and the compiler's own budget: a bound would spill them, and narrower
// chunks made the compiler unroll into twice the registers.
template <int RN>
struct NccOcc {
    static constexpr bool NARROW = RN == 2 || RN == 3;
    static constexpr int DC = NARROW ? 16 : 32;    // disparity chunk (at most D)
    static constexpr int MINB = NARROW ? 7 : 0;    // CTAs per SM of k_ncc (0: no bound)
};

template <int RN, int D>
struct NccSmem {
    static constexpr int B = 2 * RN + 1;
    static constexpr int FW = kNccTX + 2 * RN;          // fixed tile width
    static constexpr int SW = kNccTX + 2 * RN + D - 1;  // sliding tile width
    static constexpr int TH = kNccTY + 2 * RN;          // tile height
    static constexpr int XW = kNccTX + D - 1;           // sliding-block centres per tile row
    float fix_s[TH][FW];
    float sld_s[TH][SW];
    float2 sst_s[kNccTY][XW];                           // sliding block: (mean - K, 1/(n sigma))
};

// One 32 x 4 tile at (x0, y0).  All threads of the CTA take part (barrier).
template <int RN, int D, bool TARGET, typename VT>
__device__ __forceinline__ void ncc_tile(NccSmem<RN, D> &sm, const uint8_t *__restrict__ left,
                                         int pitch, const float *__restrict__ rw,
                                         const float *__restrict__ mu_l,
                                         const float *__restrict__ inv_l,
                                         const float *__restrict__ mu_r,
                                         const float *__restrict__ inv_r, int W, int H,
                                         VT *__restrict__ vol, int Wo, int x0, int y0,
                                         int dlo = 0, int dhi = D - 1) {
    using S = NccSmem<RN, D>;
    constexpr int B = S::B, FW = S::FW, SW = S::SW, TH = S::TH, XW = S::XW;
    // disparity chunk held in registers (see NccOcc)
    constexpr int DC = D < NccOcc<RN>::DC ? D : NccOcc<RN>::DC;
    const int tid = threadIdx.x;
    const int WE = W + D - 1;

    // This pixel's fixed-block statistics, loaded first so that their latency
    // overlaps the staging below.
    const int tx = tid % kNccTX, ty = tid / kNccTX;
    const int u = x0 + tx, v = y0 + ty;
    const bool inside = u < Wo && v < H;
    const size_t rowo = (size_t)(inside ? v : 0) * WE;
    const int uc = inside ? u : 0;
    const size_t fo = rowo + uc + (TARGET ? D - 1 : 0);   // statistics rows are H x WE
    const bool fok = SR_CHECK(fo, (long long)H * WE, 101);
    const float m = !fok ? 0.0f : TARGET ? mu_r[fo] : mu_l[fo];
    const float inv_f0 = !fok ? 0.0f : TARGET ? inv_r[fo] : inv_l[fo];

    // Stage the fixed and sliding tiles (clamp-to-edge).
    const int fx0 = x0 - RN;
    const int sx0 = TARGET ? x0 - RN : x0 - RN - (D - 1);
    for (int i = tid; i < TH * FW; i += kNccThreads) {
        const int r = i / FW, c = i % FW;
        const int y = clampi(y0 - RN + r, 0, H - 1), x = clampi(fx0 + c, 0, W - 1);
        if (!SR_CHECK(x, TARGET ? W : pitch, 102) || !SR_CHECK(y, H, 102)) continue;
        sm.fix_s[r][c] = TARGET ? rw[(size_t)y * W + x] : (float)left[(size_t)y * pitch + x];
    }
    for (int i = tid; i < TH * SW; i += kNccThreads) {
        const int r = i / SW, c = i % SW;
        const int y = clampi(y0 - RN + r, 0, H - 1), x = clampi(sx0 + c, 0, W - 1);
        if (!SR_CHECK(x, TARGET ? pitch : W, 103) || !SR_CHECK(y, H, 103)) continue;
        const float val = TARGET ? (float)left[(size_t)y * pitch + x] : rw[(size_t)y * W + x];
        sm.sld_s[r][c] = val - kNccOffset;
    }
    // Sliding-block statistics of the tile's rows.  In the extended stats rows
    // (see launch_stats) the centres u-d (reference) and u+d (target) of the
    // tile's pixels both occupy the index range [x0, x0 + 32 + D - 1).
    {
        const float *mu_s = TARGET ? mu_l : mu_r;
        const float *inv_s = TARGET ? inv_l : inv_r;
        for (int i = tid; i < kNccTY * XW; i += kNccThreads) {
            const int r = i / XW, t = i % XW;
            const int y = clampi(y0 + r, 0, H - 1);
            const int xi = clampi(x0 + t, 0, WE - 1);
            if (!SR_CHECK((size_t)y * WE + xi, (long long)H * WE, 104)) continue;
            sm.sst_s[r][t] = make_float2(mu_s[(size_t)y * WE + xi] - kNccOffset,
                                         inv_s[(size_t)y * WE + xi]);
        }
    }
    __syncthreads();

    if (!inside) return;

    // Statistics rows (block centres extended by D-1 columns, see launch_stats):
    // the fixed block sits at u, the sliding block at u+d (target) / u-d (reference).
    // sliding centre of disparity d at smem index base + so, so = d or -d
    const float2 *st_s_row = &sm.sst_s[ty][TARGET ? tx : tx + D - 1];

    // Centred fixed block and the sum of its (rounded) centred values.
    float a[B][B];
    float sa = 0.0f;
#pragma unroll
    for (int oy = 0; oy < B; ++oy)
#pragma unroll
        for (int ox = 0; ox < B; ++ox) {
            a[oy][ox] = sm.fix_s[ty + oy][tx + ox] - m;
            sa += a[oy][ox];
        }

    // n/(n sigma_f) of the fixed block (Eq. 3 divides n*cov by n*sigma_f*sigma_s).
    constexpr float n = (float)(B * B);
    const float inv_f = n * inv_f0;
    VT *out = vol + ((size_t)v * Wo + u) * D;

#pragma unroll 1
    for (int d0 = 0; d0 < D; d0 += DC) {
        if (d0 + DC <= dlo || d0 > dhi) continue;   // no aggregation tile reads this chunk
        float acc[DC];
#pragma unroll
        for (int i = 0; i < DC; ++i) acc[i] = 0.0f;
        // Sliding column c = u - k (reference) or u + k (target), k = d + (ox - RN)
        // resp. d - (ox - RN); k spans [d0 - RN, d0 + DC - 1 + RN].
#pragma unroll
        for (int kk = 0; kk < DC + 2 * RN; ++kk) {
            const int k = d0 - RN + kk;
            const int sc = TARGET ? tx + k + RN : tx - k + RN + D - 1;
            float col[B];
#pragma unroll
            for (int oy = 0; oy < B; ++oy)
                col[oy] = SR_CHECK(sc, SW, 105) && SR_CHECK(ty + oy, TH, 105) ? sm.sld_s[ty + oy][sc] : 0.0f;
#pragma unroll
            for (int ox = 0; ox < B; ++ox) {
                const int dl = TARGET ? kk - ox : kk + ox - 2 * RN;   // d - d0
                if (dl >= 0 && dl < DC) {
                    float s = acc[dl];
#pragma unroll
                    for (int oy = 0; oy < B; ++oy) s = fmaf(a[oy][ox], col[oy], s);
                    acc[dl] = s;
                }
            }
        }
        // Mean correction, Eq. 3 denominator, store the chunk.
        float cst[DC];
#pragma unroll
        for (int i = 0; i < DC; ++i) {
            const int so = TARGET ? d0 + i : -(d0 + i);
            const float2 ss = SR_CHECK((TARGET ? tx : tx + D - 1) + so, XW, 106) ? st_s_row[so]
                                                                                 : make_float2(0.0f, 0.0f);
            const float num = fmaf(-sa, ss.x, acc[i]);
            cst[i] = num * inv_f * ss.y;
            // extended volume: a sliding centre u - d >= W has no statistics
            // of its own; no cost is taken from there, but readers meet the
            // entry with weight zero, so it is stored as 0 (finite)
            if (!TARGET && u - (d0 + i) >= W) cst[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < DC; i += 8)
            if (SR_CHECK(((size_t)v * Wo + u) * D + d0 + i + 7, (long long)H * Wo * D, 107))
                store8(out + d0 + i, cst + i);
    }
}

template <int RN, int D, bool TARGET, typename VT>
__global__ void __launch_bounds__(kNccThreads, NccOcc<RN>::MINB)
k_ncc(const uint8_t *__restrict__ left, int pitch, const float *__restrict__ rw,
      const float *__restrict__ mu_l, const float *__restrict__ inv_l,
      const float *__restrict__ mu_r, const float *__restrict__ inv_r, int W, int H,
      VT *__restrict__ vol, int Wo, const int2 *__restrict__ range) {
    __shared__ NccSmem<RN, D> sm;
    pdl_trigger();   // a programmatic dependent may launch once every CTA is here
    int dlo = 0, dhi = D - 1;
    if (range) {   // restricted search: the disparities the tile's readers need
        const int2 r = range[blockIdx.y * gridDim.x + blockIdx.x];
        dlo = r.x;
        dhi = r.y;
    }
    ncc_tile<RN, D, TARGET, VT>(sm, left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, vol, Wo,
                                blockIdx.x * kNccTX, blockIdx.y * kNccTY, dlo, dhi);
}

// Persistent batched form: CTA b handles work items b, b + gridDim.x, ...
template <int RN, int D, bool TARGET, typename VT>
__global__ void __launch_bounds__(kNccThreads)
k_ncc_batch(const PairDesc *__restrict__ pairs, const int *__restrict__ start, int n,
            int *__restrict__ next) {
    __shared__ NccSmem<RN, D> sm;
    __shared__ int s_start[kStartSmem];
    __shared__ int s_t;
    const int *st = stage_start(s_start, start, n);
    const int total = st[n];
    int p = 0;
    for (int t = blockIdx.x;; ) {
        __syncthreads();   // the previous tile is done with shared memory
        if (next) {        // in-order work items from a counter, else strided
            if (threadIdx.x == 0) s_t = atomicAdd(next, 1);
            __syncthreads();
            t = s_t;
        }
        if (t >= total) break;
        p = find_pair(st, n, t, p);
        const PairDesc &P = pairs[p];
        const int tl = t - st[p], tx = (P.W + kNccTX - 1) / kNccTX;
        ncc_tile<RN, D, TARGET, VT>(sm, P.left, P.pitch, P.rw, P.mu_l, P.inv_l, P.mu_r, P.inv_r,
                                    P.W, P.H, static_cast<VT *>(TARGET ? P.vol_r : P.vol_l), P.W,
                                    (tl % tx) * kNccTX, (tl / tx) * kNccTY);
        if (!next) t += gridDim.x;
    }
}

template <int RN, int D, typename VT>
cudaError_t ncc_launch_t(bool target, const uint8_t *left, int pitch, const float *rw,
                         const float *mu_l, const float *inv_l, const float *mu_r,
                         const float *inv_r, int W, int H, VT *vol, int Wo, cudaStream_t st,
                         const int2 *range) {
    const dim3 grid((Wo + kNccTX - 1) / kNccTX, (H + kNccTY - 1) / kNccTY);
    if (target)
        k_ncc<RN, D, true, VT><<<grid, kNccThreads, 0, st>>>(left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, vol, Wo, range);
    else
        k_ncc<RN, D, false, VT><<<grid, kNccThreads, 0, st>>>(left, pitch, rw, mu_l, inv_l, mu_r, inv_r, W, H, vol, Wo, range);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

template <int RN, int D, typename VT>
cudaError_t ncc_batch_t(bool target, const PairDesc *pairs, const int *start, int n, int grid,
                        int *next, cudaStream_t st) {
    if (target)
        k_ncc_batch<RN, D, true, VT><<<grid, kNccThreads, 0, st>>>(pairs, start, n, next);
    else
        k_ncc_batch<RN, D, false, VT><<<grid, kNccThreads, 0, st>>>(pairs, start, n, next);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

template <int RN, int D, typename VT>
int ncc_occ_t() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ncc_batch<RN, D, false, VT>, kNccThreads, 0);
    return b;
}

#define SR_NCC_RN_SWITCH(ncc_r, CALL)                \
    switch (ncc_r) {                                 \
        case 1: { constexpr int RN_ = 1; CALL; }     \
        case 2: { constexpr int RN_ = 2; CALL; }     \
        case 3: { constexpr int RN_ = 3; CALL; }     \
        case 4: { constexpr int RN_ = 4; CALL; }     \
        case 5: { constexpr int RN_ = 5; CALL; }     \
        default: break;                              \
    }

template <int D, typename VT>
cudaError_t ncc_launch_d(bool target, const uint8_t *left, int pitch, const float *rw,
                         const float *mu_l, const float *inv_l, const float *mu_r,
                         const float *inv_r, int W, int H, int ncc_r, VT *vol, int Wo,
                         cudaStream_t st, const int2 *range) {
    SR_NCC_RN_SWITCH(ncc_r, return (ncc_launch_t<RN_, D, VT>(target, left, pitch, rw, mu_l, inv_l,
                                                             mu_r, inv_r, W, H, vol, Wo, st, range)))
    return cudaErrorInvalidValue;
}

template <int D, typename VT>
cudaError_t ncc_batch_d(bool target, const PairDesc *pairs, const int *start, int n, int ncc_r,
                        int grid, int *next, cudaStream_t st) {
    SR_NCC_RN_SWITCH(ncc_r, return (ncc_batch_t<RN_, D, VT>(target, pairs, start, n, grid, next, st)))
    return cudaErrorInvalidValue;
}

template <int D, typename VT>
int ncc_occ_d(int ncc_r) {
    SR_NCC_RN_SWITCH(ncc_r, return (ncc_occ_t<RN_, D, VT>()))
    return 0;
}

}  // namespace sr
