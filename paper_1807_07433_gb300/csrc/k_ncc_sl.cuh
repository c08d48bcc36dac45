// k_ncc_sl.cuh -- Eq. 3 reference cost volume from exact integer window sums.
//
// c(u,v,d) = N / (n sigma_l sigma_r), N the covariance sum of the left block
// at u and the warped-target block at u - d (Eqs. 3-5).  The warped target is
// a row shift (Sec. II-A): i_r'(x, y) = a(x, y) + w_y delta(x, y) with
// a = i_r(x - k_y), b = i_r(x - k_y - 1) (clamp-to-edge), delta = b - a, and
// k_y, w_y the integer part and the fraction of the row's shift s(y).  With
// uint8 images every term but w_y is an integer, so
//
//   n N = [n SP - Sl Ma] + [n SQ - Sl Mf]
//   SP = sum_block l~ a~,   SQ = sum_rows w_y sum_cols l~ delta,
//   Sl = sum_block l~,      Ma = sum_block a~,   Mf = sum_rows w_y sum_cols delta
//
// for l~ = i_l - o (any integer o) and a~ = a - 128.  The first bracket is an
// exact integer; SP and Ma are sums of integers below 2^24, exact in FP32,
// and the bracket is evaluated without rounding (the rounding error of the
// product Sl Ma is recovered by a fused multiply-add).  Only the second
// bracket, the part that the fractions w_y carry, is rounded.  o is a left
// intensity taken near the thread's columns, which keeps l~, and with it the
// rounding of the second bracket, small on smooth blocks.
//
// Work: the row sums P = sum_cols l~ a~ and Q = sum_cols l~ delta of one
// block row are exact integers; a thread holds them for 4 columns x 8
// disparities and slides them along its 4 columns (2 paired multiply-adds per
// column after the first).  A CTA walks a segment of image rows: each new row
// is added to the window sums {SP, SQ} (one paired multiply-add with
// {1, w_y}) and the row that leaves the window is recomputed and subtracted.
// The window sums are kept in registers, so the volume is written once and
// nothing else is.  SP slides exactly; SQ is rounded once per row added or
// removed, so its last bits depend on where the segment starts.  Segments
// therefore start at fixed image rows, multiples of seg counted from the
// frame's first row (row0 counts a band's first row in its frame), which
// makes a band of rows match the whole frame bit for bit when it starts a
// segment's first row minus the block radius.
//
// A CTA owns TX = 4096/D output columns and all D disparities of a segment
// of rows; thread (ug, db) holds columns x0 + 4 ug .. + 3 and disparities
// 8 db .. 8 db + 7.  Per step it stages one image row (left intensities, a~
// and delta) in a ring of 2r + 2 rows, forms the row's column sums and the
// block-centre statistics Ma, Mf of the output row, adds the new row,
// subtracts the old one and writes the output row.
#pragma once
#include "sr_internal.cuh"

namespace sr {

template <int RN, int D>
struct NslCfg {
    static constexpr int U = kNslU;                 // columns per thread
    static constexpr int DB = kNslDB;               // disparities per thread
    static constexpr int NDB = D / DB;              // disparity blocks
    static constexpr int NUG = kNslThreads / NDB;   // column groups
    static constexpr int TX = NUG * U;              // output columns per CTA
    static constexpr int B = 2 * RN + 1;            // block side
    static constexpr int NR = B + 1;                // staged rows: the window and the row leaving it
    static constexpr int LW = TX + 2 * RN;          // left row: x in [x0 - RN, x0 + TX + RN)
    static constexpr int AW = TX + 2 * RN + D - 1;  // (a~, delta) row: x in [x0 - RN - (D-1), x0 + TX + RN)
    static constexpr int CN = TX + D - 1;           // block centres x in [x0 - (D-1), x0 + TX)
    static constexpr int WIN = U + 2 * RN;          // positions of one thread and disparity
    static constexpr int MAXT = kNslMaxSeg + 2 * RN;   // steps of a segment
    // one unused entry after every four: the lanes of a warp read positions
    // 4 (ug - 2 db) + const, which this spreads over the banks
    __host__ __device__ static constexpr int pad(int i) { return i + (i >> 2); }
    static constexpr int AWP = pad(AW - 1) + 1;
    static constexpr int CNP = pad(CN - 1) + 1;
    static constexpr int NE = (LW + AW + kNslThreads - 1) / kNslThreads;   // staged values per thread
    static constexpr int NC = (CN + kNslThreads - 1) / kNslThreads;        // centres per thread
    static constexpr int NX = (TX + kNslThreads - 1) / kNslThreads;        // columns per thread
    static_assert(D == 16 || D == 32 || D == 64, "D must be 16, 32 or 64");
    static_assert(U % 4 == 0 && (DB == 4 || DB == 8), "padded indices split at multiples of 4");
};

template <int RN, int D>
struct NslSmem {
    using C = NslCfg<RN, D>;
    float2 ad[C::NR][C::AWP];     // (a - 128, b - a) of the staged rows
    float2 sums[C::NR][C::CN];    // per block centre: row sums of a~ and of delta
    float lrow[C::NR][C::LW];     // left intensities
    float lsum[C::NR][C::TX];     // per output column: row sum of the left intensities
    float4 cs[C::CNP];            // per block centre of the output row: {Ma, Mf, inv_r, 0}
    float sl[C::TX];              // per output column: block sum of the left intensities
    float il[C::TX];              // per output column: inv_l
    float rw[C::MAXT];            // per step: fraction w_y of the staged row's shift
    int rk[C::MAXT];              // per step: integer part k_y
};

template <int RN, int D, typename VT>
__global__ void __launch_bounds__(kNslThreads, kNslResident)
k_ncc_sl(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch, int W,
         int H, int row0, double alpha0, double alpha1, double delta,
         const float *__restrict__ inv_l, const float *__restrict__ inv_r,
         VT *__restrict__ vol, int Wo, int seg) {
    using C = NslCfg<RN, D>;
    constexpr int U = C::U, DB = C::DB, B = C::B, NR = C::NR, WIN = C::WIN;
    extern __shared__ __align__(16) unsigned char nsl_raw[];
    NslSmem<RN, D> &sm = *reinterpret_cast<NslSmem<RN, D> *>(nsl_raw);
    pdl_trigger();   // a programmatic dependent may launch once every CTA is here

    const int tid = threadIdx.x;
    const int db = tid % C::NDB, ug = tid / C::NDB;
    const int d0 = DB * db;
    const int x0 = blockIdx.x * C::TX;
    const int u0 = x0 + U * ug;
    const int WE = W + D - 1;   // columns of the statistics rows
    // the segment: image rows [J seg, (J+1) seg) of the frame, J counted from
    // the segment holding this image's first row
    const int J = row0 / seg + (int)blockIdx.y;
    const int ys = max(J * seg - row0, 0), ye = min((J + 1) * seg - row0, H);
    if (ys >= ye) return;
    const int T = ye - ys + 2 * RN;   // steps: rows ys - RN .. ye + RN - 1

    // row shifts of the staged rows (Sec. II-A), as the warp computes them
    for (int i = tid; i < T; i += kNslThreads) {
        const int y = clampi(ys - RN + i, 0, H - 1);
        const double s = row_shift(alpha0, alpha1, delta, y + row0);
        double k = floor(s);
        sm.rw[i] = (float)(s - k);
        k = fmin(fmax(k, -2.0 * W - 2.0), 2.0 * W + 2.0);   // beyond this every read clamps
        sm.rk[i] = (int)k;
    }
    // the thread's offset o: a left intensity next to its columns
    const float o = (float)left[(size_t)clampi(ys, 0, H - 1) * pitch + clampi(u0 + 1, 0, W - 1)];
    __syncthreads();

    // ---- staging: global loads of step t into registers, stored next step --
    int pa[C::NE], pb[C::NE];
    auto prefetch = [&](int t) {
        const int y = clampi(ys - RN + t, 0, H - 1);
        const int k = sm.rk[t];
        const uint8_t *lr = left + (size_t)y * pitch;
        const uint8_t *rr = right + (size_t)y * pitch;
#pragma unroll
        for (int i = 0; i < C::NE; ++i) {
            const int e = tid + kNslThreads * i;
            pa[i] = pb[i] = 0;
            if (e < C::LW) {
                pa[i] = lr[clampi(x0 - RN + e, 0, W - 1)];
            } else if (e < C::LW + C::AW) {
                const int x = clampi(x0 - RN - (D - 1) + (e - C::LW), 0, W - 1);
                pa[i] = rr[clampi(x - k, 0, W - 1)];
                pb[i] = rr[clampi(x - k - 1, 0, W - 1)];
            }
        }
    };
    auto stage = [&](int t) {
        const int s = t % NR;
#pragma unroll
        for (int i = 0; i < C::NE; ++i) {
            const int e = tid + kNslThreads * i;
            if (e < C::LW) {
                sm.lrow[s][e] = (float)pa[i];
            } else if (e < C::LW + C::AW) {
                const int j = C::pad(e - C::LW);
                if (SR_CHECK(j, C::AWP, 111))
                    sm.ad[s][j] = make_float2((float)(pa[i] - 128), (float)(pb[i] - pa[i]));
            }
        }
    };
    // column sums of the staged row t (exact integers)
    auto row_sums = [&](int t) {
        const int s = t % NR;
#pragma unroll
        for (int q = 0; q < C::NC; ++q) {
            const int ic = tid + kNslThreads * q;
            if (ic >= C::CN) break;
            float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int m = 0; m < B; ++m) {
                const float2 v = sm.ad[s][C::pad(ic + m)];
                a.x += v.x;
                a.y += v.y;
            }
            sm.sums[s][ic] = a;
        }
#pragma unroll
        for (int q = 0; q < C::NX; ++q) {
            const int iu = tid + kNslThreads * q;
            if (iu >= C::TX) break;
            float a = 0.0f;
#pragma unroll
            for (int m = 0; m < B; ++m) a += sm.lrow[s][iu + m];
            sm.lsum[s][iu] = a;
        }
    };
    // inv_r of the block centres and inv_l of the columns of output row v,
    // loaded a step ahead of their use
    float ir_pf[C::NC], il_pf[C::NX];
    auto prefetch_inv = [&](int v) {
#pragma unroll
        for (int q = 0; q < C::NC; ++q) {
            const int c = x0 - (D - 1) + tid + kNslThreads * q;   // block centre u - d
            ir_pf[q] = 0.0f;   // centres past the right edge: stored as 0
            if (tid + kNslThreads * q < C::CN && c < W)
                ir_pf[q] = inv_r[(size_t)v * WE + c + D - 1];
        }
#pragma unroll
        for (int q = 0; q < C::NX; ++q) {
            const int u = x0 + tid + kNslThreads * q;
            il_pf[q] = 0.0f;
            if (tid + kNslThreads * q < C::TX && u < Wo) il_pf[q] = inv_l[(size_t)v * WE + u];
        }
    };
    // block statistics of output row v, whose window rows were staged at
    // steps t - B .. t - 1
    auto centre_stats = [&](int t) {
        const float *w = sm.rw + (t - B);
#pragma unroll
        for (int q = 0; q < C::NC; ++q) {
            const int ic = tid + kNslThreads * q;
            if (ic >= C::CN) break;
            float ma = 0.0f, mf = 0.0f;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                const float2 v = sm.sums[(t - B + i) % NR][ic];
                ma += v.x;
                mf = fmaf(w[i], v.y, mf);
            }
            sm.cs[C::pad(ic)] = make_float4(ma, mf, ir_pf[q], 0.0f);
        }
#pragma unroll
        for (int q = 0; q < C::NX; ++q) {
            const int iu = tid + kNslThreads * q;
            if (iu >= C::TX) break;
            float a = 0.0f;
#pragma unroll
            for (int i = 0; i < B; ++i) a += sm.lsum[(t - B + i) % NR][iu];
            sm.sl[iu] = a;
            sm.il[iu] = il_pf[q];
        }
    };

    // ---- window sums {SP, SQ} of the thread's 4 columns x 8 disparities ----
    float2 st[U][DB];
#pragma unroll
    for (int k = 0; k < U; ++k)
#pragma unroll
        for (int j = 0; j < DB; ++j) st[k][j] = make_float2(0.0f, 0.0f);

    // add (sw = {1, w}) or remove (sw = {-1, -w}) the staged row in slot s:
    // per disparity the row sums {P, Q} of column u0, then of u0 + 1 .. + 3
    // by sliding (all exact integers), then st = sw * {P, Q} + st
    auto update = [&](int s, float2 sw) {
        float lt[WIN], nlt[U - 1];
#pragma unroll
        for (int m = 0; m < WIN; ++m) lt[m] = sm.lrow[s][U * ug + m] - o;
#pragma unroll
        for (int k = 0; k < U - 1; ++k) nlt[k] = -lt[k];
        // position of (column u0, tap -RN) at disparity d0 + DB - 1; the
        // positions of disparity d0 + j start DB - 1 - j further on.  base
        // is a multiple of 4, so pad(base + q) = pad(base) + pad(q)
        const int base = U * ug + D - DB - d0;
        const float2 *ad = sm.ad[s] + C::pad(base);
        // two halves of DB/2 disparities, each over a sliding window of WIN
        // positions (one new position per disparity)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            constexpr int HB = DB / 2;
            float2 av[WIN + HB - 1];
#pragma unroll
            for (int q = 0; q < WIN + HB - 1; ++q) {
                const int qq = h * HB + q;
                av[q] = SR_CHECK(C::pad(base + qq), C::AWP, 112) ? ad[C::pad(qq)]
                                                                 : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int jj = 0; jj < HB; ++jj) {
                const int j = DB - 1 - (h * HB + jj);
                float2 p = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int m = 0; m < B; ++m) p = __ffma2_rn(make_float2(lt[m], lt[m]), av[jj + m], p);
                st[0][j] = __ffma2_rn(sw, p, st[0][j]);
#pragma unroll
                for (int k = 1; k < U; ++k) {
                    p = __ffma2_rn(make_float2(lt[k + 2 * RN], lt[k + 2 * RN]), av[jj + k + 2 * RN], p);
                    p = __ffma2_rn(make_float2(nlt[k - 1], nlt[k - 1]), av[jj + k - 1], p);
                    st[k][j] = __ffma2_rn(sw, p, st[k][j]);
                }
            }
        }
    };

    // costs of output row v from the window sums (see the header)
    auto epilogue = [&](int v) {
        constexpr float n = (float)(B * B);
        // block centre u - d of (column k, disparity j): index U ug - d0 +
        // (D - 1 + k - j), the first part a multiple of 4 (see update)
        const float4 *csb = sm.cs + C::pad(U * ug - d0);
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int u = u0 + k;
            if (u >= Wo) break;
            const float slt = sm.sl[U * ug + k] - n * o;   // block sum of l~
            const float il = sm.il[U * ug + k];
            float cst[DB];
#pragma unroll
            for (int j = 0; j < DB; ++j) {
                const int cj = D - 1 + k - j;
                const float4 cs = SR_CHECK(C::pad(U * ug - d0 + cj), C::CNP, 114)
                                      ? csb[C::pad(cj)] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                // {-(Sl Ma), -(Sl Mf)}, rounded; e = the first one's rounding error, exact
                const float2 nts = __fmul2_rn(make_float2(-slt, -slt), make_float2(cs.x, cs.y));
                const float e = fmaf(slt, cs.x, nts.x);
                const float2 vy = __ffma2_rn(make_float2(n, n), st[k][j], nts);
                cst[j] = ((vy.x - e) + vy.y) * il * cs.z;
            }
            const size_t off = ((size_t)v * Wo + u) * D + d0;
            if (SR_CHECK(off + DB - 1, (long long)H * Wo * D, 113)) {
                if constexpr (DB == 8)
                    store8(vol + off, cst);
                else
                    store4(vol + off, cst);
            }
        }
    };

    prefetch(0);
    prefetch_inv(ys);
#pragma unroll 1
    for (int t = 0; t <= T; ++t) {
        if (t < T) {
            stage(t);
            if (t + 1 < T) prefetch(t + 1);
        }
        const int v = ys + t - B;   // output row whose window the sums hold
        if (t >= B) {
            centre_stats(t);
            if (v + 1 < ye) prefetch_inv(v + 1);
        }
        __syncthreads();
        if (t >= B) epilogue(v);
        if (t < T) {
            row_sums(t);
            update(t % NR, make_float2(1.0f, sm.rw[t]));
            if (t >= B) update((t + 1) % NR, make_float2(-1.0f, -sm.rw[t - B]));
        }
        __syncthreads();
    }
}

template <int RN, int D, typename VT>
constexpr size_t nsl_smem() {
    return sizeof(NslSmem<RN, D>);
}

template <int RN, int D, typename VT>
cudaError_t ncc_sl_launch_t(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                            int row0, double alpha0, double alpha1, double delta,
                            const float *inv_l, const float *inv_r, VT *vol, int Wo, int seg,
                            cudaStream_t st) {
    using C = NslCfg<RN, D>;
    constexpr size_t smem = nsl_smem<RN, D, VT>();
    if (seg < 1 || seg > kNslMaxSeg || row0 < 0 || H < 1 || Wo < 1) return cudaErrorInvalidValue;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_ncc_sl<RN, D, VT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int s0 = row0 / seg, s1 = (row0 + H + seg - 1) / seg;
    const dim3 grid((Wo + C::TX - 1) / C::TX, s1 - s0);
    k_ncc_sl<RN, D, VT><<<grid, kNslThreads, smem, st>>>(left, right, pitch, W, H, row0, alpha0,
                                                         alpha1, delta, inv_l, inv_r, vol, Wo, seg);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

template <int RN, int D, typename VT>
int ncc_sl_occ_t() {
    constexpr size_t smem = nsl_smem<RN, D, VT>();
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ncc_sl<RN, D, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ncc_sl<RN, D, VT>, kNslThreads, smem) !=
        cudaSuccess)
        return 0;
    return b;
}

template <int D, typename VT>
cudaError_t ncc_sl_launch_d(const uint8_t *left, const uint8_t *right, int pitch, int W, int H,
                            int ncc_r, int row0, double alpha0, double alpha1, double delta,
                            const float *inv_l, const float *inv_r, VT *vol, int Wo, int seg,
                            cudaStream_t st) {
    switch (ncc_r) {
        case 1: return ncc_sl_launch_t<1, D, VT>(left, right, pitch, W, H, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st);
        case 2: return ncc_sl_launch_t<2, D, VT>(left, right, pitch, W, H, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st);
        case 3: return ncc_sl_launch_t<3, D, VT>(left, right, pitch, W, H, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st);
        case 4: return ncc_sl_launch_t<4, D, VT>(left, right, pitch, W, H, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st);
        case 5: return ncc_sl_launch_t<5, D, VT>(left, right, pitch, W, H, row0, alpha0, alpha1, delta, inv_l, inv_r, vol, Wo, seg, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int D, typename VT>
int ncc_sl_occ_d(int ncc_r) {
    switch (ncc_r) {
        case 1: return ncc_sl_occ_t<1, D, VT>();
        case 2: return ncc_sl_occ_t<2, D, VT>();
        case 3: return ncc_sl_occ_t<3, D, VT>();
        case 4: return ncc_sl_occ_t<4, D, VT>();
        case 5: return ncc_sl_occ_t<5, D, VT>();
        default: return 0;
    }
}

}  // namespace sr
