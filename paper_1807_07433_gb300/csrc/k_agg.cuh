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
//   * the tile's source rows (+R halo rows and columns) stream through a
//     double-buffered shared-memory ring, one image row at a time: the cost
//     row (one contiguous run of (32+2R)*D floats in the d-innermost volume)
//     arrives by a single TMA bulk copy (cp.async.bulk) completing on an
//     mbarrier per ring slot (columns outside the image are zeroed once);
//     consumers wait with a bounded spin that records a timeout in an error
//     word instead of hanging.  In the same step the CTA computes the weights
//     that row needs -- tap row dy = y - v of each of the 4 output rows --
//     into a second double-buffered ring laid out [row][dx][pixel], so one
//     load gives one tap's weight for the lane's adjacent pixels.  Each
//     weight is computed exactly once, and shared memory stays ~38 KB per
//     CTA, so four CTAs (16 warps) fit on an SM;
//   * lane = 4 disparities of a block of 4 x 4 pixels (8 disparities of
//     2 x 4 pixels for FP32 costs at D = 64 and in the band kernel's
//     padded slices); the lanes of a pixel group
//     read the same weights (a broadcast) and together one cost column
//     (16-byte loads, conflict-free);
//   * each thread accumulates 64 sums, held as 32 pairs of disparities that
//     one paired multiply-add (fma.rn.f32x2) updates per tap, the weight
//     paired with itself.  Tap columns are the outer loop: per tap column
//     one new cost column enters the thread's sliding window and serves the
//     lane's pixels and every output row that uses the source row (32
//     independent paired multiply-adds);
//   * epilogue: the sums are transposed through shared memory (over the
//     rings; 16-byte stores, rows of D + 4; the band kernel keeps rows of
//     D + 1) so that each lane scans the D costs of one pixel, four per
//     load: argmax (ties to the smallest d), then Eq. 12 on the neighbours
//     of the winner.  The normalisation by sum_k w_k is a positive
//     per-pixel scale, which changes neither the argmax nor the parabola
//     vertex, so it is applied only when the aggregated volume is exported.
#pragma once
#include <cuda.h>

#include <type_traits>
#include <utility>

#include "sr_internal.cuh"

namespace sr {

constexpr int kAggTX = 32, kAggTY = 4, kAggPix = kAggTX * kAggTY;

// The 4 costs of lane sl of a pixel group in the cost column at col (layout
// [col][D]): disparities 4 sl .. 4 sl + 3, one 16-byte (FP32) or 8-byte
// (16-bit) load, widened to FP32.
__device__ __forceinline__ float4 load_col4(const float *col, int sl) {
    return *reinterpret_cast<const float4 *>(col + 4 * sl);
}
__device__ __forceinline__ float4 load_col4(const __half *col, int sl) {
    const uint2 q = *reinterpret_cast<const uint2 *>(col + 4 * sl);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 load_col4(const __nv_bfloat16 *col, int sl) {
    // a bfloat16 is the upper half of the FP32 word of equal value: one
    // shift or mask per element, no conversion instruction
    const uint2 q = *reinterpret_cast<const uint2 *>(col + 4 * sl);
    return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u),
                       __uint_as_float(q.y << 16), __uint_as_float(q.y & 0xffff0000u));
}

// SH: the tile reads a cost row sheared, pixel u at disparity d from column
// u + d of an extended reference volume (the target view of Sec. II-B-1):
// the ring slot holds D/CW boxes of CW disparities x BH pixels of a 2-D
// tensor map, one box per CW-disparity chunk.  CW = 32 (128-byte box rows:
// half the copies of CW = 16) where MINB CTAs still fit an SM, else 16; with
// CW = 16, odd chunks start one pixel earlier, which moves their words to
// the other half of the banks (the chunk stride is a multiple of 32 words).
template <int R, int D, typename VT, bool SH = false, bool BANDED = false>
struct AggCfg {
    // Lane layout.  A lane holds PX = 4 pixels x 4 output rows x DL = 4
    // disparities: 64 sums, as 32 pairs of disparities, each updated by one
    // paired multiply-add (fma.rn.f32x2) per tap, the weight paired with
    // itself.  Shared memory sets the pace of this loop, and its cost is
    // wavefronts, not lane bytes: the D/4 lanes of a pixel group read one
    // cost column together (D x 4 bytes, the fewest wavefronts a column can
    // take), and the lanes of a group share each weight load (a broadcast:
    // one wavefront for the warp's float4 of 4 pixels).  Per tap column a
    // lane loads one cost column (4 disparities) and one float4 of weights per
    // output row, which feed 32 multiply-adds.  The sheared rows of the
    // target view read the 4 disparities of a pixel from the diagonal of
    // their chunks, one element each.
    //
    // FP32 costs at D = 64, and in the band kernel's padded 16-disparity
    // slices, keep an earlier layout of 8 disparities x 2 pixels
    // (disparities 4 sl.. and D/2 + 4 sl.., two 16-byte loads per column):
    // it runs the target view 2 % and the band kernel 2 % faster, with fewer
    // registers, although it takes 40 % more wavefronts per row.  For
    // unpadded D = 16 and 32 that layout conflicts on every column load, and
    // for 16-bit costs it converts twice as many elements per multiply-add.
    static constexpr int DL = (sizeof(VT) == 4 && (D == 64 || BANDED)) ? 8 : 4;
    static constexpr int SLOTS = D / DL;           // lanes per pixel group
    static constexpr int G = 32 / SLOTS;           // pixel groups per warp
    static constexpr int PX = 16 / DL;             // pixel columns of a group
    static constexpr int PPG = kAggTY * PX;        // pixels of a group
    static constexpr int NW = D / 16;              // warps per CTA
    static constexpr int NT = 32 * NW;
    static constexpr int MINB = 512 / NT;          // CTAs per SM to fit
    static constexpr int WS = 2 * R + 1;           // window side
    static constexpr int TXE = kAggTX + 2 * R;     // ring row width (pixels)
    static constexpr int TYE = kAggTY + 2 * R;     // source rows per tile
    // sheared geometry for a chunk width cw: pixels of a box, chunk stride
    // (rounded up to 128 bytes, a tensor-map copy's destination alignment)
    static constexpr int shear_shift(int cw) { return (cw == 16 && D > 16) ? 1 : 0; }
    static constexpr int shear_bh(int cw) { return TXE + cw - 1 + shear_shift(cw); }
    static constexpr int shear_cse(int cw) {
        return (int)(((shear_bh(cw) * cw * sizeof(VT) + 127) / 128 * 128) / sizeof(VT));
    }
    // shared memory of a CTA whose cost-ring slot holds ring elements
    // epilogue: a pixel's D sums, rows padded to a multiple of 16 bytes so
    // that a lane stores its 4 disparities, and the scan loads 4, at once;
    // the band kernel, whose windows are a few disparities wide, keeps odd
    // rows (scalar stores and loads, 1 % faster there)
    static constexpr int EPS = BANDED ? D + 1 : D + 4;
    static constexpr size_t single_for(int ring) {
        const size_t rings = ((size_t)ring * sizeof(VT) + 127) / 128 * 128;
        const size_t ringsb = 2 * rings + (NW > 1 ? 2 : 1) * (size_t)(kAggTY * WS * kAggTX) * sizeof(float);
        const size_t epib = (size_t)kAggPix * EPS * sizeof(float);
        const size_t uni = ((ringsb > epib ? ringsb : epib) + 15) / 16 * 16;
        return uni + sizeof(float) * (((size_t)TYE * TXE + 3) / 4 * 4 + kAggPix) +
               2 * sizeof(unsigned long long) + sizeof(int) * 4;
    }
    static constexpr int CW = (SH && D >= 32 &&
                               MINB * (single_for((D / 32) * shear_cse(32)) + 1024) <= 228 * 1024)
                                  ? 32 : 16;
    static constexpr int NCH = D / CW;             // sheared: chunks
    static constexpr int SHIFT = shear_shift(CW);  // sheared: odd chunks start a pixel earlier
    static constexpr int BH = shear_bh(CW);        // sheared: pixels of a chunk's box
    static constexpr int CSE = shear_cse(CW);      // sheared: chunk stride (elements)
    // elements between the cost columns of a ring row: D, except for the
    // 16-disparity slices of the band kernel, whose 2-D copies widen each
    // column by 16 bytes (the next disparities, or zeros past the volume's
    // last): a 16-disparity column spans only 16 banks, and the padding
    // spreads the pixel groups of a warp over all 32
    static constexpr int CS = BANDED ? D + (int)(16 / sizeof(VT)) : D;
    // elements of one cost row of the tile
    static constexpr int RING = SH ? NCH * CSE : TXE * CS;
    // slot stride: RING rounded up to 128 bytes
    static constexpr int RINGS = (int)(((RING * sizeof(VT) + 127) / 128 * 128) / sizeof(VT));
    static constexpr int WRING = kAggTY * WS * kAggTX;  // floats per weight slot
    // weight-ring slots: two let the warps of a CTA compute the next row's
    // weights while others still read the current ones; a one-warp CTA
    // (D = 16) runs in order anyway, so one slot saves the shared memory
    static constexpr int WSL = NW > 1 ? 2 : 1;
    // shared memory, in bytes: [cost ring | weight ring] (reused by the
    // epilogue transpose), guide tile, weight sums, two mbarriers
    static constexpr size_t RINGB = 2 * (size_t)RINGS * sizeof(VT);
    static constexpr size_t RINGSB = RINGB + WSL * (size_t)WRING * sizeof(float);
    static constexpr size_t EPIB = (size_t)kAggPix * EPS * sizeof(float);
    static constexpr size_t UNIONB = ((RINGSB > EPIB ? RINGSB : EPIB) + 15) / 16 * 16;
    static constexpr int GUIDE = TYE * TXE;
    // (+ the batched kernel's work-list prefix and next-item slot, last, so
    // that the cost ring at offset 0 keeps the alignment TMA copies prefer)
    static constexpr size_t SMEM = UNIONB + sizeof(float) * ((GUIDE + 3) / 4 * 4 + kAggPix) +
                                   2 * sizeof(unsigned long long) +
                                   sizeof(int) * (kStartSmem + 4);
    // kernels that do not walk a batch work list leave out its prefix array
    static constexpr size_t SMEM_SINGLE = SMEM - sizeof(int) * kStartSmem;
    static_assert(single_for(RING) == SMEM_SINGLE, "shared-memory layouts disagree");
    static_assert(D == 16 || D == 32 || D == 64, "D must be 16, 32 or 64");
    static_assert(kAggTY == 4, "band counters assume tiles of 4 rows");
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// One-dimensional TMA copy global -> shared, completing on an mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Two-dimensional TMA tile copy global -> shared through a tensor map,
// completing on an mbarrier: box origin (x, y) in elements (x the inner
// coordinate, 16-byte aligned; y may be negative or past the end, where the
// box reads zeros).
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}
// Wait for the phase of the given parity; gives up after max_cycles SM clocks
// (then records the timeout in *err and returns false).
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          long long max_cycles, int *err) {
    const unsigned a = smem_addr(bar);
    if (mbar_try(a, parity)) return true;   // usually complete: no clock read
    const long long t0 = clock64();
    while (true) {
        if (mbar_try(a, parity)) return true;
        if (clock64() - t0 > max_cycles) {
            if (err) atomicExch(err, 1);
            return false;
        }
    }
}
__device__ __forceinline__ float ex2_approx(float x) {   // 2^x, hardware approximation
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;\n" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory carve-up of an aggregation CTA (see AggCfg).
template <int R, int D, typename VT, bool SH = false, bool BANDED = false>
struct AggSmem {
    using C = AggCfg<R, D, VT, SH, BANDED>;
    unsigned char *raw;
    __device__ float *epi() const { return reinterpret_cast<float *>(raw); }
    __device__ VT *ring() const { return reinterpret_cast<VT *>(raw); }
    __device__ float *wring() const { return reinterpret_cast<float *>(raw + C::RINGB); }
    __device__ float *guide() const { return reinterpret_cast<float *>(raw + C::UNIONB); }
    __device__ float *wsum() const { return guide() + (C::GUIDE + 3) / 4 * 4; }
    __device__ unsigned long long *bars() const {
        return reinterpret_cast<unsigned long long *>(wsum() + kAggPix);
    }
    __device__ int *next_slot() const { return reinterpret_cast<int *>(bars() + 2); }
    __device__ int *start() const { return next_slot() + 4; }
};

template <int R, int D, typename VT, bool SH, bool BANDED>
__device__ __forceinline__ void agg_init_barriers(const AggSmem<R, D, VT, SH, BANDED> &sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bars()[0], 1);
        mbar_init(&sm.bars()[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
}

// One 32 x 4 tile at (x0, y0) with all D disparities.  ph holds, per ring
// slot, the parity of the slot's next mbarrier phase; it carries over from
// tile to tile of a persistent CTA.  All threads of the CTA take part.
//
// BAND: the ring holds the D = kBandD disparities [dlo, dlo + D) of each pixel,
// loaded as one 2-D tensor-map box per row (tmap); SH: the sheared row of an
// extended volume (see AggCfg), D/16 boxes per row (tmap); otherwise the D
// disparities of the volume (rows of vpitch pixels), one bulk copy per row.
// WIN: win restricts the WTA and Eq. 12 of each pixel to its window (see
// AggWin); a compile-time choice, so that the full search keeps its own code.
template <int R, int D, bool GU8, typename VT, bool BAND = false, bool WIN = BAND, bool SH = false>
__device__ __forceinline__ void agg_tile(const AggSmem<R, D, VT, SH, BAND> &sm, unsigned &ph,
                                         const VT *__restrict__ vol, int vpitch,
                                         const uint8_t *__restrict__ gl,
                                         int pitch, const float *__restrict__ gf, int W, int H,
                                         float kd, float kr, int16_t *__restrict__ lbl,
                                         float *__restrict__ dsub, float *__restrict__ agg,
                                         int *__restrict__ err, long long wait_cycles,
                                         int withhold_last, int x0, int y0,
                                         const void *tmap = nullptr, int dlo = 0,
                                         const AggWin &win = AggWin(), int pdl = 0) {
    using C = AggCfg<R, D, VT, SH, BAND>;
    float *smem = sm.epi();                      // epilogue view
    VT *ring = sm.ring();                        // [2][TXE][D] cost rows
    float *wring = sm.wring();                   // [2][4][WS][32] weights
    float *guide = sm.guide();                   // [TYE][TXE]
    float *wsum = sm.wsum();                     // [128]
    unsigned long long *bars = sm.bars();        // [2]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // Columns of the tile's cost rows that lie inside the image; the rest of
    // each ring slot is zeroed once (those neighbours have weight 0).
    const int xs = max(x0 - R, 0), xe = min(x0 + kAggTX + R, W);
    const unsigned row_bytes = (unsigned)((xe - xs) * D * sizeof(VT));
    // withhold_last (fault injection): no arrival and no copy for the last
    // source row, whose wait then runs out; no later copy shares its slot,
    // so nothing is in flight when the CTA exits.
    auto issue_row = [&](int j) {   // thread 0: cost row of source row j -> slot j&1
        const int y = y0 - R + j;
        unsigned long long *bar = bars + (j & 1);
        if (withhold_last && j == C::TYE - 1) return;
        if (y < 0 || y >= H) {
            mbar_arrive(bar);   // no copy: complete the phase to keep the slot in step
            return;
        }
        if (BAND) {
            // the whole box: pixels beyond the row's ends come from the
            // neighbouring rows (or are zeros) and meet zero weights
            if (!SR_CHECK((dlo * (int)sizeof(VT)) & 15, 1, 201)) {   // x on a 16-byte boundary
                mbar_arrive(bar);
                return;
            }
            mbar_arrive_expect_tx(bar, (unsigned)(C::RING * sizeof(VT)));
            tma_load_2d(ring + (j & 1) * C::RINGS, tmap, dlo, y * W + x0 - R, bar);
            return;
        }
        if (SH) {
            // chunk c: disparities [16c, 16c + 16) of volume columns
            // x0 - R + 16c - (c & 1) + [0, BH); tile pixel i at disparity
            // 16c + m sits in box row i + m + (c & 1).  As for BAND, columns
            // beyond the row's ends come from the neighbouring rows (or are
            // zeros) and meet zero weights.
            if (!SR_CHECK(C::NCH * C::CSE, C::RINGS + 1, 202)) {   // boxes within the slot
                mbar_arrive(bar);
                return;
            }
            mbar_arrive_expect_tx(bar, (unsigned)(C::NCH * C::BH * C::CW * sizeof(VT)));
#pragma unroll
            for (int c = 0; c < C::NCH; ++c)
                tma_load_2d(ring + (j & 1) * C::RINGS + c * C::CSE, tmap, C::CW * c,
                            y * vpitch + x0 - R + C::CW * c - C::SHIFT * (c & 1), bar);
            return;
        }
        VT *dst = ring + (j & 1) * C::RINGS + (xs - (x0 - R)) * D;
        const VT *src = vol + ((size_t)y * vpitch + xs) * D;
        // the copy stays inside its slot and inside the volume row
        if (!SR_CHECK((xe - (x0 - R)) * D - 1, C::RINGS, 203) || !SR_CHECK(xe - 1, vpitch, 203) ||
            !SR_CHECK(xs, xe, 203)) {
            mbar_arrive(bar);
            return;
        }
        mbar_arrive_expect_tx(bar, row_bytes);
        tma_load_1d(dst, src, row_bytes, bar);
    };

    // Weights (Eqs. 9-10) that source row j contributes with: for output row
    // py the tap row is dyi = j - py.  w = exp(-r^2/gd^2 - dg^2/gr^2)
    // = exp2(-(r^2 kd + dg^2 kr)), zero for neighbours outside the image.
    // Warp k computes rows py = k, k + NW, ...; lane = pixel column.  In a
    // tile whose pixels and neighbourhoods all lie inside the image
    // (interior == true) no weight needs the border test.
    auto make_weights = [&](int j, auto interior) {
        float *wslot = wring + (j % C::WSL) * C::WRING;
#pragma unroll
        for (int k = 0; k < 4 / C::NW; ++k) {
            const int py = warp + k * C::NW;
            const int dyi = j - py;
            if (dyi < 0 || dyi >= C::WS) continue;
            const int px = lane, u = x0 + px, v = y0 + py, y = v + dyi - R;
            const bool rowok = decltype(interior)::value || ((u < W) && (v < H) && (y >= 0) && (y < H));
            const bool inner = decltype(interior)::value || (rowok && (u - R >= 0) && (u + R < W));
            if (!SR_CHECK((py + dyi) * C::TXE + px + C::WS - 1, C::GUIDE, 204) ||
                !SR_CHECK((py * C::WS + C::WS - 1) * kAggTX + px, C::WRING, 204))
                continue;
            const float gc = guide[(py + R) * C::TXE + px + R];
            const float *grow = guide + (py + dyi) * C::TXE + px;
            const float fy = (float)((dyi - R) * (dyi - R)) * kd;
            float *wout = wslot + (py * C::WS) * kAggTX + px;
#pragma unroll
            for (int dxi = 0; dxi < C::WS; ++dxi) {
                const float dg = grow[dxi] - gc;
                float w = ex2_approx(-fmaf(dg * dg, kr, fmaf((float)((dxi - R) * (dxi - R)), kd, fy)));
                if (!inner) {
                    const int x = u + dxi - R;
                    w = (rowok && x >= 0 && x < W) ? w : 0.0f;
                }
                wout[dxi * kAggTX] = w;
            }
        }
    };

    // ---- prologue: first row in flight, guide tile, zeroed columns ---------
    // (the copy writes only the in-image columns of slot 0, the zeroing only
    // the others; in a persistent CTA the barrier before this tile ordered
    // the previous epilogue's reads of this memory)
    if (tid == 0) {
        if (pdl == 1) {   // the volume's producer grid is complete (see pdl_trigger)
            pdl_wait();
            asm volatile("fence.proxy.async.global;\n" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        issue_row(0);
    }
    {   // all loads of a thread first, then the stores: their latencies overlap
        constexpr int NG = (C::GUIDE + C::NT - 1) / C::NT;
        float g[NG];
#pragma unroll
        for (int k = 0; k < NG; ++k) {
            const int i = tid + k * C::NT;
            const int r = i / C::TXE, c = i % C::TXE;
            const int y = y0 - R + r, x = x0 - R + c;
            g[k] = 0.0f;
            if (i < C::GUIDE && y >= 0 && y < H && x >= 0 && x < W && SR_CHECK(x, GU8 ? pitch : W, 205))
                g[k] = GU8 ? (float)gl[(size_t)y * pitch + x] : gf[(size_t)y * W + x];
        }
#pragma unroll
        for (int k = 0; k < NG; ++k)
            if (tid + k * C::NT < C::GUIDE) guide[tid + k * C::NT] = g[k];
    }
    if (!BAND && !SH && (xs > x0 - R || xe < x0 + kAggTX + R)) {
        for (int i = tid; i < 2 * C::RINGS; i += C::NT) {
            const int c = (i % C::RINGS) / D + x0 - R;
            if (c < xs || c >= xe) ring[i] = VT(0.0f);
        }
    }
    const bool interior = x0 - R >= 0 && x0 + kAggTX + R <= W && y0 - R >= 0 && y0 + kAggTY + R <= H;
    auto weights_of_row = [&](int j) {
        if (interior)
            make_weights(j, std::integral_constant<bool, true>());
        else
            make_weights(j, std::integral_constant<bool, false>());
    };
    __syncthreads();
    // (pdl == 1) every thread is past thread 0's wait for the volume's
    // producer: a programmatic dependent may launch once all CTAs are here
    if (pdl == 1) pdl_trigger();
    if (C::WSL == 2) weights_of_row(0);
    __syncthreads();

    // ---- main loop: stream the tile's source rows --------------------------
    constexpr int PX = C::PX, DL = C::DL;
    const int sl = lane % C::SLOTS, grp = lane / C::SLOTS;
    const int bcol = warp * C::G + grp;          // block column of PX pixels
    const int bx = bcol * PX;                    // first tile column of the block
    // sheared rows: pair q of the lane holds disparities m_q and m_q + D/2,
    // m_q = (sl + SLOTS q + c grp) mod D/2, the x half of the pair being
    // m_q + D/2 in odd groups (sh_hx); with c = D^2/256 and the swap (4
    // disparities per lane), or c = 8 and no swap (8 per lane, D = 64), the
    // 32 lanes of a warp load from 32 different banks for D = 32 and 64 (2
    // per bank for D = 16).  The element of disparity d for tile pixel i sits
    // at offset (d / CW) CSE + (i + d % CW + SHIFT ((d / CW) & 1)) CW + d % CW
    int sh_m[DL / 2] = {}, sh_off[DL] = {}, sh_hx = 0;
    if constexpr (SH) {
        sh_hx = DL == 4 ? (grp & 1) : 0;
#pragma unroll
        for (int q = 0; q < DL / 2; ++q) {
            sh_m[q] = (sl + C::SLOTS * q + (DL == 4 ? D * D / 256 : 8) * grp) % (D / 2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {   // h = 0: the pair's x element
                const int d = sh_m[q] + (h ^ sh_hx) * (D / 2), c = d / C::CW, m = d % C::CW;
                sh_off[q + (DL / 2) * h] = c * C::CSE + (m + C::SHIFT * (c & 1)) * C::CW + m;
            }
        }
    }

    float2 acc[kAggTY][PX][DL / 2];
#pragma unroll
    for (int py = 0; py < kAggTY; ++py)
#pragma unroll
        for (int px = 0; px < PX; ++px)
#pragma unroll
            for (int q = 0; q < DL / 2; ++q) acc[py][px][q] = make_float2(0.0f, 0.0f);

#pragma unroll 1
    for (int j = 0; j < C::TYE; ++j) {
        if (j + 1 < C::TYE) {
            if (tid == 0) {
                // slot (j+1)&1 was last read before the barrier that ended step j-1
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                issue_row(j + 1);
            }
            if (C::WSL == 2) weights_of_row(j + 1);
        }
        if (C::WSL == 1) {   // the single slot was last read before the previous barrier
            weights_of_row(j);
            __syncthreads();
        }
        const int y = y0 - R + j;
        if (y >= 0 && y < H) {
            mbar_wait(bars + (j & 1), (ph >> (j & 1)) & 1u, wait_cycles, err);
            const float *ws = wring + (j % C::WSL) * C::WRING + bx;
            // taps outer: a cost column (4 disparities) enters per tap
            // column and serves PX pixels x the valid output rows
            const VT *rs = SH ? ring + (j & 1) * C::RINGS + bx * C::CW
                              : ring + (j & 1) * C::RINGS + bx * C::CS;
            // output rows lo..hi (compile-time) use source row j: row py
            // takes tap row j - py, valid for j - WS < py <= j
            // (chk: test each output row at run time instead, one body for all
            // partial rows)
            auto body = [&](auto lo_c, auto hi_c, auto chk) {
                constexpr int LO = decltype(lo_c)::value, HI = decltype(hi_c)::value;
                float2 cst[PX + 2 * R][DL / 2];
                auto load_col = [&](int i) {
                    if constexpr (SH) {
                        // pair q: the diagonal elements at sh_off[q] (x)
                        // and sh_off[q + DL/2] (y)
#pragma unroll
                        for (int q = 0; q < DL / 2; ++q) {
                            const int o = (bx + i) * C::CW;
                            cst[i][q] = SR_CHECK(o + sh_off[q], C::RING, 206) &&
                                                SR_CHECK(o + sh_off[q + DL / 2], C::RING, 206)
                                            ? make_float2(load_one(rs + sh_off[q] + i * C::CW),
                                                          load_one(rs + sh_off[q + DL / 2] + i * C::CW))
                                            : make_float2(0.0f, 0.0f);
                        }
                        return;
                    }
                    // (checked builds: the column's last element lies in the slot)
                    if (!SR_CHECK((bx + i) * C::CS + 4 * sl + (DL == 8 ? D / 2 : 0) + 3, C::RING, 206)) {
#pragma unroll
                        for (int q = 0; q < DL / 2; ++q) cst[i][q] = make_float2(0.0f, 0.0f);
                        return;
                    }
                    if constexpr (DL == 8) {
                        // disparities 4 sl .. 4 sl + 3 and D/2 + 4 sl .. D/2 + 4 sl + 3
                        const float4 a = load_col4(rs + i * C::CS, sl);
                        const float4 b = load_col4(rs + i * C::CS + D / 2, sl);
                        cst[i][0] = make_float2(a.x, a.y);
                        cst[i][1] = make_float2(a.z, a.w);
                        cst[i][2] = make_float2(b.x, b.y);
                        cst[i][3] = make_float2(b.z, b.w);
                    } else {
                        const float4 c = load_col4(rs + i * C::CS, sl);
                        cst[i][0] = make_float2(c.x, c.y);
                        cst[i][1] = make_float2(c.z, c.w);
                    }
                };
#pragma unroll
                for (int i = 0; i < PX - 1; ++i) load_col(i);
#pragma unroll
                for (int dx = 0; dx < C::WS; ++dx) {
                    load_col(dx + PX - 1);
#pragma unroll
                    for (int py = 0; py < kAggTY; ++py) {
                        if (py >= LO && py <= HI &&
                            (!decltype(chk)::value || (unsigned)(j - py) < (unsigned)C::WS)) {
                            // the weights of the lane's pixels, each paired
                            // with itself for the paired multiply-add
                            float2 w[PX];
                            if (!SR_CHECK((py * C::WS + dx) * kAggTX + bx + PX - 1, C::WRING, 207)) {
#pragma unroll
                                for (int px = 0; px < PX; ++px) w[px] = make_float2(0.0f, 0.0f);
                            } else if constexpr (PX == 2) {
                                const float2 w2 = *reinterpret_cast<const float2 *>(
                                    ws + (py * C::WS + dx) * kAggTX);
                                w[0] = make_float2(w2.x, w2.x);
                                w[1] = make_float2(w2.y, w2.y);
                            } else {
                                const float4 w4 = *reinterpret_cast<const float4 *>(
                                    ws + (py * C::WS + dx) * kAggTX);
                                w[0] = make_float2(w4.x, w4.x);
                                w[1] = make_float2(w4.y, w4.y);
                                w[2] = make_float2(w4.z, w4.z);
                                w[3] = make_float2(w4.w, w4.w);
                            }
#pragma unroll
                            for (int px = 0; px < PX; ++px)
#pragma unroll
                                for (int q = 0; q < DL / 2; ++q)
                                    acc[py][px][q] = __ffma2_rn(w[px], cst[px + dx][q], acc[py][px][q]);
                        }
                    }
                }
            };
            // the rows that use source row j: 0..min(3, j) for the first
            // rows, lo..3 with lo = j - WS + 1 for the last; all four between.
            // Each range has a body of its own; for 15 x 15 windows the seven
            // bodies cost more than the tests they save (1.2585 against
            // 1.2247 ms for both views at 1280x720x64), so there the partial
            // rows share one body with run-time tests
            const int lo = max(0, j - C::WS + 1), hi = min(kAggTY - 1, j);
            using std::integral_constant;
            using I0 = integral_constant<int, 0>;
            using I1 = integral_constant<int, 1>;
            using I2 = integral_constant<int, 2>;
            using I3 = integral_constant<int, 3>;
            using NC = integral_constant<bool, false>;
            if (lo == 0 && hi == 3) body(I0(), I3(), NC());
            else if constexpr (R >= 7) body(I0(), I3(), integral_constant<bool, true>());
            else if (lo == 0 && hi == 0) body(I0(), I0(), NC());
            else if (lo == 0 && hi == 1) body(I0(), I1(), NC());
            else if (lo == 0 && hi == 2) body(I0(), I2(), NC());
            else if (lo == 1 && hi == 3) body(I1(), I3(), NC());
            else if (lo == 2 && hi == 3) body(I2(), I3(), NC());
            else if (lo == 3 && hi == 3) body(I3(), I3(), NC());
            else if (lo == 1 && hi == 2) body(I1(), I2(), NC());
        }
        ph ^= 1u << (j & 1);   // every source row completes one phase of its slot
        __syncthreads();
    }

    // ---- epilogue: transpose (over the rings), WTA, parabola ----------------
    if (agg) {   // weight sums for the exported (normalised) volume only
        for (int k = 0; k < 4 / C::NW; ++k) {
            const int py = warp + k * C::NW, px = lane, u = x0 + px, v = y0 + py;
            const float gc = guide[(py + R) * C::TXE + px + R];
            float s = 0.0f;
            for (int dyi = 0; dyi < C::WS; ++dyi)
                for (int dxi = 0; dxi < C::WS; ++dxi) {
                    const int x = u + dxi - R, y = v + dyi - R;
                    if (u >= W || v >= H || x < 0 || x >= W || y < 0 || y >= H) continue;
                    const float dg = guide[(py + dyi) * C::TXE + px + dxi] - gc;
                    const float fy = (float)((dyi - R) * (dyi - R)) * kd;
                    s += ex2_approx(-fmaf(dg * dg, kr, fmaf((float)((dxi - R) * (dxi - R)), kd, fy)));
                }
            wsum[py * kAggTX + px] = s > 0.0f ? s : 1.0f;
        }
    }
    float *E = smem + warp * (C::PPG * C::G) * C::EPS;     // this warp's pixels x D
#pragma unroll
    for (int py = 0; py < kAggTY; ++py)
#pragma unroll
        for (int px = 0; px < PX; ++px) {
            float *e = E + (grp * C::PPG + py * PX + px) * C::EPS;
            if (!SR_CHECK((warp * C::PPG * C::G + grp * C::PPG + py * PX + px) * C::EPS + D - 1,
                          kAggPix * C::EPS, 208))
                continue;
            if constexpr (SH) {
#pragma unroll
                for (int q = 0; q < DL / 2; ++q) {
                    e[sh_m[q] + sh_hx * (D / 2)] = acc[py][px][q].x;
                    e[sh_m[q] + (1 - sh_hx) * (D / 2)] = acc[py][px][q].y;
                }
            } else {
                // quad k of the lane: disparities 4 sl + k D/2 .. + 3
#pragma unroll
                for (int k = 0; k < DL / 4; ++k) {
                    float *q4 = e + 4 * sl + k * (D / 2);
                    if constexpr (C::EPS % 4 == 0) {
                        *reinterpret_cast<float4 *>(q4) =
                            make_float4(acc[py][px][2 * k].x, acc[py][px][2 * k].y,
                                        acc[py][px][2 * k + 1].x, acc[py][px][2 * k + 1].y);
                    } else {
                        q4[0] = acc[py][px][2 * k].x;
                        q4[1] = acc[py][px][2 * k].y;
                        q4[2] = acc[py][px][2 * k + 1].x;
                        q4[3] = acc[py][px][2 * k + 1].y;
                    }
                }
            }
        }
    if (pdl == 2) pdl_wait();   // the target labels' grid is complete (see pdl_trigger)
    __syncthreads();
    for (int pw = lane; pw < C::PPG * C::G; pw += 32) {
        const int g = pw / C::PPG, py = (pw % C::PPG) / PX, px = pw % PX;
        const int tpx = (warp * C::G + g) * PX + px;
        const int u = x0 + tpx, v = y0 + py;
        if (u >= W || v >= H) continue;
        if (!SR_CHECK((warp * C::PPG * C::G + pw) * C::EPS + D - 1, kAggPix * C::EPS, 209)) continue;
        const float *e = E + pw * C::EPS;
        const size_t o = (size_t)v * W + u;
        // search window in slice indices: 0..D-1, or the pixel's window
        int lo = 0, hi = D - 1;
        int best = 0;
        float cb = e[0];
        if constexpr (!WIN) {
            // four sums per load, in disparity order (ties keep the smaller d)
            auto take = [&](float c, int d) {
                if (c > cb) { cb = c; best = d; }
            };
#pragma unroll 4
            for (int k = 0; k < D / 4; ++k) {
                const float4 c = *reinterpret_cast<const float4 *>(e + 4 * k);
                if (k > 0) take(c.x, 4 * k);
                take(c.y, 4 * k + 1);
                take(c.z, 4 * k + 2);
                take(c.w, 4 * k + 3);
            }
        } else {
            int cc = win.centre ? win.centre[o] : win.centre_const;
            cc = min(max(cc, 0), win.dfull - 1);
            lo = max(max(cc - win.radius, 0) - dlo, 0);         // the clamps only
            hi = min(min(cc + win.radius, win.dfull - 1) - dlo, D - 1);   // keep bad input in bounds
            if (hi < lo) hi = lo;
            best = lo;
            cb = e[lo];
            // the aligned quads that cover the window, in disparity order
            if constexpr (C::EPS % 4 != 0) {
                for (int d = lo + 1; d <= hi; ++d)
                    if (e[d] > cb) { cb = e[d]; best = d; }
            } else for (int k = lo >> 2; k <= hi >> 2; ++k) {
                const float4 c = *reinterpret_cast<const float4 *>(e + 4 * k);
                const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int d = 4 * k + t;
                    if (d > lo && d <= hi && cv[t] > cb) { cb = cv[t]; best = d; }
                }
            }
        }
        lbl[o] = (int16_t)(best + dlo);
        if (dsub) {
            float ds = (float)(best + dlo);
            if (best > lo && best < hi) {
                const float cm = e[best - 1], cp = e[best + 1];
                const float den = 2.0f * cm + 2.0f * cp - 4.0f * cb;
                if (den < 0.0f) ds += (cm - cp) / den;
            }
            dsub[o] = ds;
            if (!WIN && win.post.disp) {   // Eq. 11 and Sec. II-C (see AggPost)
                const int l = best + dlo, ur = u - l;
                bool ok = false;
                if (ur >= 0 && SR_CHECK(ur, W, 210))
                    ok = fabsf((float)(l - (int)win.post.lbl_r[(size_t)v * W + ur])) <=
                         win.post.lr_thresh;
                win.post.disp[o] = ok ? post_disp(ds, win.post.rowsh[v]) : __int_as_float(0x7fc00000);
                if (win.post.wta) win.post.wta[o] = (int16_t)l;
            }
        }
    }
    if (agg) {
        for (int pw = 0; pw < C::PPG * C::G; ++pw) {
            const int g = pw / C::PPG, py = (pw % C::PPG) / PX, px = pw % PX;
            const int tpx = (warp * C::G + g) * PX + px;
            const int u = x0 + tpx, v = y0 + py;
            if (u >= W || v >= H) continue;
            const float sc = 1.0f / wsum[py * kAggTX + tpx];
            for (int d = lane; d < D; d += 32)
                agg[((size_t)v * W + u) * D + d] = E[pw * C::EPS + d] * sc;
        }
    }
}

template <int R, int D, bool GU8, typename VT, bool WIN>
__global__ void __launch_bounds__(AggCfg<R, D, VT>::NT, AggCfg<R, D, VT>::MINB)
k_agg_wta(const VT *__restrict__ vol, const uint8_t *__restrict__ gl, int pitch,
          const float *__restrict__ gf, int W, int H, float kd, float kr,
          int16_t *__restrict__ lbl, float *__restrict__ dsub, float *__restrict__ agg,
          int *__restrict__ err, long long wait_cycles, int withhold_last, AggWin win,
          int vpitch, int pdl) {
    // restricted search: tiles of the band kernel are not this kernel's
    if (WIN && win.band && win.band[blockIdx.y * gridDim.x + blockIdx.x] >= 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const AggSmem<R, D, VT> sm{smem_raw};
    agg_init_barriers(sm);
    unsigned ph = 0;
    agg_tile<R, D, GU8, VT, false, WIN>(sm, ph, vol, vpitch, gl, pitch, gf, W, H, kd, kr, lbl, dsub, agg,
                                        err, wait_cycles, withhold_last, blockIdx.x * kAggTX,
                                        blockIdx.y * kAggTY, nullptr, 0, win, pdl);
}

// Target view from the extended reference volume (see AggCfg): the guide is
// the warped target, no subpixel map.
template <int R, int D, typename VT>
__global__ void __launch_bounds__(AggCfg<R, D, VT, true>::NT, AggCfg<R, D, VT, true>::MINB)
k_agg_shear(const __grid_constant__ CUtensorMap tmap, int vpitch, const float *__restrict__ gf,
            int W, int H, float kd, float kr, int16_t *__restrict__ lbl, float *__restrict__ agg,
            int *__restrict__ err, long long wait_cycles, int withhold_last, int pdl) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const AggSmem<R, D, VT, true> sm{smem_raw};
    agg_init_barriers(sm);
    unsigned ph = 0;
    agg_tile<R, D, false, VT, false, false, true>(sm, ph, nullptr, vpitch, nullptr, 0, gf, W, H,
                                                  kd, kr, lbl, nullptr, agg, err, wait_cycles,
                                                  withhold_last, blockIdx.x * kAggTX,
                                                  blockIdx.y * kAggTY, &tmap, 0, AggWin(), pdl);
}

// Band kernel of the restricted search: the tile's kBandD-disparity slice
// [band, band + kBandD) through a 2-D tensor map of the volume.
template <int R, bool GU8, typename VT>
__global__ void __launch_bounds__(AggCfg<R, kBandD, VT, false, true>::NT,
                                  AggCfg<R, kBandD, VT, false, true>::MINB)
k_agg_band(const __grid_constant__ CUtensorMap tmap, const uint8_t *__restrict__ gl, int pitch,
           const float *__restrict__ gf, int W, int H, float kd, float kr,
           int16_t *__restrict__ lbl, float *__restrict__ dsub, int *__restrict__ err,
           long long wait_cycles, AggWin win) {
    const int dlo = win.band[blockIdx.y * gridDim.x + blockIdx.x];
    if (dlo < 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const AggSmem<R, kBandD, VT, false, true> sm{smem_raw};
    agg_init_barriers(sm);
    unsigned ph = 0;
    agg_tile<R, kBandD, GU8, VT, true>(sm, ph, nullptr, W, gl, pitch, gf, W, H, kd, kr, lbl, dsub,
                                       nullptr, err, wait_cycles, 0, blockIdx.x * kAggTX,
                                       blockIdx.y * kAggTY, &tmap, dlo, win);
}

// Persistent batched form: CTA b handles work items b, b + gridDim.x, ... of
// the batch's flat (pair, tile) list.  TARGET selects the target volume
// (guide = warped target, no subpixel map) or the reference volume.
template <int R, int D, bool TARGET, typename VT>
__global__ void __launch_bounds__(AggCfg<R, D, VT>::NT, AggCfg<R, D, VT>::MINB)
k_agg_batch(const PairDesc *__restrict__ pairs, const int *__restrict__ start, int n, float kd,
            float kr, int *__restrict__ err, long long wait_cycles, int *__restrict__ next) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const AggSmem<R, D, VT> sm{smem_raw};
    agg_init_barriers(sm);
    // The loop state lives in shared memory and is re-read after each tile,
    // so that none of it occupies registers while a tile runs (the tile
    // needs all 128).  s_state[0]: current work item, s_state[1]: its pair.
    int *s_state = sm.next_slot();
    stage_start(sm.start(), start, n);
    if (threadIdx.x == 0) { s_state[0] = -1; s_state[1] = 0; }
    unsigned ph = 0;
    for (;;) {
        // next work item: in order from a counter (keeps the tiles in flight a
        // contiguous band, so halo rows are shared through L2), or strided
        __syncthreads();   // the previous tile's epilogue is done with shared memory
        if (threadIdx.x == 0) {
            const int *st = n + 1 <= kStartSmem ? sm.start() : start;
            const int prev = s_state[0];
            const int t = next ? atomicAdd(next, 1) : (prev < 0 ? (int)blockIdx.x : prev + (int)gridDim.x);
            s_state[0] = t;
            s_state[1] = t < st[n] ? find_pair(st, n, t, s_state[1]) : -1;
        }
        __syncthreads();
        const int t = s_state[0], p = s_state[1];
        if (p < 0) break;
        const int *st = n + 1 <= kStartSmem ? sm.start() : start;
        const PairDesc &P = pairs[p];
        const int tl = t - st[p], tx = (P.W + kAggTX - 1) / kAggTX;
        agg_tile<R, D, !TARGET, VT>(sm, ph, static_cast<const VT *>(TARGET ? P.vol_r : P.vol_l),
                                    P.W, TARGET ? nullptr : P.left, P.pitch, TARGET ? P.rw : nullptr,
                                    P.W, P.H, kd, kr, TARGET ? P.lbl_r : P.lbl_l,
                                    TARGET ? nullptr : P.dsub, nullptr, err, wait_cycles, 0,
                                    (tl % tx) * kAggTX, (tl / tx) * kAggTY);
    }
}

// Launch k on st; with pdl, as a programmatic dependent of the stream's
// previous kernel (it may start before that kernel ends; see pdl_trigger).
template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args &&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

template <int R, int D, typename VT, bool WIN>
cudaError_t agg_launch_t(const VT *vol, const uint8_t *gl, int pitch, const float *gf, int W,
                         int H, float kd, float kr, int16_t *lbl, float *dsub, float *agg,
                         const AggDebug &dbg, cudaStream_t st, const AggWin &win, int vpitch) {
    using C = AggCfg<R, D, VT>;
    const dim3 grid((W + kAggTX - 1) / kAggTX, (H + kAggTY - 1) / kAggTY);
    auto k = gl ? k_agg_wta<R, D, true, VT, WIN> : k_agg_wta<R, D, false, VT, WIN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_SINGLE);
    if (e != cudaSuccess) return e;
    // the fused L-R check waits for the target view's grid (see pdl_trigger)
    const int pdl = dbg.pdl && win.post.disp ? 2 : 0;
    e = launch_k(pdl != 0, k, grid, dim3(C::NT), C::SMEM_SINGLE, st, vol, gl, pitch, gf, W, H, kd,
                 kr, lbl, dsub, agg, dbg.err, dbg.wait_cycles, dbg.withhold_last, win, vpitch,
                 pdl);
    cudaError_t el = e != cudaSuccess ? e : cudaGetLastError();
    SR_OOB_COLLECT(el, st);
    return el;
}

template <int R, int D, typename VT>
cudaError_t agg_shear_launch_t(const CUtensorMap &tmap, int vpitch, const float *gf, int W,
                               int H, float kd, float kr, int16_t *lbl, float *agg,
                               const AggDebug &dbg, cudaStream_t st) {
    using C = AggCfg<R, D, VT, true>;
    const dim3 grid((W + kAggTX - 1) / kAggTX, (H + kAggTY - 1) / kAggTY);
    auto k = k_agg_shear<R, D, VT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_SINGLE);
    if (e != cudaSuccess) return e;
    const int pdl = dbg.pdl ? 1 : 0;   // the first cost-row copy waits for the NCC grid
    e = launch_k(pdl != 0, k, grid, dim3(C::NT), C::SMEM_SINGLE, st, tmap, vpitch, gf, W, H, kd,
                 kr, lbl, agg, dbg.err, dbg.wait_cycles, dbg.withhold_last, pdl);
    cudaError_t el = e != cudaSuccess ? e : cudaGetLastError();
    SR_OOB_COLLECT(el, st);
    return el;
}

template <int R, typename VT>
cudaError_t agg_band_launch_t(const CUtensorMap &tmap, const uint8_t *gl, int pitch,
                              const float *gf, int W, int H, float kd, float kr, int16_t *lbl,
                              float *dsub, const AggDebug &dbg, const AggWin &win,
                              cudaStream_t st) {
    using C = AggCfg<R, kBandD, VT, false, true>;
    const dim3 grid((W + kAggTX - 1) / kAggTX, (H + kAggTY - 1) / kAggTY);
    auto k = gl ? k_agg_band<R, true, VT> : k_agg_band<R, false, VT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_SINGLE);
    if (e != cudaSuccess) return e;
    k<<<grid, C::NT, C::SMEM_SINGLE, st>>>(tmap, gl, pitch, gf, W, H, kd, kr, lbl, dsub, dbg.err,
                                    dbg.wait_cycles, win);
    cudaError_t el = cudaGetLastError();
    SR_OOB_COLLECT(el, st);
    return el;
}

template <int R, int D, typename VT>
cudaError_t agg_batch_t(bool target, const PairDesc *pairs, const int *start, int n, float kd,
                        float kr, const AggDebug &dbg, int grid, int *next, cudaStream_t st) {
    using C = AggCfg<R, D, VT>;
    auto k = target ? k_agg_batch<R, D, true, VT> : k_agg_batch<R, D, false, VT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    k<<<grid, C::NT, C::SMEM, st>>>(pairs, start, n, kd, kr, dbg.err, dbg.wait_cycles, next);
    cudaError_t el = cudaGetLastError();
    SR_OOB_COLLECT(el, st);
    return el;
}

template <int R, int D, typename VT>
int agg_occ_t() {
    using C = AggCfg<R, D, VT>;
    int b = 0;
    cudaFuncSetAttribute(k_agg_batch<R, D, false, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)C::SMEM);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_agg_batch<R, D, false, VT>, C::NT, C::SMEM);
    return b;
}

#define SR_AGG_R_SWITCH(agg_r, CALL)                 \
    switch (agg_r) {                                 \
        case 1: { constexpr int R_ = 1; CALL; }      \
        case 2: { constexpr int R_ = 2; CALL; }      \
        case 3: { constexpr int R_ = 3; CALL; }      \
        case 4: { constexpr int R_ = 4; CALL; }      \
        case 5: { constexpr int R_ = 5; CALL; }      \
        case 6: { constexpr int R_ = 6; CALL; }      \
        case 7: { constexpr int R_ = 7; CALL; }      \
        default: break;                              \
    }

template <int D, typename VT, bool WIN>
cudaError_t agg_launch_d(const VT *vol, const uint8_t *gl, int pitch, const float *gf, int W,
                         int H, int agg_r, float kd, float kr, int16_t *lbl, float *dsub,
                         float *agg, const AggDebug &dbg, cudaStream_t st, const AggWin &win,
                         int vpitch) {
    SR_AGG_R_SWITCH(agg_r, return (agg_launch_t<R_, D, VT, WIN>(vol, gl, pitch, gf, W, H, kd, kr,
                                                                lbl, dsub, agg, dbg, st, win,
                                                                vpitch)))
    return cudaErrorInvalidValue;
}

// The box of the sheared kernel's tensor map: CW disparities x BH pixels.
template <int R, int D, typename VT>
void agg_shear_box_t(int *cw, int *bh) {
    using C = AggCfg<R, D, VT, true>;
    *cw = C::CW;
    *bh = C::BH;
}

template <int D, typename VT>
bool agg_shear_box_d(int agg_r, int *cw, int *bh) {
    SR_AGG_R_SWITCH(agg_r, return (agg_shear_box_t<R_, D, VT>(cw, bh), true))
    return false;
}

template <int D, typename VT>
cudaError_t agg_shear_launch_d(const CUtensorMap &tmap, int vpitch, const float *gf, int W, int H,
                               int agg_r, float kd, float kr, int16_t *lbl, float *agg,
                               const AggDebug &dbg, cudaStream_t st) {
    SR_AGG_R_SWITCH(agg_r, return (agg_shear_launch_t<R_, D, VT>(tmap, vpitch, gf, W, H, kd, kr,
                                                                 lbl, agg, dbg, st)))
    return cudaErrorInvalidValue;
}

template <typename VT>
cudaError_t agg_band_launch_d(const CUtensorMap &tmap, const uint8_t *gl, int pitch,
                              const float *gf, int W, int H, int agg_r, float kd, float kr,
                              int16_t *lbl, float *dsub, const AggDebug &dbg, const AggWin &win,
                              cudaStream_t st) {
    SR_AGG_R_SWITCH(agg_r, return (agg_band_launch_t<R_, VT>(tmap, gl, pitch, gf, W, H, kd, kr,
                                                             lbl, dsub, dbg, win, st)))
    return cudaErrorInvalidValue;
}

template <int D, typename VT>
cudaError_t agg_batch_d(bool target, const PairDesc *pairs, const int *start, int n, int agg_r,
                        float kd, float kr, const AggDebug &dbg, int grid, int *next,
                        cudaStream_t st) {
    SR_AGG_R_SWITCH(agg_r, return (agg_batch_t<R_, D, VT>(target, pairs, start, n, kd, kr, dbg,
                                                          grid, next, st)))
    return cudaErrorInvalidValue;
}

template <int D, typename VT>
int agg_occ_d(int agg_r) {
    SR_AGG_R_SWITCH(agg_r, return (agg_occ_t<R_, D, VT>()))
    return 0;
}

}  // namespace sr
