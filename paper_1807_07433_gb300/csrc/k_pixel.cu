// k_pixel.cu -- per-pixel stages: perspective transformation (Sec. II-A),
// block statistics (Eqs. 4-5), L-R check + post-processing (Eq. 11,
// Sec. II-C) and 3-D reconstruction (Sec. II-D).  All are O(W*H) and
// bandwidth-trivial next to the cost volumes; one thread per output pixel,
// 2-D blocks of 32x8 so that a warp reads 32 consecutive pixels of a row.
#include <math.h>

#include "sr_internal.cuh"

namespace sr {
namespace {

constexpr int kBX = kPixTX, kBY = kPixTY;

__device__ __forceinline__ void warp_px(const uint8_t *__restrict__ right, int pitch, int W,
                                        double alpha0, double alpha1, double delta,
                                        float *__restrict__ rw, int x, int v) {
    // s(v) of Sec. II-A, evaluated per pixel here (the batched form)
    const double s = row_shift(alpha0, alpha1, delta, v);
    double k = floor(s);
    const float w = (float)(s - k);
    k = fmin(fmax(k, -2.0 * W - 2.0), 2.0 * W + 2.0);   // beyond this every read clamps
    const int ki = (int)k;
    const uint8_t *row = right + (size_t)v * pitch;
    const float a = row[clampi(x - ki, 0, W - 1)];
    const float b = row[clampi(x - ki - 1, 0, W - 1)];
    rw[(size_t)v * W + x] = fmaf(w, b - a, a);        // (1-w) a + w b
}

__global__ void k_warp(const uint8_t *__restrict__ right, int pitch, int W, int H, double alpha0,
                       double alpha1, double delta, float *__restrict__ rw) {
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int v = blockIdx.y * kBY + threadIdx.y;
    if (x >= W || v >= H) return;
    warp_px(right, pitch, W, alpha0, alpha1, delta, rw, x, v);
}

// Left block statistics from exact integer sums: n^2 sigma^2 = n S2 - S^2.
// Centres x in [0, W+D-1) (the target volume needs left blocks at u+d).
template <int RN>
__device__ __forceinline__ void stats_left_px(const uint8_t *__restrict__ left, int pitch, int W,
                                              int H, int WE, float *__restrict__ mu,
                                              float *__restrict__ inv, int x, int v) {
    constexpr int n = (2 * RN + 1) * (2 * RN + 1);
    unsigned s = 0, s2 = 0;
#pragma unroll
    for (int j = -RN; j <= RN; ++j) {
        const uint8_t *row = left + (size_t)clampi(v + j, 0, H - 1) * pitch;
#pragma unroll
        for (int i = -RN; i <= RN; ++i) {
            const unsigned val = row[clampi(x + i, 0, W - 1)];
            s += val;
            s2 += val * val;
        }
    }
    const long long q = (long long)n * s2 - (long long)s * s;   // n^2 var, exact
    const float var = (float)q / (float)(n * n);
    inv[(size_t)v * WE + x] = (var < kFlatVar) ? 0.0f : 1.0f / sqrtf((float)q);
    mu[(size_t)v * WE + x] = (float)s / (float)n;
}

template <int RN>
__global__ void k_stats_left(const uint8_t *__restrict__ left, int pitch, int W, int H, int WE,
                             float *__restrict__ mu, float *__restrict__ inv) {
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int v = blockIdx.y * kBY + threadIdx.y;
    if (x >= WE || v >= H) return;
    stats_left_px<RN>(left, pitch, W, H, WE, mu, inv, x, v);
}

template <int RN>
__device__ __forceinline__ void stats_right_px(const float *__restrict__ rw, int W, int H, int D,
                                               int WE, float *__restrict__ mu,
                                               float *__restrict__ inv, int xi, int v) {
    const int x = xi - (D - 1);
    constexpr int n = (2 * RN + 1) * (2 * RN + 1);
    // Mean: row sums of (value - 128) then their sum, so that no partial sum
    // grows past a few thousand (FP32 rounding ~1e-6 of an intensity).
    float val[2 * RN + 1][2 * RN + 1];
    float s = 0.0f;
#pragma unroll
    for (int j = -RN; j <= RN; ++j) {
        const float *row = rw + (size_t)clampi(v + j, 0, H - 1) * W;
        float rs = 0.0f;
#pragma unroll
        for (int i = -RN; i <= RN; ++i) {
            val[j + RN][i + RN] = row[clampi(x + i, 0, W - 1)];
            rs += val[j + RN][i + RN] - kNccOffset;
        }
        s += rs;
    }
    const float m = kNccOffset + s / (float)n;
    float q = 0.0f;
#pragma unroll
    for (int j = 0; j <= 2 * RN; ++j)
#pragma unroll
        for (int i = 0; i <= 2 * RN; ++i) {
            const float c = val[j][i] - m;
            q = fmaf(c, c, q);
        }
    // q = n sigma^2; 1/(n sigma) = 1/sqrt(n q)
    inv[(size_t)v * WE + xi] = (q / (float)n < kFlatVar) ? 0.0f : 1.0f / sqrtf((float)n * q);
    mu[(size_t)v * WE + xi] = m;
}

// Warped-target block statistics, two-pass (mean, then centred squares).
// Centres x in [-(D-1), W), stored at x + D - 1.
template <int RN>
__global__ void k_stats_right(const float *__restrict__ rw, int W, int H, int D, int WE,
                              float *__restrict__ mu, float *__restrict__ inv) {
    const int xi = blockIdx.x * kBX + threadIdx.x;
    const int v = blockIdx.y * kBY + threadIdx.y;
    if (xi >= WE || v >= H) return;
    stats_right_px<RN>(rw, W, H, D, WE, mu, inv, xi, v);
}

__device__ __forceinline__ void lrc_px(const int16_t *__restrict__ lbl_l,
                                       const int16_t *__restrict__ lbl_r,
                                       const float *__restrict__ dsub, int W, float2 sh,
                                       float lr_thresh, float *__restrict__ disp,
                                       int16_t *__restrict__ wta_out, int u, int v) {
    const size_t i = (size_t)v * W + u;
    const int l = lbl_l[i];
    const int ur = u - l;
    bool ok = false;
    if (ur >= 0 && SR_CHECK(ur, W, 301)) ok = fabsf((float)(l - (int)lbl_r[(size_t)v * W + ur])) <= lr_thresh;
    disp[i] = ok ? post_disp(dsub[i], sh) : __int_as_float(0x7fc00000);
    if (wta_out) wta_out[i] = (int16_t)l;
}

// Each thread checks kLrcPX pixels of one row, kBX apart (so that every
// access of a warp stays coalesced): independent loads in flight per thread
// and a grid of about one wave, for a kernel that is all memory latency.
constexpr int kLrcPX = 4;

__global__ void k_lrc_post(const int16_t *__restrict__ lbl_l, const int16_t *__restrict__ lbl_r,
                           const float *__restrict__ dsub, int W, int H,
                           const float2 *__restrict__ rowsh, float lr_thresh,
                           float *__restrict__ disp, int16_t *__restrict__ wta_out) {
    const int u0 = blockIdx.x * kBX * kLrcPX + threadIdx.x;
    const int v = blockIdx.y * kBY + threadIdx.y;
    if (v >= H) return;
    const float2 sh = rowsh[v];
#pragma unroll
    for (int i = 0; i < kLrcPX; ++i) {
        const int u = u0 + i * kBX;
        if (u < W) lrc_px(lbl_l, lbl_r, dsub, W, sh, lr_thresh, disp, wta_out, u, v);
    }
}

// ---- batched forms: persistent 32x8 blocks over a batch's flat tile list --
// Tile t of pair p covers columns [tx*32, tx*32+32) of the stage's width
// (W, or W + D - 1 for the statistics) and rows [ty*8, ty*8+8).
__device__ __forceinline__ bool batch_pixel(const PairDesc *pairs, const int *start, int n, int t,
                                            int extra_w, const PairDesc **P, int *x, int *v,
                                            int *pp) {
    const int p = find_pair(start, n, t, *pp);
    *pp = p;
    *P = &pairs[p];
    const int w = (*P)->W + extra_w;
    const int tl = t - start[p], tx = (w + kBX - 1) / kBX;
    *x = (tl % tx) * kBX + threadIdx.x;
    *v = (tl / tx) * kBY + threadIdx.y;
    return *x < w && *v < (*P)->H;
}

__global__ void k_warp_batch(const PairDesc *__restrict__ pairs, const int *__restrict__ start,
                             int n) {
    __shared__ int s_start[kStartSmem];
    const int *st = stage_start(s_start, start, n);
    int pp = 0;
    for (int t = blockIdx.x; t < st[n]; t += gridDim.x) {
        const PairDesc *P;
        int x, v;
        if (batch_pixel(pairs, st, n, t, 0, &P, &x, &v, &pp)) {
            warp_px(P->right, P->pitch, P->W, P->alpha0, P->alpha1, P->delta, P->rw, x, v);
            if (x == 0) P->rowsh[v] = split_shift(row_shift(P->alpha0, P->alpha1, P->delta, v));
        }
    }
}

template <int RN>
__global__ void k_stats_batch(const PairDesc *__restrict__ pairs, const int *__restrict__ start,
                              int n, int D) {
    __shared__ int s_start[kStartSmem];
    const int *st = stage_start(s_start, start, n);
    int pp = 0;
    for (int t = blockIdx.x; t < st[n]; t += gridDim.x) {
        const PairDesc *P;
        int x, v;
        if (batch_pixel(pairs, st, n, t, D - 1, &P, &x, &v, &pp)) {
            const int WE = P->W + D - 1;
            stats_left_px<RN>(P->left, P->pitch, P->W, P->H, WE, P->mu_l, P->inv_l, x, v);
            stats_right_px<RN>(P->rw, P->W, P->H, D, WE, P->mu_r, P->inv_r, x, v);
        }
    }
}

__global__ void k_lrc_post_batch(const PairDesc *__restrict__ pairs, const int *__restrict__ start,
                                 int n, float lr_thresh) {
    __shared__ int s_start[kStartSmem];
    const int *st = stage_start(s_start, start, n);
    int pp = 0;
    for (int t = blockIdx.x; t < st[n]; t += gridDim.x) {
        const PairDesc *P;
        int x, v;
        if (batch_pixel(pairs, st, n, t, 0, &P, &x, &v, &pp))
            lrc_px(P->lbl_l, P->lbl_r, P->dsub, P->W, P->rowsh[v], lr_thresh, P->disp, P->wta,
                   x, v);
    }
}

__global__ void k_xyz(const float *__restrict__ disp, int W, int H, float f, float fb, float u0,
                      float v0, float *__restrict__ xyz, int selftest) {
    const int u = blockIdx.x * kBX + threadIdx.x;
    const int v = blockIdx.y * kBY + threadIdx.y;
    if (selftest && u == 0 && v == 0) (void)SR_CHECK(-1, 1, 399);   // no access follows
    if (u >= W || v >= H) return;
    const size_t i = (size_t)v * W + u, npx = (size_t)W * H;
    const float d = disp[i];
    float X, Y, Z;
    if (!(d > 0.0f) || isinf(d)) {
        X = Y = Z = __int_as_float(0x7fc00000);
    } else {
        Z = fb / d;
        X = ((float)u - u0) * Z / f;
        Y = ((float)v - v0) * Z / f;
    }
    xyz[i] = X;
    xyz[npx + i] = Y;
    xyz[2 * npx + i] = Z;
}

dim3 grid_for(int w, int h) { return dim3((w + kBX - 1) / kBX, (h + kBY - 1) / kBY); }

// Fused perspective transformation (Sec. II-A) and block statistics (Eqs.
// 4-5) of both images, for one 32 x 8 tile of extended block centres: the
// tile's left rows and its warped-target rows (each with the block halo,
// clamp-to-edge) are staged in shared memory once, the row shifts once per
// row, and the warped image is written for the columns this tile owns.
// Left statistics: sliding-window sums, separable -- column sums of the
// block's rows for every staged column, then each centre sums 2 RN + 1 of
// them -- in exact integers, so they equal stats_left_px's.  Warped-target
// statistics: the centred two-pass form of stats_right_px, in its order (a
// running sum of squares would cancel in FP32 on smooth blocks).  A thread
// computes two vertically adjacent centres, whose blocks share 2 RN rows:
// their 2 RN + 2 rows of values are read from shared memory once, into
// registers, and the row sums of (value - 128) serve both means.
template <int RN>
__global__ void __launch_bounds__(kBX * kBY / 2)
k_prep(const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, int pitch, int W,
       int H, int D, double alpha0, double alpha1, double delta, int row0,
       float *__restrict__ rw, float *__restrict__ mu_l, float *__restrict__ inv_l,
       float *__restrict__ mu_r, float *__restrict__ inv_r, float2 *__restrict__ rowsh) {
    constexpr int B = 2 * RN + 1, TH = kBY + 2 * RN, TW = kBX + 2 * RN;
    constexpr int n = B * B;
    constexpr int NT = kBX * kBY / 2;     // threads: each computes two rows of the tile
    __shared__ int s_l[TH][TW];           // left intensities
    __shared__ float s_r[TH][TW];         // warped target intensities
    __shared__ unsigned s_cs[kBY][TW];    // left column sums over the block rows
    __shared__ unsigned s_cs2[kBY][TW];   // ... of squares
    __shared__ int s_k[TH];               // row shift: integer part
    __shared__ float s_w[TH];             // row shift: fraction
    const int WE = W + D - 1;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY;
    const int xr0 = x0 - (D - 1);         // first target-block centre of the tile
    if (tid < TH) {
        const int y = clampi(y0 - RN + tid, 0, H - 1);
        const double sh = row_shift(alpha0, alpha1, delta, y + row0);
        if (blockIdx.x == 0 && tid >= RN && tid < RN + kBY && y0 - RN + tid < H &&
            SR_CHECK(y0 - RN + tid, H, 302))
            rowsh[y0 - RN + tid] = split_shift(sh);   // one column of tiles writes each row
        double k = floor(sh);
        s_w[tid] = (float)(sh - k);
        k = fmin(fmax(k, -2.0 * W - 2.0), 2.0 * W + 2.0);   // beyond this every read clamps
        s_k[tid] = (int)k;
    }
    __syncthreads();
    {   // all loads of a thread first, then the stores: their latencies overlap
        constexpr int NI = (TH * TW + NT - 1) / NT;
        int lv[NI];
        float av[NI], bv[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int i = min(tid + k * NT, TH * TW - 1);
            const int r = i / TW, c = i % TW;
            const int y = clampi(y0 - RN + r, 0, H - 1);
            const int xl = clampi(x0 - RN + c, 0, W - 1);
            const int x = clampi(xr0 - RN + c, 0, W - 1);
            const int xa = clampi(x - s_k[r], 0, W - 1), xb = clampi(x - s_k[r] - 1, 0, W - 1);
            const uint8_t *row = right + (size_t)y * pitch;
            const bool okl = SR_CHECK(xl, pitch, 303) && SR_CHECK(y, H, 303);
            const bool okr = SR_CHECK(xa, pitch, 304) && SR_CHECK(xb, pitch, 304);
            lv[k] = okl ? left[(size_t)y * pitch + xl] : 0;
            av[k] = okr && okl ? row[xa] : 0.0f;
            bv[k] = okr && okl ? row[xb] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            const int i = tid + k * NT;
            if (i < TH * TW) {
                const int r = i / TW, c = i % TW;
                s_l[r][c] = lv[k];
                s_r[r][c] = fmaf(s_w[r], bv[k] - av[k], av[k]);   // (1-w) a + w b
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < kBY * TW; i += NT) {   // column sums of B rows
        const int r = i / TW, c = i % TW;
        unsigned cs = 0, cs2 = 0;
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const unsigned val = (unsigned)s_l[r + j][c];
            cs += val;
            cs2 += val * val;
        }
        s_cs[r][c] = cs;
        s_cs2[r][c] = cs2;
    }
    __syncthreads();
    // this thread: tile rows ty and ty + 1 of column tx; their warped blocks
    // share B - 1 rows, so the B + 1 rows of values are read once into
    // registers.  Each pixel's arithmetic is the order of stats_right_px.
    const int tx = threadIdx.x, ty = 2 * threadIdx.y;
    const int xi = x0 + tx;
    if (xi >= WE) return;
    float vv[B + 1][B];
#pragma unroll
    for (int j = 0; j < B + 1; ++j)
#pragma unroll
        for (int i = 0; i < B; ++i) vv[j][i] = s_r[ty + j][tx + i];
    // row sums of (value - 128), shared by the two blocks
    float rsum[B + 1];
#pragma unroll
    for (int j = 0; j < B + 1; ++j) {
        float rs = 0.0f;
#pragma unroll
        for (int i = 0; i < B; ++i) rs += vv[j][i] - kNccOffset;
        rsum[j] = rs;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = ty + h, v = y0 + r;
        if (v >= H) break;
        if (!SR_CHECK((size_t)v * WE + xi, (long long)H * WE, 305)) break;
        // left block at centre xi (exact integer sums)
        {
            unsigned su = 0, s2 = 0;
#pragma unroll
            for (int i = 0; i < B; ++i) {
                su += s_cs[r][tx + i];
                s2 += s_cs2[r][tx + i];
            }
            const long long q = (long long)n * s2 - (long long)su * su;   // n^2 var, exact
            const float var = (float)q / (float)(n * n);
            inv_l[(size_t)v * WE + xi] = (var < kFlatVar) ? 0.0f : 1.0f / sqrtf((float)q);
            mu_l[(size_t)v * WE + xi] = (float)su / (float)n;
        }
        // warped-target block at centre xi - (D-1): mean from row sums of
        // (value - 128), then centred squares
        {
            float s = 0.0f;
#pragma unroll
            for (int j = 0; j < B; ++j) s += rsum[h + j];
            const float m = kNccOffset + s / (float)n;
            float q = 0.0f;
#pragma unroll
            for (int j = 0; j < B; ++j)
#pragma unroll
                for (int i = 0; i < B; ++i) {
                    const float c = vv[h + j][i] - m;
                    q = fmaf(c, c, q);
                }
            inv_r[(size_t)v * WE + xi] = (q / (float)n < kFlatVar) ? 0.0f : 1.0f / sqrtf((float)n * q);
            mu_r[(size_t)v * WE + xi] = m;
        }
        // the warped image, at the target columns this tile owns
        const int xr = xi - (D - 1);
        if (xr >= 0 && SR_CHECK(xr, W, 306)) rw[(size_t)v * W + xr] = vv[h + RN][RN];
    }
}

}  // namespace

cudaError_t launch_prep(const uint8_t *left, const uint8_t *right, int pitch, int W, int H, int D,
                        int ncc_r, double alpha0, double alpha1, double delta, int row0,
                        float *rw, float *mu_l, float *inv_l, float *mu_r, float *inv_r,
                        float2 *rowsh, cudaStream_t st) {
    const dim3 grid = grid_for(W + D - 1, H), block(kBX, kBY / 2);
    switch (ncc_r) {
#define SR_PREP(RN_)                                                                          \
    case RN_:                                                                                 \
        k_prep<RN_><<<grid, block, 0, st>>>(left, right, pitch, W, H, D, alpha0, alpha1, delta, \
                                            row0, rw, mu_l, inv_l, mu_r, inv_r, rowsh);        \
        break;
        SR_PREP(1) SR_PREP(2) SR_PREP(3) SR_PREP(4) SR_PREP(5)
#undef SR_PREP
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_warp(const uint8_t *right, int pitch, int W, int H, double alpha0,
                        double alpha1, double delta, float *rw, cudaStream_t st) {
    k_warp<<<grid_for(W, H), dim3(kBX, kBY), 0, st>>>(right, pitch, W, H, alpha0, alpha1, delta, rw);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

template <int RN>
static void stats_rn(const uint8_t *left, int pitch, const float *rw, int W, int H, int D,
                     float *mu_l, float *inv_l, float *mu_r, float *inv_r, cudaStream_t st) {
    const int WE = W + D - 1;
    k_stats_left<RN><<<grid_for(WE, H), dim3(kBX, kBY), 0, st>>>(left, pitch, W, H, WE, mu_l, inv_l);
    k_stats_right<RN><<<grid_for(WE, H), dim3(kBX, kBY), 0, st>>>(rw, W, H, D, WE, mu_r, inv_r);
}

cudaError_t launch_stats(const uint8_t *left, int pitch, const float *rw, int W, int H, int D,
                         int ncc_r, float *mu_l, float *inv_l, float *mu_r, float *inv_r,
                         cudaStream_t st) {
    switch (ncc_r) {
        case 1: stats_rn<1>(left, pitch, rw, W, H, D, mu_l, inv_l, mu_r, inv_r, st); break;
        case 2: stats_rn<2>(left, pitch, rw, W, H, D, mu_l, inv_l, mu_r, inv_r, st); break;
        case 3: stats_rn<3>(left, pitch, rw, W, H, D, mu_l, inv_l, mu_r, inv_r, st); break;
        case 4: stats_rn<4>(left, pitch, rw, W, H, D, mu_l, inv_l, mu_r, inv_r, st); break;
        case 5: stats_rn<5>(left, pitch, rw, W, H, D, mu_l, inv_l, mu_r, inv_r, st); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_lrc_post(const int16_t *lbl_l, const int16_t *lbl_r, const float *dsub, int W,
                            int H, const float2 *rowsh, float lr_thresh, float *disp,
                            int16_t *wta_out, cudaStream_t st) {
    k_lrc_post<<<grid_for(ceil_div(W, kLrcPX), H), dim3(kBX, kBY), 0, st>>>(
        lbl_l, lbl_r, dsub, W, H, rowsh, lr_thresh, disp, wta_out);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_warp_batch(const PairDesc *pairs, const int *start, int n, int grid,
                              cudaStream_t st) {
    k_warp_batch<<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_stats_batch(const PairDesc *pairs, const int *start, int n, int D, int ncc_r,
                               int grid, cudaStream_t st) {
    switch (ncc_r) {
        case 1: k_stats_batch<1><<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, D); break;
        case 2: k_stats_batch<2><<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, D); break;
        case 3: k_stats_batch<3><<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, D); break;
        case 4: k_stats_batch<4><<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, D); break;
        case 5: k_stats_batch<5><<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, D); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_lrc_post_batch(const PairDesc *pairs, const int *start, int n, float lr_thresh,
                                  int grid, cudaStream_t st) {
    k_lrc_post_batch<<<grid, dim3(kBX, kBY), 0, st>>>(pairs, start, n, lr_thresh);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

cudaError_t launch_xyz(const float *disp, int W, int H, double f_px, double baseline, double u0,
                       double v0, float *xyz, cudaStream_t st, bool selftest) {
    k_xyz<<<grid_for(W, H), dim3(kBX, kBY), 0, st>>>(disp, W, H, (float)f_px,
                                                    (float)(f_px * baseline), (float)u0,
                                                    (float)v0, xyz, selftest ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    SR_OOB_COLLECT(e, st);
    return e;
}

}  // namespace sr
