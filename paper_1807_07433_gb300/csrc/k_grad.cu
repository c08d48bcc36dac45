// k_grad.cu -- adjoint of the matching cost with respect to the road plane
// (Sec. II-A, Eq. 2) and the images, for plane refinement.
//
// Objective: L = sum over pixels p with dstar[p] >= 0 of c_agg(p, dstar[p]),
// the aggregated reference cost (Eq. 8) at disparities held fixed.  Chain:
//   c_agg = sum_k w_k c_k / W_p, W_p = sum_k w_k, w_k = omega_d omega_r
//     dL/dc_k += w_k / W_p;  dL/dw_k += (c_k - c_agg) / W_p;
//     d omega_r / d delta = -2 delta / gamma_r^2 omega_r     (Eq. 10, guide i_l)
//   c = n cov / (n sigma_l sigma_r) of the centred blocks a, b (Eq. 3)
//     dc/dr_j = (a_j - c (sigma_l/sigma_r) b_j) / (n sigma_l sigma_r)
//     dc/dl_j = (b_j - c (sigma_r/sigma_l) a_j) / (n sigma_l sigma_r)
//   r = (1-w) i_r(x-k) + w i_r(x-k-1), s = alpha0 + alpha1 v - delta
//     dr/ds = i_r(x-k-1) - i_r(x-k), ds/dalpha = (1, v)
// The forward reference volume c(x, y, d) (Eq. 3, FP32, [H][W][D]) and the
// block statistics are inputs; the weights are recomputed where needed.
//   k_grad_pixel   per pixel of the set: weights, the costs of its window
//                  (read from the volume), c_agg, the pixel's share of L, the
//                  guide-weight gradient (scattered into dL/di_l), and W_p.
//   k_grad_ncc     per (x, y): G(x, y, d) = dL/dc(x, y, d), gathered from the
//                  window pixels whose fixed disparity is d (no atomics), then
//                  the NCC adjoint of each (x, y, d) with G != 0; dL/dalpha is
//                  accumulated in FP64 (block partials, reduced by
//                  k_grad_reduce in a fixed order), the image gradients are
//                  scattered with FP32 atomics.
//   k_grad_warp    per row: adjoint of the warp, dL/di_r from dL/di_r'.
#include <math.h>

#include "sr_internal.cuh"

namespace sr {
namespace {

constexpr int kGT = 256;

struct GradArgs {
    const uint8_t *left, *right;
    int pitch, W, H, D, RN, R;
    const float *rw, *mu_l, *inv_l, *mu_r, *inv_r;   // stats rows of width W + D - 1
    const float *cost;                                 // reference volume [H][W][D]
    const int16_t *dstar;
    double alpha0, alpha1, delta;
    float kd, kr, inv_gr2;                             // log2e/gd^2, log2e/gr^2, 1/gr^2
};

// Block statistics of the Eq. 3 pair at left centre (xl, y), right centre
// (xl - d, y): means and 1/(n sigma) (0 for a flat block).
__device__ __forceinline__ void pair_stats(const GradArgs &a, int xl, int y, int d, float *ml,
                                           float *mr, float *il_, float *ir_) {
    const size_t row = (size_t)y * (a.W + a.D - 1);
    *ml = a.mu_l[row + xl];
    *il_ = a.inv_l[row + xl];
    *mr = a.mu_r[row + xl - d + a.D - 1];
    *ir_ = a.inv_r[row + xl - d + a.D - 1];
}

__device__ __forceinline__ float cost_at(const GradArgs &a, int x, int y, int d) {
    return a.cost[((size_t)y * a.W + x) * a.D + d];
}

__device__ __forceinline__ float weight(const GradArgs &a, int dx, int dy, float dg) {
    return exp2f(-fmaf(dg * dg, a.kr, (float)(dx * dx + dy * dy) * a.kd));
}

// Block-wide FP64 sum of up to three values; thread 0 writes partial[blockIdx].
__device__ void block_sum3(double v0, double v1, double v2, double *partial) {
    __shared__ double s[3][kGT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
        v2 += __shfl_down_sync(0xffffffffu, v2, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s[0][warp] = v0; s[1][warp] = v1; s[2][warp] = v2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int w = 0; w < kGT / 32; ++w) { t0 += s[0][w]; t1 += s[1][w]; t2 += s[2][w]; }
        partial[3 * blockIdx.x + 0] = t0;
        partial[3 * blockIdx.x + 1] = t1;
        partial[3 * blockIdx.x + 2] = t2;
    }
}

// Cost slice tile of k_grad_pixel: rows y-R..y+R, columns x0-R..x0+kGT-1+R
// of c(., ., d) for a block whose pixels share one row y and one label d.
constexpr int kMaxAggR = 7;
constexpr int kTileW = kGT + 2 * kMaxAggR;

__global__ void __launch_bounds__(kGT) k_grad_pixel(GradArgs a, float *__restrict__ wsum,
                                                    float *__restrict__ gl,
                                                    double *__restrict__ partial) {
    __shared__ float tile[(2 * kMaxAggR + 1) * kTileW];
    const int npx = a.W * a.H;
    const int i0 = blockIdx.x * kGT, i = i0 + threadIdx.x;
    const int y0 = i0 / a.W, x0 = i0 % a.W;
    const int d0 = a.dstar[i0];
    // fast path: one row, one in-range label for every pixel of the block
    const bool one_row = x0 + kGT <= a.W || i0 + kGT >= npx && x0 + (npx - i0) <= a.W;
    const int my_d = i < npx ? a.dstar[i] : d0;
    const bool uniform = __syncthreads_and(one_row && d0 >= 0 && d0 < a.D && my_d == d0) != 0;
    if (uniform) {
        const int rows = 2 * a.R + 1, cols = min(kGT, npx - i0) + 2 * a.R;
        for (int t = threadIdx.x; t < rows * cols; t += kGT) {
            const int r = t / cols, cc = t % cols;
            const int y = y0 - a.R + r, x = x0 - a.R + cc;
            if (y >= 0 && y < a.H && x >= 0 && x < a.W)
                tile[r * kTileW + cc] = cost_at(a, x, y, d0);
        }
        __syncthreads();
    }
    double Lp = 0.0;
    if (i < npx) {
        const int u = i % a.W, v = i / a.W;
        const int d = my_d;
        float Wp = 0.0f;
        if (d >= 0 && d < a.D) {   // other values leave the pixel out
            const float gc = (float)a.left[(size_t)v * a.pitch + u];
            // window cost c(u + dx, v + dy, d): from the tile or the volume
            auto cost_w = [&](int dx, int dy) -> float {
                return uniform ? tile[(dy + a.R) * kTileW + (u - x0) + dx + a.R]
                               : cost_at(a, u + dx, v + dy, d);
            };
            float num = 0.0f;
            for (int dy = -a.R; dy <= a.R; ++dy) {
                const int y = v + dy;
                if (y < 0 || y >= a.H) continue;
                for (int dx = -a.R; dx <= a.R; ++dx) {
                    const int x = u + dx;
                    if (x < 0 || x >= a.W) continue;
                    const float w = weight(a, dx, dy, (float)a.left[(size_t)y * a.pitch + x] - gc);
                    num = fmaf(w, cost_w(dx, dy), num);
                    Wp += w;
                }
            }
            const float cagg = num / Wp;
            Lp = cagg;
            // guide-weight gradient: dL/dw_k (dw_k/ddelta_k), delta_k = g(n_k) - g(p)
            float self = 0.0f;
            for (int dy = -a.R; gl && dy <= a.R; ++dy) {
                const int y = v + dy;
                if (y < 0 || y >= a.H) continue;
                for (int dx = -a.R; dx <= a.R; ++dx) {
                    const int x = u + dx;
                    if (x < 0 || x >= a.W) continue;
                    const float dg = (float)a.left[(size_t)y * a.pitch + x] - gc;
                    const float w = weight(a, dx, dy, dg);
                    const float gw = (cost_w(dx, dy) - cagg) / Wp * w * (-2.0f * dg * a.inv_gr2);
                    if (dx != 0 || dy != 0) atomicAdd(&gl[(size_t)y * a.W + x], gw);
                    self -= gw;
                }
            }
            if (gl) atomicAdd(&gl[(size_t)v * a.W + u], self);
        }
        wsum[i] = Wp;
    }
    block_sum3(Lp, 0.0, 0.0, partial);
}

// Integer part k of the row shift s(y) = alpha0 + alpha1 y - delta (Sec. II-A),
// clamped where every read clamps anyway; dr/ds at (x, y) is then
// i_r(x-k-1) - i_r(x-k).
__device__ __forceinline__ int row_shift_floor(const GradArgs &a, int y) {
    const double s = a.alpha0 + a.alpha1 * (double)y - a.delta;
    return (int)fmin(fmax(floor(s), -2.0 * a.W - 2.0), 2.0 * a.W + 2.0);
}

// NCC adjoint of the entry (x, y, d) with incoming gradient g = dL/dc:
// scatters dL/di_r' and dL/di_l (when wanted) and adds dL/dalpha to s0, s1.
__device__ void ncc_adjoint(const GradArgs &a, int x, int y, int d, float g, float *grw,
                            float *gl, double &s0, double &s1) {
    float ml, mr, il_, ir_;
    pair_stats(a, x, y, d, &ml, &mr, &il_, &ir_);
    if (il_ == 0.0f || ir_ == 0.0f) return;            // flat block: c == 0 locally
    const float c = cost_at(a, x, y, d);
    const float n = (float)((2 * a.RN + 1) * (2 * a.RN + 1));
    const float scale = g * n * il_ * ir_;              // g / (n sigma_l sigma_r)
    const float rr = ir_ / il_, rl = il_ / ir_;         // sigma_l/sigma_r, sigma_r/sigma_l
    for (int j = -a.RN; j <= a.RN; ++j) {
        const int yy = clampi(y + j, 0, a.H - 1);
        const uint8_t *lrow = a.left + (size_t)yy * a.pitch;
        const uint8_t *rrow = a.right + (size_t)yy * a.pitch;
        const float *wrow = a.rw + (size_t)yy * a.W;
        const int k = row_shift_floor(a, yy);
        float acc = 0.0f;                               // sum of dr * dr/ds over the row
        for (int q = -a.RN; q <= a.RN; ++q) {
            const int xl = clampi(x + q, 0, a.W - 1), xr = clampi(x - d + q, 0, a.W - 1);
            const float av = (float)lrow[xl] - ml;
            const float bv = wrow[xr] - mr;
            const float dr = scale * (av - c * rr * bv);
            if (grw) atomicAdd(&grw[(size_t)yy * a.W + xr], dr);
            if (gl) atomicAdd(&gl[(size_t)yy * a.W + xl], scale * (bv - c * rl * av));
            const float dds = (float)rrow[clampi(xr - k - 1, 0, a.W - 1)] -
                              (float)rrow[clampi(xr - k, 0, a.W - 1)];
            acc = fmaf(dr, dds, acc);
        }
        s0 += (double)acc;
        s1 += (double)acc * (double)yy;
    }
}

// Per (x, y): G(x, y, d) = sum over window pixels p with dstar[p] = d of
// w(p -> (x, y)) / W_p, gathered into kSlots (d, G) register slots; each
// slot's NCC adjoint runs when the slot is evicted or at the end (the adjoint
// is linear in G, so a d evicted and met again is simply run twice).
constexpr int kSlots = 4;

__global__ void __launch_bounds__(kGT) k_grad_ncc(GradArgs a, const float *__restrict__ wsum,
                                                  float *__restrict__ grw, float *__restrict__ gl,
                                                  double *__restrict__ partial) {
    const int i = blockIdx.x * kGT + threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    if (i < a.W * a.H) {
        const int x = i % a.W, y = i / a.W;
        const float gq = (float)a.left[(size_t)y * a.pitch + x];
        int sd[kSlots];
        float sg[kSlots];
#pragma unroll
        for (int k = 0; k < kSlots; ++k) { sd[k] = -1; sg[k] = 0.0f; }
        int victim = 0;
        for (int dy = -a.R; dy <= a.R; ++dy) {
            const int v = y - dy;                       // window pixel p = (x - dx, y - dy)
            if (v < 0 || v >= a.H) continue;
            for (int dx = -a.R; dx <= a.R; ++dx) {
                const int u = x - dx;
                if (u < 0 || u >= a.W) continue;
                const int d = a.dstar[(size_t)v * a.W + u];
                if (d < 0 || d >= a.D) continue;
                const float w = weight(a, dx, dy, gq - (float)a.left[(size_t)v * a.pitch + u]) /
                                wsum[(size_t)v * a.W + u];
                bool hit = false;
#pragma unroll
                for (int k = 0; k < kSlots; ++k)
                    if (sd[k] == d) { sg[k] += w; hit = true; }
                if (hit) continue;
                int free_k = -1;
#pragma unroll
                for (int k = kSlots - 1; k >= 0; --k)
                    if (sd[k] < 0) free_k = k;
                if (free_k < 0) {                       // evict round-robin
                    free_k = victim;
                    victim = (victim + 1) % kSlots;
                    int ed = 0;
                    float eg = 0.0f;
#pragma unroll
                    for (int k = 0; k < kSlots; ++k)
                        if (k == free_k) { ed = sd[k]; eg = sg[k]; }
                    ncc_adjoint(a, x, y, ed, eg, grw, gl, s0, s1);
                }
#pragma unroll
                for (int k = 0; k < kSlots; ++k)
                    if (k == free_k) { sd[k] = d; sg[k] = w; }
            }
        }
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
            if (sd[k] >= 0) ncc_adjoint(a, x, y, sd[k], sg[k], grw, gl, s0, s1);
    }
    block_sum3(s0, s1, 0.0, partial);
}

// Adjoint of i_r'(x) = (1-w) i_r(x-k) + w i_r(x-k-1), one thread per row.
__global__ void k_grad_warp(GradArgs a, const float *__restrict__ grw, float *__restrict__ gr) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= a.H) return;
    const double s = a.alpha0 + a.alpha1 * (double)y - a.delta;
    double k = floor(s);
    const float w = (float)(s - k);
    k = fmin(fmax(k, -2.0 * a.W - 2.0), 2.0 * a.W + 2.0);
    const int ki = (int)k;
    float *row = gr + (size_t)y * a.W;
    for (int x = 0; x < a.W; ++x) row[x] = 0.0f;
    for (int x = 0; x < a.W; ++x) {
        const float g = grw[(size_t)y * a.W + x];
        row[clampi(x - ki, 0, a.W - 1)] += (1.0f - w) * g;
        row[clampi(x - ki - 1, 0, a.W - 1)] += w * g;
    }
}

// Fixed-order FP64 sum of the block partials: out = {L, dL/dalpha0, dL/dalpha1}.
__global__ void k_grad_reduce(const double *__restrict__ pl, int nl, const double *__restrict__ pa,
                              int na, double *__restrict__ out) {
    __shared__ double s[3][kGT];
    double t0 = 0, t1 = 0, t2 = 0;
    for (int b = threadIdx.x; b < nl; b += kGT) t0 += pl[3 * b];
    for (int b = threadIdx.x; b < na; b += kGT) { t1 += pa[3 * b]; t2 += pa[3 * b + 1]; }
    s[0][threadIdx.x] = t0; s[1][threadIdx.x] = t1; s[2][threadIdx.x] = t2;
    __syncthreads();
    for (int o = kGT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = s[0][0]; out[1] = s[1][0]; out[2] = s[2][0]; }
}

}  // namespace

size_t grad_partial_count(int W, int H) { return (size_t)2 * ((W * H + kGT - 1) / kGT); }

cudaError_t launch_grad(const uint8_t *left, const uint8_t *right, int pitch, int W, int H, int D,
                        int ncc_r, int agg_r, float gamma_d, float gamma_r, double alpha0,
                        double alpha1, double delta, const float *rw, const float *mu_l,
                        const float *inv_l, const float *mu_r, const float *inv_r,
                        const float *cost, const int16_t *dstar, float *wsum, float *grw,
                        float *gl, float *gr, double *partial, double *out3, cudaStream_t st) {
    const float log2e = 1.4426950408889634f;
    GradArgs a{left, right, pitch, W, H, D, ncc_r, agg_r, rw, mu_l, inv_l, mu_r, inv_r, cost, dstar,
               alpha0, alpha1, delta, log2e / (gamma_d * gamma_d), log2e / (gamma_r * gamma_r),
               1.0f / (gamma_r * gamma_r)};
    const int npx = W * H, nb = (npx + kGT - 1) / kGT;
    cudaError_t e;
    if (grw && (e = cudaMemsetAsync(grw, 0, (size_t)npx * sizeof(float), st)) != cudaSuccess)
        return e;
    if (gl && (e = cudaMemsetAsync(gl, 0, (size_t)npx * sizeof(float), st)) != cudaSuccess)
        return e;
    k_grad_pixel<<<nb, kGT, 0, st>>>(a, wsum, gl, partial);
    k_grad_ncc<<<nb, kGT, 0, st>>>(a, wsum, grw, gl, partial + 3 * (size_t)nb);
    if (gr && grw) k_grad_warp<<<(H + 127) / 128, 128, 0, st>>>(a, grw, gr);
    k_grad_reduce<<<1, kGT, 0, st>>>(partial, nb, partial + 3 * (size_t)nb, nb, out3);
    return cudaGetLastError();
}

}  // namespace sr
