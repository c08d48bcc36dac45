// k_fit.cu -- road-plane fitting from a full-disparity map (Sec. II-A).
//
// alpha of Eq. 2 is fitted by least squares with RANSAC, the valid pixels of
// the disparity map serving as the correspondences; the roll angle comes
// from a linear plane d = g0 + g1 u + g2 v fitted to a near-field patch,
// gamma = atan(-g1 / g2).
//   k_fit_models   one thread per hypothesis: the line d = a0 + a1 v through
//                  its two given points (double, no fused operations), then
//                  rounded to float;
//   k_fit_count    inliers of every hypothesis: a pixel is an inlier when
//                  |d - fmaf(a1, v, a0)| <= tau in single precision; each
//                  warp votes with a ballot per hypothesis, counts are exact
//                  integers (order-free);
//   k_fit_ls       FP64 sums n, sum v, sum v^2, sum d, sum v d over the
//                  inliers of the chosen model (block partials);
//   k_roll_sums    FP64 sums of the 3x3 normal equations over the patch;
//   k_sum_partials fixed-order FP64 reduction of block partials.
#include <math.h>

#include "sr_internal.cuh"

namespace sr {
namespace {

constexpr int kFT = 256;          // threads per block
constexpr int kHypChunk = 256;    // hypotheses per shared-memory chunk

__global__ void k_fit_models(const float *__restrict__ disp, int W, long long npx,
                             const int *__restrict__ pairs, int n, float2 *__restrict__ model,
                             int *__restrict__ has_model) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= n) return;
    const int i1 = pairs[2 * h], i2 = pairs[2 * h + 1];
    int ok = i1 >= 0 && i2 >= 0 && i1 < npx && i2 < npx;
    float2 m = make_float2(0.0f, 0.0f);
    if (ok) {
        const float d1 = disp[i1], d2 = disp[i2];
        const int v1 = i1 / W, v2 = i2 / W;
        ok = !isnan(d1) && !isnan(d2) && v1 != v2;
        if (ok) {
            const double a1 = __ddiv_rn(__dsub_rn((double)d2, (double)d1), (double)(v2 - v1));
            const double a0 = __dsub_rn((double)d1, __dmul_rn(a1, (double)v1));
            m = make_float2((float)a0, (float)a1);
        }
    }
    model[h] = m;
    has_model[h] = ok;
}

__device__ __forceinline__ bool inlier(float d, int v, float a0, float a1, float tau) {
    return !isnan(d) && fabsf(d - fmaf(a1, (float)v, a0)) <= tau;
}

__global__ void __launch_bounds__(kFT) k_fit_count(const float *__restrict__ disp, int W,
                                                   long long npx, const float2 *__restrict__ model,
                                                   const int *__restrict__ has_model, int n,
                                                   float tau, int *__restrict__ counts) {
    __shared__ float2 s_m[kHypChunk];
    __shared__ int s_c[kHypChunk];
    const int lane = threadIdx.x & 31;
    for (int h0 = 0; h0 < n; h0 += kHypChunk) {
        const int nh = min(kHypChunk, n - h0);
        __syncthreads();
        for (int k = threadIdx.x; k < nh; k += kFT) {
            s_m[k] = model[h0 + k];
            s_c[k] = 0;
        }
        __syncthreads();
        // grid-stride over warps of 32 consecutive pixels
        for (long long base = ((long long)blockIdx.x * kFT + (threadIdx.x & ~31));
             base < npx; base += (long long)gridDim.x * kFT) {
            const long long i = base + lane;
            const float d = i < npx ? disp[i] : __int_as_float(0x7fc00000);
            const int v = (int)(i / W);
            for (int k = 0; k < nh; ++k) {
                const unsigned b = __ballot_sync(0xffffffffu, inlier(d, v, s_m[k].x, s_m[k].y, tau));
                if (lane == 0 && b) atomicAdd(&s_c[k], __popc(b));
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nh; k += kFT)
            if (has_model[h0 + k] && s_c[k]) atomicAdd(&counts[h0 + k], s_c[k]);
    }
}

// Fixed-order block sum of K doubles per thread into partial[blockIdx][K].
template <int K>
__device__ void block_sums(const double (&x)[K], double *__restrict__ partial) {
    __shared__ double s[K][kFT / 32];
    double y[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        y[k] = x[k];
        for (int o = 16; o > 0; o >>= 1) y[k] += __shfl_down_sync(0xffffffffu, y[k], o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) s[k][warp] = y[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = 0.0;
            for (int w = 0; w < kFT / 32; ++w) t += s[k][w];
            partial[(size_t)blockIdx.x * K + k] = t;
        }
}

__global__ void __launch_bounds__(kFT) k_fit_ls(const float *__restrict__ disp, int W,
                                                long long npx, float a0, float a1, float tau,
                                                double *__restrict__ partial) {
    double x[5] = {0, 0, 0, 0, 0};   // n, sum v, sum v^2, sum d, sum v d
    for (long long i = (long long)blockIdx.x * kFT + threadIdx.x; i < npx;
         i += (long long)gridDim.x * kFT) {
        const float d = disp[i];
        const int v = (int)(i / W);
        if (!inlier(d, v, a0, a1, tau)) continue;
        const double dv = v, dd = d;
        x[0] += 1.0;
        x[1] += dv;
        x[2] += dv * dv;
        x[3] += dd;
        x[4] += dv * dd;
    }
    block_sums<5>(x, partial);
}

__global__ void __launch_bounds__(kFT) k_roll_sums(const float *__restrict__ disp, int W,
                                                   int u_lo, int v_lo, int pw, int ph,
                                                   double *__restrict__ partial) {
    // [1 u v] x [1 u v]^T (6 distinct entries, the first is the count), [1 u v] d
    double x[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const long long np = (long long)pw * ph;
    for (long long i = (long long)blockIdx.x * kFT + threadIdx.x; i < np;
         i += (long long)gridDim.x * kFT) {
        const int u = u_lo + (int)(i % pw), v = v_lo + (int)(i / pw);
        const float df = disp[(size_t)v * W + u];
        if (isnan(df)) continue;
        const double du = u, dv = v, d = df;
        x[0] += 1.0;
        x[1] += du;
        x[2] += dv;
        x[3] += du * du;
        x[4] += du * dv;
        x[5] += dv * dv;
        x[6] += d;
        x[7] += du * d;
        x[8] += dv * d;
    }
    block_sums<9>(x, partial);
}

__global__ void k_sum_partials(const double *__restrict__ partial, int nb, int K,
                               double *__restrict__ out) {
    // one thread per component, blocks summed in index order
    const int k = threadIdx.x;
    if (k >= K) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partial[(size_t)b * K + k];
    out[k] = t;
}

}  // namespace

// Blocks of a grid-stride pass over items: enough for every SM several times
// over, at most one per kFT items.
int fit_blocks(long long items) {
    const long long need = (items + kFT - 1) / kFT;
    return (int)(need < 1 ? 1 : need > 4 * 152 ? 4 * 152 : need);
}

cudaError_t launch_fit_count(const float *disp, int W, int H, const int *pairs, int n, float tau,
                             float2 *model, int *has_model, int *counts, cudaStream_t st) {
    const long long npx = (long long)W * H;
    cudaError_t e = cudaMemsetAsync(counts, 0, n * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_fit_models<<<(n + 127) / 128, 128, 0, st>>>(disp, W, npx, pairs, n, model, has_model);
    k_fit_count<<<fit_blocks(npx), kFT, 0, st>>>(disp, W, npx, model, has_model, n, tau, counts);
    return cudaGetLastError();
}

cudaError_t launch_fit_ls(const float *disp, int W, int H, float a0, float a1, float tau,
                          double *partial, double *out5, cudaStream_t st) {
    const long long npx = (long long)W * H;
    const int nb = fit_blocks(npx);
    k_fit_ls<<<nb, kFT, 0, st>>>(disp, W, npx, a0, a1, tau, partial);
    k_sum_partials<<<1, 32, 0, st>>>(partial, nb, 5, out5);
    return cudaGetLastError();
}

cudaError_t launch_roll_sums(const float *disp, int W, int u_lo, int v_lo, int u_hi, int v_hi,
                             double *partial, double *out9, cudaStream_t st) {
    const int pw = u_hi - u_lo, ph = v_hi - v_lo;
    const int nb = fit_blocks((long long)pw * ph);
    k_roll_sums<<<nb, kFT, 0, st>>>(disp, W, u_lo, v_lo, pw, ph, partial);
    k_sum_partials<<<1, 32, 0, st>>>(partial, nb, 9, out9);
    return cudaGetLastError();
}

}  // namespace sr
