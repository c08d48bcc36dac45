// sr_batch.cu -- sr_match_batch: many stereo pairs of mixed sizes per call.
//
// Schedule A runs each stage as ONE persistent launch over the flat list of
// (pair, tile) work items of the whole batch (kernels *_batch in k_pixel.cu,
// k_ncc.cuh, k_agg.cuh), except the reference NCC volume, which every
// schedule computes per pair with sr_match's exact-sum kernel (k_ncc_sl.cuh)
// so that a pair's costs equal sr_match's bit for bit; the launches are
// captured into a CUDA graph and replayed.  Per call the host writes the pair
// descriptors and the per-stage tile prefixes into pinned staging memory and
// copies them to the device ahead of the graph on the context's stream.
//
// Two schedules, chosen by a small autotuner when enabled:
//   A (variants 0-3): one persistent launch per stage over all pairs' tiles,
//     with knobs grid factor f (the NCC and aggregation launches get
//     f x (SMs x resident CTAs per SM) CTAs) and tile order (the caller's, or
//     largest pair first, so small pairs fill the tail).  NCC and aggregation
//     CTAs take tiles in order from a device counter (reset by a memset node
//     of the graph), so the tiles in flight stay a contiguous band and
//     neighbouring tiles share their halo rows through L2;
//   B (variants 4-5): per pair, its seven stages as non-persistent launches
//     (one CTA per tile, as sr_match), the pairs spread over 4 or 8 forked
//     capture streams, largest first, so that one pair's kernels fill the
//     tails of another's;
//   C (variants 6-7): per pair, the four kernels of sr_match itself (one
//     extended NCC volume read by both aggregations) with the pair's pointers
//     and plane as kernel parameters, on 1 or 4 forked capture streams,
//     largest first.
// A graph holds per-pair parameters (all of them in C, the reference NCC
// launches in A and B), so a call with other pointers or planes re-captures
// it and updates the executable graph in place (cudaGraphExecUpdate; a fresh
// instantiation if that fails).
// The tuner times each candidate on the caller's own batch the first time a
// batch shape is seen and keeps the fastest; with a cache path the choice is
// stored as one JSON object per line, keyed by GPU name, method parameters
// and the multiset of image sizes.  An unreadable cache line is ignored (the
// defaults are used) and reported through sr_last_error.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "sr_ctx.cuh"

namespace {

constexpr int kBatchStages = 3;     // tile lists: 32x8 pixels, 32x8 stats, 32x4 NCC/agg
constexpr int kVariants = 8;        // 0-3: schedule A (bit 0: f = 2; bit 1: largest first)
                                    // 4, 5: schedule B on 4 / 8 streams, largest first
                                    // 6, 7: schedule C on 1 / 4 streams, largest first
constexpr int kMaxSide = 8;         // capture streams of schedules B and C
inline bool sched_b(int v) { return v == 4 || v == 5; }
inline bool sched_c(int v) { return v >= 6; }
inline bool per_pair(int v) { return v >= 4; }
inline int pair_streams(int v) { return v == 4 ? 4 : v == 5 ? 8 : v == 6 ? 1 : 4; }

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

struct SrBatch {
    int cap = 0;                              // pairs the descriptor buffers hold
    sr::PairDesc *d_desc = nullptr, *h_desc = nullptr;
    // [kBatchStages][cap + 1] flat prefixes (schedule A), then [cap][3][2]
    // per-pair {0, tiles} arrays (schedule B)
    int *d_start = nullptr, *h_start = nullptr;
    int *d_next = nullptr;                    // work counters of the persistent NCC / agg launches
    cudaEvent_t staged = nullptr;             // last copy out of the staging buffers
    bool staged_pending = false;
    void *pool = nullptr;
    size_t pool_bytes = 0;
    bool tuning = false;                      // inside the autotuner's loop
    bool shrink_next = false;                 // the tuner chose: fit the pool to it
    cudaStream_t cap_stream = nullptr;        // capture stream (never the legacy one)
    cudaStream_t side[kMaxSide] = {};         // forked capture streams (schedule B)
    cudaEvent_t fork = nullptr, join[kMaxSide] = {};
    cudaGraphExec_t graph = nullptr;
    int graph_n = -1, graph_variant = -1;
    std::vector<int> tiles_pix, tiles_stat, tiles_t4;     // staged order
    std::vector<long long> graph_sizes;                   // size sequence the graph was built for
    std::vector<sr::PairDesc> graph_desc;                 // descriptors a schedule-C graph holds
    std::vector<CUtensorMap> tmaps;                       // sheared view of each pair's vol_l
    bool tune = false;
    std::string cache_path;
    std::map<std::string, int> tuned;
    int variant = 0;
    int forced = -1;                          // sr_set_batch_schedule, -1 = automatic
    float tune_ms[kVariants] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool cache_bad = false;
    int sms = 0;
};

void sr_batch_free(sr_ctx *c) {
    SrBatch *b = c->batch;
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_start) cudaFree(b->d_start);
    if (b->h_desc) cudaFreeHost(b->h_desc);
    if (b->h_start) cudaFreeHost(b->h_start);
    if (b->pool) cudaFree(b->pool);
    if (b->d_next) cudaFree(b->d_next);
    if (b->staged) cudaEventDestroy(b->staged);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int i = 0; i < kMaxSide; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    c->batch = nullptr;
}

namespace {

// Scratch of one pair (the arrays sr_create allocates for one frame).
// vol_l holds the extended reference volume [H][WE][D] (schedule C) or the
// reference volume [H][W][D] (the other schedules, a prefix of it); the
// target volume vol_r is needed by all schedules but C, which reads both
// views from vol_l.
size_t pair_scratch_bytes(const sr_params &p, int W, int H, bool with_vol_r) {
    const size_t npx = (size_t)W * H, WE = (size_t)W + p.max_disp - 1;
    const size_t e = sr::vol_elem_bytes(p.vol_dtype);
    return 2 * a256(npx * 4) + 4 * a256((size_t)H * WE * 4) + a256((size_t)H * WE * p.max_disp * e) +
           (with_vol_r ? a256(npx * p.max_disp * e) : 0) + 2 * a256(npx * 2) + a256((size_t)H * 8);
}

// Scratch slots of a schedule: the per-pair schedules run the pairs of one
// stream in order (pair k on stream k mod S), so the pairs of a stream share
// one slot sized for the largest of them; the persistent schedules run all
// pairs at once, one slot each.  Fills slot_of (per staged pair) and returns
// the pool bytes.
size_t slot_layout(const sr_params &p, int n, const sr_pair_desc *pairs, const int *order,
                   int variant, std::vector<size_t> *slot_off, std::vector<int> *slot_of) {
    const bool pp = per_pair(variant);
    const int S = pp ? pair_streams(variant) : n;
    std::vector<size_t> bytes(S, 0);
    slot_of->resize(n);
    for (int k = 0; k < n; ++k) {
        const int s = pp ? k % S : k;
        (*slot_of)[k] = s;
        const sr_pair_desc &q = pairs[order[k]];
        bytes[s] = std::max(bytes[s], pair_scratch_bytes(p, q.width, q.height, !sched_c(variant)));
    }
    slot_off->assign(S, 0);
    size_t total = 0;
    for (int s = 0; s < S; ++s) {
        (*slot_off)[s] = total;
        total += bytes[s];
    }
    return total;
}

// Order of the staged pairs: caller order, or largest first.
std::vector<int> stage_order(int n, const sr_pair_desc *pairs, int variant) {
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if ((variant & 2) || per_pair(variant))
        std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
            return (long long)pairs[a].width * pairs[a].height >
                   (long long)pairs[b2].width * pairs[b2].height;
        });
    return order;
}

std::string tune_key(const sr_ctx *c, int n, const sr_pair_desc *pairs) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, c->device);
    std::vector<std::pair<int, int>> sizes;
    for (int i = 0; i < n; ++i) sizes.push_back({pairs[i].width, pairs[i].height});
    std::sort(sizes.begin(), sizes.end());
    std::string k = std::string(prop.name) + "|D" + std::to_string(c->p.max_disp) + "|r" +
                    std::to_string(c->p.ncc_radius) + "|R" + std::to_string(c->p.agg_radius) +
                    "|t" + std::to_string((int)c->p.vol_dtype) + "|";
    for (auto &s : sizes) k += std::to_string(s.first) + "x" + std::to_string(s.second) + ",";
    return k;
}

// Cache file: one {"key": "...", "variant": v} per line.
void load_cache(SrBatch *b, sr_ctx *c) {
    if (b->cache_path.empty()) return;
    FILE *f = fopen(b->cache_path.c_str(), "r");
    if (!f) return;
    char line[4096];
    while (fgets(line, sizeof(line), f)) {
        const char *kp = strstr(line, "\"key\": \"");
        const char *vp = strstr(line, "\"variant\": ");
        int v = -1;
        if (!kp || !vp || sscanf(vp + 11, "%d", &v) != 1 || v < 0 || v >= kVariants) {
            b->cache_bad = true;
            continue;
        }
        kp += 8;
        const char *ke = strchr(kp, '"');
        if (!ke) { b->cache_bad = true; continue; }
        b->tuned[std::string(kp, ke - kp)] = v;
    }
    fclose(f);
    if (b->cache_bad)
        snprintf(c->err, sizeof(c->err), "autotune cache %s has unreadable lines; defaults used",
                 b->cache_path.c_str());
}

void append_cache(SrBatch *b, const std::string &key, int v, const float *ms) {
    if (b->cache_path.empty()) return;
    FILE *f = fopen(b->cache_path.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"key\": \"%s\", \"variant\": %d, \"ms\": [", key.c_str(), v);
    for (int i = 0; i < kVariants; ++i) fprintf(f, i ? ", %.4f" : "%.4f", ms[i]);
    fprintf(f, "]}\n");
    fclose(f);
}

cudaError_t ensure_capacity(SrBatch *b, int n) {
    if (n <= b->cap) return cudaSuccess;
    if (b->staged_pending) cudaEventSynchronize(b->staged);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_start) cudaFree(b->d_start);
    if (b->h_desc) cudaFreeHost(b->h_desc);
    if (b->h_start) cudaFreeHost(b->h_start);
    b->d_desc = b->h_desc = nullptr;
    b->d_start = b->h_start = nullptr;
    b->cap = 0;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    const int cap = std::max(n, 8);
    cudaError_t e = cudaMalloc(&b->d_desc, cap * sizeof(sr::PairDesc));
    const size_t nstart = kBatchStages * (cap + 1) + 6 * (size_t)cap;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_start, nstart * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_desc, cap * sizeof(sr::PairDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_start, nstart * sizeof(int));
    if (e == cudaSuccess) b->cap = cap;
    return e;
}

// The reference volume of one pair (W columns) by the exact-sum NCC kernel
// of sr_match, which every schedule uses for it, so that each pair's
// reference costs equal those of sr_match on that pair bit for bit.  Its
// launch holds the pair's pointers and plane, so the graph of any schedule is
// rebuilt when they change (graph_stale).
cudaError_t launch_ref_ncc(sr_ctx *c, const sr::PairDesc &P, cudaStream_t st) {
    const sr_params &p = c->p;
    const int D = p.max_disp;
    return sr::launch_ncc_sl(P.left, P.right, P.pitch, P.W, P.H, D, p.ncc_radius, 0, P.alpha0,
                             P.alpha1, P.delta, P.inv_l, P.inv_r, P.vol_l, p.vol_dtype, P.W,
                             sr::ncc_segment(P.W, P.H, D, p.ncc_radius, p.vol_dtype), st);
}

// The seven stage launches of one pair (schedule B) or of the whole batch
// (schedule A), queued on st.
cudaError_t launch_pair(sr_ctx *c, SrBatch *b, int k, cudaStream_t st) {
    const sr_params &p = c->p;
    const int D = p.max_disp;
    const int *ps = b->d_start + kBatchStages * (b->cap + 1) + 6 * k;
    const sr::PairDesc *d = b->d_desc + k;
    const sr::AggDebug dbg = agg_debug(c);
    const int tp = b->tiles_pix[k], ts = b->tiles_stat[k], t4 = b->tiles_t4[k];
    cudaError_t e;
    if ((e = sr::launch_warp_batch(d, ps, 1, tp, st)) != cudaSuccess) return e;
    if ((e = sr::launch_stats_batch(d, ps + 2, 1, D, p.ncc_radius, ts, st)) != cudaSuccess) return e;
    if ((e = launch_ref_ncc(c, b->h_desc[k], st)) != cudaSuccess) return e;
    if ((e = sr::launch_ncc_batch(true, d, ps + 4, 1, D, p.ncc_radius, p.vol_dtype, t4, nullptr, st)) != cudaSuccess) return e;
    if ((e = sr::launch_agg_batch(false, d, ps + 4, 1, D, p.agg_radius, p.vol_dtype, p.gamma_d,
                                  p.gamma_r, dbg, t4, nullptr, st)) != cudaSuccess) return e;
    if ((e = sr::launch_agg_batch(true, d, ps + 4, 1, D, p.agg_radius, p.vol_dtype, p.gamma_d,
                                  p.gamma_r, dbg, t4, nullptr, st)) != cudaSuccess) return e;
    return sr::launch_lrc_post_batch(d, ps, 1, p.lr_thresh, tp, st);
}

// Schedule C: the kernels of sr_match for pair k, parameters from the host
// copy of its descriptor.
cudaError_t launch_pair_direct(sr_ctx *c, SrBatch *b, int k, cudaStream_t st) {
    const sr_params &p = c->p;
    const int D = p.max_disp;
    const sr::PairDesc &P = b->h_desc[k];
    const sr::AggDebug dbg = agg_debug(c);
    cudaError_t e;
    if ((e = sr::launch_prep(P.left, P.right, P.pitch, P.W, P.H, D, p.ncc_radius, P.alpha0,
                             P.alpha1, P.delta, 0, P.rw, P.mu_l, P.inv_l, P.mu_r, P.inv_r,
                             P.rowsh, st)) != cudaSuccess) return e;
    // one extended reference volume for both views, as in sr_match
    const int WE = P.W + D - 1;
    if ((e = sr::launch_ncc_sl(P.left, P.right, P.pitch, P.W, P.H, D, p.ncc_radius, 0, P.alpha0,
                               P.alpha1, P.delta, P.inv_l, P.inv_r, P.vol_l, p.vol_dtype, WE,
                               sr::ncc_segment(P.W, P.H, D, p.ncc_radius, p.vol_dtype), st)) != cudaSuccess) return e;
    // target view first; the reference view runs the L-R check and the
    // post-processing in its epilogue, as in sr_match
    if ((e = sr::launch_agg_shear(&b->tmaps[k], p.vol_dtype, P.rw, P.W, P.H, D, p.agg_radius,
                                  p.gamma_d, p.gamma_r, P.lbl_r, nullptr, dbg, st)) != cudaSuccess) return e;
    sr::AggWin post;
    post.post.lbl_r = P.lbl_r;
    post.post.disp = P.disp;
    post.post.wta = P.wta;
    post.post.rowsh = P.rowsh;
    post.post.lr_thresh = p.lr_thresh;
    return sr::launch_agg(P.vol_l, p.vol_dtype, P.left, P.pitch, nullptr, P.W, P.H, D,
                          p.agg_radius, p.gamma_d, p.gamma_r, P.lbl_l, P.dsub, nullptr, dbg, st,
                          post, WE);
}

cudaError_t launch_stages(sr_ctx *c, SrBatch *b, int n, int variant, cudaStream_t st) {
    const sr_params &p = c->p;
    const int D = p.max_disp;
    cudaError_t e;
    if (per_pair(variant)) {
        // fork the pairs over S streams, join back into st
        const int S = pair_streams(variant);
        if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
        for (int i = 0; i < S; ++i)
            if ((e = cudaStreamWaitEvent(b->side[i], b->fork, 0)) != cudaSuccess) return e;
        for (int k = 0; k < n; ++k) {
            e = sched_c(variant) ? launch_pair_direct(c, b, k, b->side[k % S])
                                 : launch_pair(c, b, k, b->side[k % S]);
            if (e != cudaSuccess) return e;
        }
        for (int i = 0; i < S; ++i) {
            if ((e = cudaEventRecord(b->join[i], b->side[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, b->join[i], 0)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int f = (variant & 1) ? 2 : 1;
    const int g_pix = b->sms * 8;
    const int g_ncc = b->sms * std::max(1, sr::ncc_batch_occupancy(D, p.ncc_radius, p.vol_dtype)) * f;
    const int g_agg = b->sms * std::max(1, sr::agg_batch_occupancy(D, p.agg_radius, p.vol_dtype)) * f;
    const int *s_pix = b->d_start, *s_stat = b->d_start + (b->cap + 1),
              *s_t4 = b->d_start + 2 * (b->cap + 1);
    const sr::AggDebug dbg = agg_debug(c);
    int *nx = b->d_next;   // [4]: NCC reference, NCC target, agg reference, agg target
    if ((e = cudaMemsetAsync(nx, 0, 4 * sizeof(int), st)) != cudaSuccess) return e;
    if ((e = sr::launch_warp_batch(b->d_desc, s_pix, n, g_pix, st)) != cudaSuccess) return e;
    if ((e = sr::launch_stats_batch(b->d_desc, s_stat, n, D, p.ncc_radius, g_pix, st)) != cudaSuccess) return e;
    for (int k = 0; k < n; ++k)
        if ((e = launch_ref_ncc(c, b->h_desc[k], st)) != cudaSuccess) return e;
    if ((e = sr::launch_ncc_batch(true, b->d_desc, s_t4, n, D, p.ncc_radius, p.vol_dtype, g_ncc, nx + 1, st)) != cudaSuccess) return e;
    if ((e = sr::launch_agg_batch(false, b->d_desc, s_t4, n, D, p.agg_radius, p.vol_dtype, p.gamma_d,
                                  p.gamma_r, dbg, g_agg, nx + 2, st)) != cudaSuccess) return e;
    if ((e = sr::launch_agg_batch(true, b->d_desc, s_t4, n, D, p.agg_radius, p.vol_dtype, p.gamma_d,
                                  p.gamma_r, dbg, g_agg, nx + 3, st)) != cudaSuccess) return e;
    return sr::launch_lrc_post_batch(b->d_desc, s_pix, n, p.lr_thresh, g_pix, st);
}

// Fill the staging buffers for one variant's pair order and queue the copies.
cudaError_t stage_batch(sr_ctx *c, SrBatch *b, int n, const sr_pair_desc *pairs, int variant,
                        cudaStream_t st) {
    const sr_params &p = c->p;
    const int D = p.max_disp;
    const std::vector<int> order = stage_order(n, pairs, variant);
    if (b->staged_pending) {
        cudaError_t e = cudaEventSynchronize(b->staged);   // staging buffers free again
        if (e != cudaSuccess) return e;
    }
    std::vector<size_t> slot_off;
    std::vector<int> slot_of;
    const size_t need = slot_layout(p, n, pairs, order.data(), variant, &slot_off, &slot_of);
    // grow the pool; shrink it to the schedule's need right after the
    // tuner's choice, and otherwise when it holds more than twice the need
    const bool shrink = !b->tuning && (b->shrink_next ? need < b->pool_bytes : need < b->pool_bytes / 2);
    if (!b->tuning) b->shrink_next = false;
    if (need > b->pool_bytes || shrink) {
        cudaError_t e = cudaStreamSynchronize(st);   // no launch still reads the pool
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) return e;
        if (b->pool) cudaFree(b->pool);
        b->pool = nullptr;
        b->pool_bytes = 0;
        if ((e = cudaMalloc(&b->pool, need)) != cudaSuccess) return e;
        b->pool_bytes = need;
    }
    int *sp = b->h_start, *ss = b->h_start + (b->cap + 1), *s4 = b->h_start + 2 * (b->cap + 1);
    int *per = b->h_start + kBatchStages * (b->cap + 1);
    sp[0] = ss[0] = s4[0] = 0;
    b->tiles_pix.resize(n);
    b->tiles_stat.resize(n);
    b->tiles_t4.resize(n);
    b->tmaps.resize(n);
    for (int k = 0; k < n; ++k) {
        const sr_pair_desc &in = pairs[order[k]];
        const int W = in.width, H = in.height;
        const size_t npx = (size_t)W * H, WE = (size_t)W + D - 1;
        sr::PairDesc &o = b->h_desc[k];
        o.W = W; o.H = H; o.pitch = in.pitch_bytes;
        o.left = in.d_left; o.right = in.d_right;
        o.alpha0 = in.alpha0; o.alpha1 = in.alpha1; o.delta = in.delta;
        o.disp = in.d_disp; o.wta = in.d_wta_or_null;
        unsigned char *q = static_cast<unsigned char *>(b->pool) + slot_off[slot_of[k]];
        auto take = [&q](size_t bytes) { unsigned char *r = q; q += a256(bytes); return r; };
        o.rw = reinterpret_cast<float *>(take(npx * 4));
        o.dsub = reinterpret_cast<float *>(take(npx * 4));
        o.mu_l = reinterpret_cast<float *>(take((size_t)H * WE * 4));
        o.inv_l = reinterpret_cast<float *>(take((size_t)H * WE * 4));
        o.mu_r = reinterpret_cast<float *>(take((size_t)H * WE * 4));
        o.inv_r = reinterpret_cast<float *>(take((size_t)H * WE * 4));
        o.vol_l = take((size_t)H * WE * D * sr::vol_elem_bytes(p.vol_dtype));
        o.vol_r = sched_c(variant) ? nullptr : take(npx * D * sr::vol_elem_bytes(p.vol_dtype));
        o.lbl_l = reinterpret_cast<int16_t *>(take(npx * 2));
        o.lbl_r = reinterpret_cast<int16_t *>(take(npx * 2));
        o.rowsh = reinterpret_cast<float2 *>(take((size_t)H * 8));
        if (!sr::encode_shear_map(&b->tmaps[k], o.vol_l, p.vol_dtype, W, H, D, p.agg_radius))
            return cudaErrorNotSupported;
        b->tiles_pix[k] = sr::ceil_div(W, sr::kPixTX) * sr::ceil_div(H, sr::kPixTY);
        b->tiles_stat[k] = sr::ceil_div(W + D - 1, sr::kPixTX) * sr::ceil_div(H, sr::kPixTY);
        b->tiles_t4[k] = sr::ceil_div(W, 32) * sr::ceil_div(H, 4);
        sp[k + 1] = sp[k] + b->tiles_pix[k];
        ss[k + 1] = ss[k] + b->tiles_stat[k];
        s4[k + 1] = s4[k] + b->tiles_t4[k];
        int *q6 = per + 6 * k;
        q6[0] = 0; q6[1] = b->tiles_pix[k];
        q6[2] = 0; q6[3] = b->tiles_stat[k];
        q6[4] = 0; q6[5] = b->tiles_t4[k];
    }
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc, n * sizeof(sr::PairDesc),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_start, b->h_start,
                            (kBatchStages * (b->cap + 1) + 6 * (size_t)b->cap) * sizeof(int),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->staged, st);
    b->staged_pending = (e == cudaSuccess);
    return e;
}

// Tile counts in staged order: what a schedule-B graph's grid sizes depend on.
std::vector<long long> size_signature(const SrBatch *b, int n) {
    std::vector<long long> v;
    for (int k = 0; k < n; ++k)
        v.push_back(((long long)b->tiles_pix[k] << 40) ^ ((long long)b->tiles_stat[k] << 20) ^
                    b->tiles_t4[k]);
    return v;
}

cudaError_t capture_graph(sr_ctx *c, SrBatch *b, int n, int variant) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = launch_stages(c, b, n, variant, b->cap_stream);
    e = cudaStreamEndCapture(b->cap_stream, &g);
    if (el != cudaSuccess) { if (g) cudaGraphDestroy(g); return el; }
    if (e != cudaSuccess) return e;
    bool updated = false;
    if (b->graph && b->graph_n == n && b->graph_variant == variant) {
        // same kernels in the same order, other parameters: update in place
        cudaGraphExecUpdateResultInfo info{};
        updated = cudaGraphExecUpdate(b->graph, g, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();
    }
    if (!updated) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        e = cudaGraphInstantiate(&b->graph, g, 0);
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return e; }
    b->graph_n = n;
    b->graph_variant = variant;
    b->graph_sizes = size_signature(b, n);
    b->graph_desc.assign(b->h_desc, b->h_desc + n);
    return cudaSuccess;
}

// Whether the executable graph must be (re)built for this call's staged batch.
bool graph_stale(const SrBatch *b, int n, int variant) {
    if (!b->graph || b->graph_n != n || b->graph_variant != variant) return true;
    if (sched_b(variant) && b->graph_sizes != size_signature(b, n)) return true;
    // every schedule's graph holds per-pair launches (the reference NCC
    // volume at least) with the pairs' pointers and planes
    return b->graph_desc.size() != (size_t)n ||
           memcmp(b->graph_desc.data(), b->h_desc, n * sizeof(sr::PairDesc)) != 0;
}

}  // namespace

extern "C" {

sr_status sr_set_autotune(sr_ctx *c, int enable, const char *cache_path) {
    if (!c) return SR_ERR_INVALID_ARG;
    if (!c->batch) {
        c->batch = new (std::nothrow) SrBatch();
        if (!c->batch) return SR_ERR_OOM;
    }
    SrBatch *b = c->batch;
    b->tune = enable != 0;
    // no path given: the SR_TUNE_CACHE environment variable, if set
    const char *env = getenv("SR_TUNE_CACHE");
    b->cache_path = cache_path ? cache_path : (env ? env : "");
    b->tuned.clear();
    b->cache_bad = false;
    load_cache(b, c);
    return SR_OK;
}

sr_status sr_match_batch(sr_ctx *c, int n, const sr_pair_desc *pairs) {
    if (!c || n < 1 || !pairs) return SR_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const sr_pair_desc &q = pairs[i];
        if (q.width < 1 || q.height < 1 || q.width > 16384 || q.height > 16384 ||
            q.pitch_bytes < q.width || !q.d_left || !q.d_right || !q.d_disp ||
            !isfinite(q.alpha0) || !isfinite(q.alpha1) || !isfinite(q.delta))
            return SR_ERR_INVALID_ARG;
    }
    if (!c->batch) {
        c->batch = new (std::nothrow) SrBatch();
        if (!c->batch) return SR_ERR_OOM;
    }
    SrBatch *b = c->batch;
    if (!b->staged) SR_TRY(c, cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming), "event");
    if (!b->cap_stream) {
        SR_TRY(c, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
        SR_TRY(c, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
        for (int i = 0; i < kMaxSide; ++i) {
            SR_TRY(c, cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking), "stream");
            SR_TRY(c, cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming), "event");
        }
    }
    if (!b->sms) SR_TRY(c, cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
    if (!b->d_next) SR_TRY(c, cudaMalloc(&b->d_next, 4 * sizeof(int)), "cudaMalloc(counters)");
    SR_TRY(c, ensure_capacity(b, n), "batch descriptors");
    // (the scratch pool is sized by stage_batch for the schedule it stages)

    b->tuning = false;
    int variant = 0;
    if (b->forced >= 0) {
        variant = b->forced;
    } else if (b->tune) {
        const std::string key = tune_key(c, n, pairs);
        auto it = b->tuned.find(key);
        if (it != b->tuned.end()) {
            variant = it->second;
        } else {
            // time every candidate on this batch (one warm-up, best of two)
            cudaEvent_t e0, e1;
            SR_TRY(c, cudaEventCreate(&e0), "event");
            SR_TRY(c, cudaEventCreate(&e1), "event");
            float best = 1e30f;
            b->tuning = true;   // the pool keeps the largest layout until the choice
            for (int v = 0; v < kVariants; ++v) {
                // a schedule whose scratch would not fit the free memory
                // (keeping 1 GiB) is not timed: tune_ms -1
                std::vector<size_t> so;
                std::vector<int> sl;
                const std::vector<int> ord = stage_order(n, pairs, v);
                const size_t need = slot_layout(c->p, n, pairs, ord.data(), v, &so, &sl);
                size_t free_b = 0, total_b = 0;
                cudaMemGetInfo(&free_b, &total_b);
                if (need > b->pool_bytes && need - b->pool_bytes + (size_t(1) << 30) > free_b) {
                    b->tune_ms[v] = -1.0f;
                    continue;
                }
                float t_best = 1e30f;
                for (int rep = 0; rep < 3; ++rep) {
                    SR_TRY(c, stage_batch(c, b, n, pairs, v, c->st), "stage");
                    SR_TRY(c, cudaEventRecord(e0, c->st), "event");
                    SR_TRY(c, launch_stages(c, b, n, v, c->st), "batch launch");
                    SR_TRY(c, cudaEventRecord(e1, c->st), "event");
                    SR_TRY(c, cudaEventSynchronize(e1), "event");
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) t_best = std::min(t_best, ms);
                }
                b->tune_ms[v] = t_best;
                if (t_best < best) { best = t_best; variant = v; }
            }
            b->tuning = false;
            b->shrink_next = true;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            b->tuned[key] = variant;
            SR_LOG(2, "batch autotuner: variant %d for %s", variant, key.c_str());
            append_cache(b, key, variant, b->tune_ms);
        }
    }
    SR_TRY(c, stage_batch(c, b, n, pairs, variant, c->st), "stage");
    if (graph_stale(b, n, variant)) SR_TRY(c, capture_graph(c, b, n, variant), "graph capture");
    SR_TRY(c, cudaGraphLaunch(b->graph, c->st), "cudaGraphLaunch");
    b->variant = variant;
    return SR_OK;
}

sr_status sr_set_batch_schedule(sr_ctx *c, int variant) {
    if (!c || variant < -1 || variant >= kVariants) return SR_ERR_INVALID_ARG;
    if (!c->batch) {
        c->batch = new (std::nothrow) SrBatch();
        if (!c->batch) return SR_ERR_OOM;
    }
    c->batch->forced = variant;
    return SR_OK;
}

sr_status sr_batch_info(sr_ctx *c, char *buf, size_t size) {
    if (!c || !buf || size == 0) return SR_ERR_INVALID_ARG;
    if (!c->batch || c->batch->graph_n < 0) return SR_ERR_STATE;
    const SrBatch *b = c->batch;
    const int D = c->p.max_disp;
    const char *sched = sched_c(b->variant)   ? "per-pair-direct"
                        : sched_b(b->variant) ? "per-pair-streams"
                                              : "persistent";
    char ms[160];
    int o = 0;
    for (int i = 0; i < kVariants; ++i)
        o += snprintf(ms + o, sizeof(ms) - o, i ? ", %.4f" : "%.4f", b->tune_ms[i]);
    snprintf(buf, size,
             "{\"pairs\": %d, \"variant\": %d, \"schedule\": \"%s\", \"grid_factor\": %d, "
             "\"largest_first\": %d, \"streams\": %d, \"kernels\": %d, "
             "\"ncc_ctas_per_sm\": %d, \"agg_ctas_per_sm\": %d, \"sms\": %d, "
             "\"tune_ms\": [%s], \"scratch_bytes\": %zu}",
             b->graph_n, b->variant, sched, per_pair(b->variant) ? 1 : ((b->variant & 1) ? 2 : 1),
             per_pair(b->variant) ? 1 : (b->variant >> 1) & 1,
             per_pair(b->variant) ? pair_streams(b->variant) : 1,
             sched_c(b->variant) ? 4 * b->graph_n : sched_b(b->variant) ? 7 * b->graph_n : 7,
             sr::ncc_batch_occupancy(D, c->p.ncc_radius, c->p.vol_dtype),
             sr::agg_batch_occupancy(D, c->p.agg_radius, c->p.vol_dtype), b->sms, ms,
             b->pool_bytes);
    return SR_OK;
}

}  // extern "C"
