// Host side of the C ABI declared in include/splatloam.h: the context (workspace owned and
// sized at creation), view registration (FP64 pose inversion, per-tile frame tables), and the
// stream-ordered call sequences.  No call after splat_ctx_create allocates or synchronises,
// except the ones the header marks as synchronous.

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <vector>

#include "splat_internal.cuh"

using splat::PairRec;
using splat::PixFrame;
using splat::TileInfo;
using splat::SinCos2;
using splat::ViewDesc;

namespace {
thread_local char g_cuda_err[256] = "";
}  // namespace

namespace splat {
int cuda_fail(cudaError_t e, const char *what)
{
    std::snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", what, cudaGetErrorString(e));
    return SPLAT_ERR_CUDA;
}
}  // namespace splat

namespace {
using splat::cuda_fail;

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count);
}

bool supported_tile(int th, int tw)
{
    return (th == 16 && tw == 16) || (th == 8 && tw == 32) || (th == 32 && tw == 8) ||
           (th == 4 && tw == 64);
}

int bits_for(int64_t n)   // bits to hold values 0 .. n-1, rounded up to whole bytes
{
    int b = 0;
    while ((int64_t{1} << b) < n) ++b;
    return ((b + 7) / 8) * 8;
}

void split(double x, float &hi, float &lo)
{
    hi = static_cast<float>(x);
    lo = static_cast<float>(x - static_cast<double>(hi));
}

}  // namespace

struct splat_ctx {
    splat_render_config cfg{};
    splat_capacity cap{};
    int device = 0;
    int sms = 0;
    int grid_fwd = 0, grid_bwd = 0;
    int64_t max_pairs_views = 0;   // max_gaussians * max_views
    int64_t frame_cap = 0;

    // registered views
    int n_views = 0;
    std::vector<ViewDesc> views;
    int64_t n_pixels = 0, n_tiles = 0;
    ViewDesc *d_views = nullptr;
    SinCos2 *d_frames = nullptr;
    int32_t *d_tile_view = nullptr;
    PixFrame *d_pixframes = nullptr;   // grown by splat_set_views
    int64_t pixframe_cap = 0;
    TileInfo *d_tileinfo = nullptr;
    uint32_t *d_tile_order = nullptr;

    // workspace
    PairRec *d_recs = nullptr;
    uint32_t *d_dkeys = nullptr, *d_dvals = nullptr, *d_dkeys2 = nullptr, *d_dvals2 = nullptr;
    uint64_t *d_trect = nullptr, *d_srect = nullptr;   // pair tile rectangles, and in range order
    uint64_t *d_prect = nullptr;   // pair pixel rectangles with the normal-flip bit
    uint32_t *d_tkeys = nullptr, *d_tvals = nullptr, *d_tkeys2 = nullptr, *d_tvals2 = nullptr;
    uint32_t *d_block_sums = nullptr, *d_hist = nullptr;
    uint2 *d_ranges = nullptr;
    float *d_tfinal = nullptr;
    int32_t *d_nlast = nullptr;
    float4 *d_wgrad = nullptr;
    float4 *d_prim = nullptr;      // per primitive: the staged axes, normal and opacity
    float *d_pose = nullptr;        // per view (dL/drho, dL/domega) of the last backward
    uint2 *d_rec = nullptr;         // contributor records: chunks of 32 (forward -> backward)
    uint32_t *d_rec_prev = nullptr, *d_rec_head = nullptr, *d_rec_fill = nullptr;
    uint32_t rec_cap = 0;           // chunks in the record pool
    float *d_img = nullptr;     // refine: depth, normal(3), alpha  (5 x max_pixels)
    float *d_gimg = nullptr;    // refine: their gradients
    uint32_t *d_counters = nullptr;   // [0] pairs M, [1] status, [2] queue f, [3] queue b,
                                      // [4] (view, primitive) pairs that touch a tile,
                                      // [5] record chunks taken, [6] map-growth draws,
                                      // [7] sampling step
    unsigned long long *d_grow_sums = nullptr;  // map growth: block sums, Q, offset
    unsigned long long *d_evals = nullptr;      // [0] forward, [1] backward

    // profiling events: [0,1] forward compositing, [2,3] backward compositing, then one event
    // after each stage of the last profiled render / refinement step (stage_ev[k] ends stage k,
    // stage_ev[0] is recorded before the projection): projection, range sort, emission, tile
    // sort, ranges and work order, loss, fused Adam
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    static constexpr int kStageEvents = 8;
    cudaEvent_t stage_ev[kStageEvents] = {};
    bool stage_rec[kStageEvents] = {};
    bool profiling = false;
    bool rec_fwd = false, rec_bwd = false;
    int64_t launches = 0;

    // state of the last render
    bool rendered = false;
    bool have_pose = false;         // a backward with pose terms ran since the views were set
    int samp_draws = 0;             // keyframe sampling: draws per step (0 = every view)
    uint64_t samp_seed = 0;
    uint32_t *d_samp_thr = nullptr;   // integer thresholds of the sampling law
    uint8_t *d_active = nullptr;      // per view: sampled for the current step
    bool want_pose = false;         // backward calls also accumulate the pose gradient
    int64_t last_n = 0;
    uint32_t *sorted_keys = nullptr, *sorted_vals = nullptr;
    uint32_t *entry_rect = nullptr;   // per list entry: rectangle inside its tile (K4)
    uint8_t *entry_blocks = nullptr;  // per list entry: 4 x 8 blocks it meets (K4)
};

namespace {

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

int check_gaussians(const splat_ctx *ctx, const splat_gaussians *g)
{
    if (!g || g->n < 0 || g->n > ctx->cap.max_gaussians) return SPLAT_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->pos_logit || !g->quat_wxyz || !g->log_scale)) return SPLAT_ERR_INVALID_ARG;
    auto aligned = [](const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; };
    if (g->n > 0 && (!aligned(g->pos_logit, 16) || !aligned(g->quat_wxyz, 16) ||
                     !aligned(g->log_scale, 8)))
        return SPLAT_ERR_INVALID_ARG;
    return SPLAT_OK;
}

splat::RenderArgs render_args(splat_ctx *ctx, const splat_gaussians *g)
{
    splat::RenderArgs a{};
    a.pos_logit = reinterpret_cast<const float4 *>(g->pos_logit);
    a.prim = ctx->d_prim;
    a.n = g->n;
    a.tiles = ctx->d_tileinfo;
    a.pixframes = ctx->d_pixframes;
    a.ranges = ctx->d_ranges;
    a.tile_order = ctx->d_tile_order;
    a.sorted_vals = ctx->sorted_vals;
    a.entry_rect = ctx->entry_rect;
    a.entry_blocks = ctx->entry_blocks;
    a.rec = ctx->d_rec;
    a.rec_prev = ctx->d_rec_prev;
    a.rec_alloc = ctx->d_counters + 5;
    a.rec_cap = ctx->rec_cap;
    a.rec_head = ctx->d_rec_head;
    a.rec_fill = ctx->d_rec_fill;
    a.status = ctx->d_counters + 1;
    a.n_tiles = ctx->n_tiles;
    a.n_items = ctx->n_tiles * (splat::kBlock / 32);
    a.alpha_min = ctx->cfg.alpha_min;
    a.alpha_max = ctx->cfg.alpha_max;
    a.t_min = ctx->cfg.t_min;
    a.sigma = ctx->cfg.sigma_cut;
    a.n_pixels = ctx->n_pixels;
    a.t_final = ctx->d_tfinal;
    a.n_last = ctx->d_nlast;
    a.wgrad = ctx->d_wgrad;
    return a;
}

// forward pipeline: projection -> range sort -> emission -> tile sort -> ranges -> composite
int render_core(splat_ctx *ctx, const splat_gaussians *g, float *depth, float *normal,
                float *alpha, cudaStream_t st)
{
    const int64_t n = g->n;
    const int64_t npv = n * ctx->n_views;
    const int th = ctx->cfg.tile_h, tw = ctx->cfg.tile_w;
    uint32_t *cnt = ctx->d_counters;
    CK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st));           // pair count
    CK(cudaMemsetAsync(cnt + 4, 0, 2 * sizeof(uint32_t), st));   // touching pairs, chunks
    CK(cudaMemsetAsync(cnt + 2, 0, sizeof(uint32_t), st));       // forward queue
    CK(cudaMemsetAsync(ctx->d_evals, 0, sizeof(unsigned long long), st));
    const uint8_t *active = nullptr;
    if (ctx->samp_draws > 0) {
        CK(splat::launch_sample_views(ctx->n_views, ctx->samp_draws, ctx->d_samp_thr,
                                      static_cast<uint32_t>(ctx->samp_seed),
                                      static_cast<uint32_t>(ctx->samp_seed >> 32), cnt + 7,
                                      ctx->d_active, st));
        active = ctx->d_active;
    }
    const bool prof = ctx->profiling && !capturing(st);
    auto stage_mark = [&](int k) -> cudaError_t {
        if (!prof) return cudaSuccess;
        ctx->stage_rec[k] = true;
        return cudaEventRecord(ctx->stage_ev[k], st);
    };
    if (prof)
        for (int k = 0; k < splat_ctx::kStageEvents; ++k) ctx->stage_rec[k] = false;
    CK(stage_mark(0));
    CK(splat::launch_project(reinterpret_cast<const float4 *>(g->pos_logit),
                             reinterpret_cast<const float4 *>(g->quat_wxyz),
                             reinterpret_cast<const float2 *>(g->log_scale), n, ctx->d_views,
                             ctx->n_views, ctx->cfg.sigma_cut, ctx->cfg.alpha_min, th, tw,
                             ctx->cfg.flip_normals,
                             ctx->d_recs, ctx->d_dkeys, ctx->d_dvals, ctx->d_trect,
                             ctx->d_prect, ctx->d_prim, cnt + 1,
                             cnt + 4, st,
                             active));
    CK(stage_mark(1));
    uint32_t *dk, *dv;
    // the range sort drops the pairs that touch no tile (key 0xFFFFFFFF) in its first pass
    // (its last pass also lays the pairs' tile rectangles out in range order for the emission)
    CK(splat::radix_sort_pairs(ctx->d_dkeys, ctx->d_dvals, ctx->d_dkeys2, ctx->d_dvals2, nullptr,
                               npv, 32, ctx->d_hist, &dk, &dv, st, cnt + 4, ctx->d_trect,
                               ctx->d_srect));
    CK(stage_mark(2));
    CK(splat::launch_emit(dv, ctx->d_srect, npv, cnt + 4, ctx->d_views, n, ctx->d_block_sums,
                          ctx->d_tkeys, ctx->d_tvals, ctx->cap.max_pairs, cnt, cnt + 1, st));
    CK(stage_mark(3));
    uint32_t *tk, *tv;
    CK(splat::radix_sort_pairs(ctx->d_tkeys, ctx->d_tvals, ctx->d_tkeys2, ctx->d_tvals2, cnt,
                               ctx->cap.max_pairs, bits_for(ctx->n_tiles), ctx->d_hist, &tk, &tv,
                               st));
    CK(stage_mark(4));
    // the tile sort's other buffers are free: they take the entries' tile rectangles and the
    // blocks each meets
    uint32_t *rects = tv == ctx->d_tvals ? ctx->d_tvals2 : ctx->d_tvals;
    uint8_t *blocks = reinterpret_cast<uint8_t *>(tk == ctx->d_tkeys ? ctx->d_tkeys2 : ctx->d_tkeys);
    CK(splat::launch_ranges(tk, tv, ctx->d_prect, ctx->d_tileinfo, th, tw, cnt,
                            ctx->cap.max_pairs, ctx->d_ranges, ctx->n_tiles, rects, blocks, st));
    CK(splat::launch_order_tiles(ctx->d_ranges, ctx->n_tiles, ctx->d_tile_order, st));
    CK(stage_mark(5));
    ctx->sorted_keys = tk;
    ctx->sorted_vals = tv;
    ctx->entry_rect = rects;
    ctx->entry_blocks = blocks;
    splat::RenderArgs a = render_args(ctx, g);
    a.depth = depth;
    a.normal = normal;
    a.alpha = alpha;
    a.queue = cnt + 2;
    a.evals = ctx->d_evals;
    if (prof) CK(cudaEventRecord(ctx->ev[0], st));
    CK(splat::launch_render_fwd(a, th, tw, ctx->grid_fwd, st));
    if (prof) {
        CK(cudaEventRecord(ctx->ev[1], st));
        ctx->rec_fwd = true;
    }
    // project 1, range sort 4 x 3, emission 3, tile sort 3 per byte, ranges 1, order 1,
    // composite 1
    ctx->launches += 1 + 12 + 3 + 3 * (bits_for(ctx->n_tiles) / 8) + 1 + 1 + 1;
    ctx->rendered = true;
    ctx->last_n = n;
    return SPLAT_OK;
}

// backward into the per-primitive world-frame accumulators
int backward_core(splat_ctx *ctx, const splat_gaussians *g, const float *gD, const float *gN,
                  const float *gO, cudaStream_t st)
{
    uint32_t *cnt = ctx->d_counters;
    CK(cudaMemsetAsync(ctx->d_wgrad, 0, sizeof(float4) * 4 * static_cast<size_t>(g->n), st));
    if (ctx->want_pose)
        CK(cudaMemsetAsync(ctx->d_pose, 0, sizeof(float) * 6 * static_cast<size_t>(ctx->n_views),
                           st));
    CK(cudaMemsetAsync(cnt + 3, 0, sizeof(uint32_t), st));
    CK(cudaMemsetAsync(ctx->d_evals + 1, 0, sizeof(unsigned long long), st));
    splat::RenderArgs a = render_args(ctx, g);
    a.g_depth = gD;
    a.g_normal = gN;
    a.g_alpha = gO;
    a.queue = cnt + 3;
    a.evals = ctx->d_evals + 1;
    a.pose_grad = ctx->want_pose ? ctx->d_pose : nullptr;
    const bool prof = ctx->profiling && !capturing(st);
    if (prof) CK(cudaEventRecord(ctx->ev[2], st));
    CK(splat::launch_render_bwd(a, ctx->cfg.tile_h, ctx->cfg.tile_w, ctx->grid_bwd, st));
    if (prof) {
        CK(cudaEventRecord(ctx->ev[3], st));
        ctx->rec_bwd = true;
    }
    ctx->launches += 1;
    ctx->have_pose = ctx->want_pose;
    return SPLAT_OK;
}

void free_ctx(splat_ctx *c)
{
    void *ptrs[] = {c->d_views, c->d_frames, c->d_tile_view, c->d_recs, c->d_dkeys, c->d_dvals,
                    c->d_dkeys2, c->d_dvals2, c->d_trect, c->d_srect, c->d_prect, c->d_tkeys, c->d_tvals, c->d_tkeys2, c->d_tvals2,
                    c->d_block_sums, c->d_hist, c->d_ranges, c->d_tfinal, c->d_nlast, c->d_wgrad, c->d_prim,
                    c->d_pose, c->d_rec, c->d_rec_prev, c->d_rec_head, c->d_rec_fill,
                    c->d_samp_thr, c->d_active, c->d_grow_sums,
                    c->d_img, c->d_gimg, c->d_counters, c->d_evals, c->d_pixframes,
                    c->d_tileinfo, c->d_tile_order};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->stage_ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

}  // namespace

extern "C" {

SPLAT_API int splat_version(void) { return 100; }

SPLAT_API const char *splat_error_string(int code)
{
    switch (code) {
    case SPLAT_OK: return "ok";
    case SPLAT_ERR_INVALID_ARG: return "invalid argument";
    case SPLAT_ERR_CUDA: return "CUDA error";
    case SPLAT_ERR_CAPACITY: return "pair capacity exceeded";
    case SPLAT_ERR_TIMEOUT: return "device wait timed out";
    case SPLAT_ERR_NONFINITE: return "non-finite primitive parameter";
    case SPLAT_ERR_STATE: return "call order violated";
    case SPLAT_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown error";
    }
}

SPLAT_API const char *splat_last_cuda_error(void) { return g_cuda_err; }

SPLAT_API void splat_default_config(splat_render_config *cfg)
{
    if (!cfg) return;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->t_min = 1e-4f;
    cfg->sigma_cut = 3.0f;
    cfg->tile_h = 16;
    cfg->tile_w = 16;
    cfg->work_cap = 0;
    cfg->flip_normals = 1;
}

SPLAT_API int splat_ctx_create(const splat_render_config *cfg, const splat_capacity *cap,
                               splat_ctx **out)
{
    if (!cfg || !cap || !out) return SPLAT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!supported_tile(cfg->tile_h, cfg->tile_w)) return SPLAT_ERR_UNSUPPORTED;
    if (cfg->work_cap != 0) return SPLAT_ERR_UNSUPPORTED;
    if (!(cfg->alpha_min > 0.0f && cfg->alpha_min < cfg->alpha_max && cfg->alpha_max < 1.0f &&
          cfg->t_min > 0.0f && cfg->t_min < 1.0f && cfg->sigma_cut > 0.0f))
        return SPLAT_ERR_INVALID_ARG;
    if (cap->max_gaussians < 1 || cap->max_views < 1 || cap->max_views > splat::kMaxViews ||
        cap->max_pixels < 4 || cap->max_pairs < 1 || cap->max_pairs >= (int64_t{1} << 32) ||
        cap->max_tiles < 0)
        return SPLAT_ERR_INVALID_ARG;
    const int64_t mpv = cap->max_gaussians * cap->max_views;
    if (mpv >= (int64_t{1} << 32)) return SPLAT_ERR_INVALID_ARG;

    splat_ctx *c = new splat_ctx;
    c->cfg = *cfg;
    c->cap = *cap;
    if (c->cap.max_tiles == 0)
        c->cap.max_tiles = 2 * (cap->max_pixels / (cfg->tile_h * cfg->tile_w)) +
                           int64_t{256} * cap->max_views;
    c->max_pairs_views = mpv;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t P = cap->max_pixels, M = cap->max_pairs, TT = c->cap.max_tiles;
    c->frame_cap = TT + int64_t{8} * cap->max_views + 64;   // tile rows + tile columns per view
    if (e == cudaSuccess) e = dalloc(&c->d_views, cap->max_views);
    if (e == cudaSuccess) e = dalloc(&c->d_frames, static_cast<size_t>(c->frame_cap) * 4);
    if (e == cudaSuccess) e = dalloc(&c->d_tile_view, TT);
    if (e == cudaSuccess) e = dalloc(&c->d_tileinfo, TT);
    if (e == cudaSuccess) e = dalloc(&c->d_tile_order, TT);
    if (e == cudaSuccess) e = dalloc(&c->d_recs, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_dkeys, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_dvals, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_dkeys2, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_dvals2, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_trect, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_srect, mpv);
    if (e == cudaSuccess) e = dalloc(&c->d_prect, mpv);
    // the tile-sort buffers also hold the sorted lists the forward reads four entries at a
    // time from a 4-aligned index: 128 spare entries keep the last vector in bounds
    if (e == cudaSuccess) e = dalloc(&c->d_tkeys, M + 128);
    if (e == cudaSuccess) e = dalloc(&c->d_tvals, M + 128);
    if (e == cudaSuccess) e = dalloc(&c->d_tkeys2, M + 128);
    if (e == cudaSuccess) e = dalloc(&c->d_tvals2, M + 128);
    if (e == cudaSuccess) e = dalloc(&c->d_block_sums, splat::kScanGrid);
    if (e == cudaSuccess) e = dalloc(&c->d_hist, static_cast<size_t>(splat::kHistWords));
    if (e == cudaSuccess) e = dalloc(&c->d_ranges, TT);
    if (e == cudaSuccess) e = dalloc(&c->d_tfinal, P);
    if (e == cudaSuccess) e = dalloc(&c->d_nlast, P);
    if (e == cudaSuccess) e = dalloc(&c->d_wgrad, static_cast<size_t>(cap->max_gaussians) * 4);
    if (e == cudaSuccess) e = dalloc(&c->d_prim, static_cast<size_t>(cap->max_gaussians) * 3);
    if (e == cudaSuccess) e = dalloc(&c->d_pose, static_cast<size_t>(cap->max_views) * 6);
    if (e == cudaSuccess) e = dalloc(&c->d_samp_thr, static_cast<size_t>(splat::kMaxViews));
    if (e == cudaSuccess) e = dalloc(&c->d_active, static_cast<size_t>(cap->max_views));
    if (e == cudaSuccess) e = dalloc(&c->d_grow_sums, static_cast<size_t>(splat::kGrowMaxGrid + 2));
    // contributor records: at most one per (block, staged entry); the pool takes two per
    // (tile, primitive) pair of capacity plus one partial chunk per work item
    const int64_t items = TT * (splat::kBlock / 32);
    const int64_t chunks = (2 * M + 31) / 32 + items;
    c->rec_cap = static_cast<uint32_t>(chunks < 0xFFFFFFF0ll ? chunks : 0xFFFFFFF0ll);
    if (e == cudaSuccess) e = dalloc(&c->d_rec, static_cast<size_t>(c->rec_cap) * 32);
    if (e == cudaSuccess) e = dalloc(&c->d_rec_prev, static_cast<size_t>(c->rec_cap));
    if (e == cudaSuccess) e = dalloc(&c->d_rec_head, static_cast<size_t>(items));
    if (e == cudaSuccess) e = dalloc(&c->d_rec_fill, static_cast<size_t>(items));
    if (e == cudaSuccess) e = dalloc(&c->d_img, static_cast<size_t>(P) * 5);
    if (e == cudaSuccess) e = dalloc(&c->d_gimg, static_cast<size_t>(P) * 5);
    if (e == cudaSuccess) e = dalloc(&c->d_counters, 8);
    if (e == cudaSuccess) e = dalloc(&c->d_evals, 2);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    for (int k = 0; k < splat_ctx::kStageEvents && e == cudaSuccess; ++k)
        e = cudaEventCreate(&c->stage_ev[k]);
    if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, 8 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_evals, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int r = cuda_fail(e, "splat_ctx_create");
        free_ctx(c);
        return r;
    }
    c->grid_fwd = c->sms * splat::render_occupancy(cfg->tile_h, cfg->tile_w, false);
    c->grid_bwd = c->sms * splat::render_occupancy(cfg->tile_h, cfg->tile_w, true);
    *out = c;
    return SPLAT_OK;
}

SPLAT_API void splat_ctx_destroy(splat_ctx *ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

SPLAT_API int splat_set_views(splat_ctx *ctx, int32_t n_views, const double *T_ws,
                              const splat_lidar_intrinsics *intr)
{
    if (!ctx || !T_ws || !intr || n_views < 1 || n_views > ctx->cap.max_views)
        return SPLAT_ERR_INVALID_ARG;
    const int th = ctx->cfg.tile_h, tw = ctx->cfg.tile_w;
    std::vector<ViewDesc> views(n_views);
    std::vector<SinCos2> frames;
    std::vector<PixFrame> pixframes;
    std::vector<TileInfo> tileinfo;
    std::vector<int32_t> tile_view;
    int64_t pix = 0, tiles = 0;
    for (int v = 0; v < n_views; ++v) {
        const double *T = T_ws + 16 * v;
        const splat_lidar_intrinsics &in = intr[v];
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(T[k])) return SPLAT_ERR_INVALID_ARG;
        if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0) return SPLAT_ERR_INVALID_ARG;
        for (int i = 0; i < 3; ++i)       // R^T R = I
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += T[4 * k + i] * T[4 * k + j];
                if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-6) return SPLAT_ERR_INVALID_ARG;
            }
        const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                           T[2] * (T[4] * T[9] - T[5] * T[8]);
        if (det < 0.5) return SPLAT_ERR_INVALID_ARG;
        if (in.rows < 2 || in.cols < 2 || in.rows > 32767 || in.cols > 32767)
            return SPLAT_ERR_INVALID_ARG;
        if (!(std::isfinite(in.elev_min) && std::isfinite(in.elev_max) &&
              in.elev_min < in.elev_max && in.elev_min > -1.5707f && in.elev_max < 1.5707f))
            return SPLAT_ERR_INVALID_ARG;

        ViewDesc &vd = views[v];
        std::memset(&vd, 0, sizeof vd);
        // T^c_w = inverse of the rigid sensor->world pose; t entries summed as ((a + b) + c)
        double Rcw[9], tcw[3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rcw[3 * i + j] = T[4 * j + i];
        for (int i = 0; i < 3; ++i) {
            const double a = T[4 * 0 + i] * T[3];
            const double b = T[4 * 1 + i] * T[7];
            const double c = T[4 * 2 + i] * T[11];
            tcw[i] = -((a + b) + c);
        }
        for (int k = 0; k < 9; ++k) split(Rcw[k], vd.R_hi[k], vd.R_lo[k]);
        for (int k = 0; k < 3; ++k) split(tcw[k], vd.t_hi[k], vd.t_lo[k]);
        vd.rows = in.rows;
        vd.cols = in.cols;
        vd.elev_min = in.elev_min;
        vd.elev_max = in.elev_max;
        vd.kr = static_cast<float>(in.rows - 1) / (in.elev_max - in.elev_min);
        const double emin = in.elev_min, emax = in.elev_max;
        const double dth = (emax - emin) / (in.rows - 1);
        vd.dgamma = static_cast<float>(2.0 * M_PI / in.cols);
        vd.dtheta = static_cast<float>(dth);
        splat::set_cull_cones(vd, emin, emax, dth);
        vd.tiles_r = (in.rows + th - 1) / th;
        vd.tiles_c = (in.cols + tw - 1) / tw;
        vd.tile_offset = tiles;
        vd.pixel_offset = pix;
        vd.table_offset = static_cast<int32_t>(frames.size());
        for (int tr = 0; tr < vd.tiles_r; ++tr) {
            const double r0 = tr * th + 0.5 * (th - 1);
            const double t0 = emax - r0 * dth;
            SinCos2 e;
            split(std::sin(t0), e.s_hi, e.s_lo);
            split(std::cos(t0), e.c_hi, e.c_lo);
            frames.push_back(e);
        }
        for (int tc = 0; tc < vd.tiles_c; ++tc) {
            const double c0 = tc * tw + 0.5 * (tw - 1);
            const double g0 = M_PI - 2.0 * M_PI * (c0 + 0.5) / in.cols;
            SinCos2 e;
            split(std::sin(g0), e.s_hi, e.s_lo);
            split(std::cos(g0), e.c_hi, e.c_lo);
            frames.push_back(e);
        }
        // pixel planes in the tile frame, in FP64 from exact small angle offsets:
        // dg = gamma - gamma0, dt = theta - theta0, omc = 1 - cos(dg) = 2 sin^2(dg / 2)
        vd.pix_offset = static_cast<int32_t>(pixframes.size());
        for (int tr = 0; tr < vd.tiles_r; ++tr) {
            const double t0 = emax - (tr * th + 0.5 * (th - 1)) * dth;
            const double s0 = std::sin(t0), c0 = std::cos(t0);
            for (int lr = 0; lr < th; ++lr)
                for (int lc = 0; lc < tw; ++lc) {
                    const double dt = -(lr - 0.5 * (th - 1)) * dth;
                    const double dg = -(lc - 0.5 * (tw - 1)) * (2.0 * M_PI / in.cols);
                    const double sg = std::sin(dg), cg = std::cos(dg);
                    const double sh = std::sin(0.5 * dg), omc = 2.0 * sh * sh;
                    const double sdt = std::sin(dt), cdt = std::cos(dt);
                    const double sth = std::sin(t0 + dt), cth = std::cos(t0 + dt);
                    const double hx[3] = {c0 * sg, cg, -s0 * sg};
                    const double hy[3] = {-sdt + c0 * sth * omc, sth * sg, cdt - s0 * sth * omc};
                    const double vv[3] = {cdt - c0 * cth * omc, -cth * sg, sdt + s0 * cth * omc};
                    PixFrame f;
                    std::memset(&f, 0, sizeof f);
                    for (int k = 0; k < 3; ++k) {
                        split(hx[k], f.hx[k], f.hx_lo[k]);
                        split(hy[k], f.hy[k], f.hy_lo[k]);
                        f.v[k] = static_cast<float>(vv[k]);
                    }
                    pixframes.push_back(f);
                }
        }
        // per-tile frames: Q rows e1 = v(theta0, gamma0), e2 = h_x(gamma0), e3 = h_y(theta0,
        // gamma0); M = Q R^c_w, u = Q t^c_w in FP64, stored as float pairs
        for (int tr = 0; tr < vd.tiles_r; ++tr) {
            const double t0 = emax - (tr * th + 0.5 * (th - 1)) * dth;
            const double s0 = std::sin(t0), c0 = std::cos(t0);
            for (int tc = 0; tc < vd.tiles_c; ++tc) {
                const double g0 = M_PI - 2.0 * M_PI * (tc * tw + 0.5 * (tw - 1) + 0.5) / in.cols;
                const double sg = std::sin(g0), cg = std::cos(g0);
                const double Q[9] = {c0 * cg, c0 * sg, s0, sg, -cg, 0.0, -s0 * cg, -s0 * sg, c0};
                TileInfo ti;
                std::memset(&ti, 0, sizeof ti);
                for (int r = 0; r < 3; ++r) {
                    for (int c = 0; c < 3; ++c) {
                        const double m = Q[3 * r] * Rcw[c] + Q[3 * r + 1] * Rcw[3 + c] +
                                         Q[3 * r + 2] * Rcw[6 + c];
                        split(m, ti.M_hi[3 * r + c], ti.M_lo[3 * r + c]);
                    }
                    const double u = Q[3 * r] * tcw[0] + Q[3 * r + 1] * tcw[1] + Q[3 * r + 2] * tcw[2];
                    split(u, ti.u_hi[r], ti.u_lo[r]);
                }
                for (int k = 0; k < 9; ++k) ti.R[k] = vd.R_hi[k];
                ti.view = v;
                ti.tr = tr;
                ti.tc = tc;
                ti.cols = in.cols;
                ti.valid_r = std::min(th, in.rows - tr * th);
                ti.valid_c = std::min(tw, in.cols - tc * tw);
                ti.pix_base = vd.pix_offset + tr * th * tw;
                ti.out_base = pix + static_cast<int64_t>(tr) * th * in.cols + static_cast<int64_t>(tc) * tw;
                tileinfo.push_back(ti);
            }
        }
        const int64_t nt = static_cast<int64_t>(vd.tiles_r) * vd.tiles_c;
        tile_view.insert(tile_view.end(), static_cast<size_t>(nt), v);
        tiles += nt;
        pix += static_cast<int64_t>(in.rows) * in.cols;
    }
    if (pix > ctx->cap.max_pixels || tiles > ctx->cap.max_tiles ||
        static_cast<int64_t>(frames.size()) > ctx->frame_cap)
        return SPLAT_ERR_INVALID_ARG;
    CK(cudaMemcpy(ctx->d_views, views.data(), sizeof(ViewDesc) * views.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_frames, frames.data(), sizeof(SinCos2) * frames.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tile_view, tile_view.data(), sizeof(int32_t) * tile_view.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tileinfo, tileinfo.data(), sizeof(TileInfo) * tileinfo.size(),
                  cudaMemcpyHostToDevice));
    if (static_cast<int64_t>(pixframes.size()) > ctx->pixframe_cap) {
        CK(cudaDeviceSynchronize());
        if (ctx->d_pixframes) CK(cudaFree(ctx->d_pixframes));
        ctx->d_pixframes = nullptr;
        ctx->pixframe_cap = 0;
        CK(dalloc(&ctx->d_pixframes, pixframes.size()));
        ctx->pixframe_cap = static_cast<int64_t>(pixframes.size());
    }
    CK(cudaMemcpy(ctx->d_pixframes, pixframes.data(), sizeof(PixFrame) * pixframes.size(),
                  cudaMemcpyHostToDevice));
    ctx->views = views;
    ctx->n_views = n_views;
    ctx->n_pixels = pix;
    ctx->n_tiles = tiles;
    ctx->rendered = false;
    ctx->have_pose = false;
    ctx->samp_draws = 0;   // the sampling law depends on the views: set it again
    return SPLAT_OK;
}

SPLAT_API int64_t splat_view_pixel_offset(const splat_ctx *ctx, int32_t v)
{
    if (!ctx || v < 0 || v >= ctx->n_views) return -1;
    return ctx->views[v].pixel_offset;
}

SPLAT_API int splat_render_views(splat_ctx *ctx, const splat_gaussians *g, float *depth,
                                 float *normal, float *alpha, void *stream)
{
    if (!ctx) return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    int r = check_gaussians(ctx, g);
    if (r) return r;
    if (!depth || !normal || !alpha) return SPLAT_ERR_INVALID_ARG;
    return render_core(ctx, g, depth, normal, alpha, static_cast<cudaStream_t>(stream));
}

SPLAT_API int splat_render_views_backward(splat_ctx *ctx, const splat_gaussians *g,
                                          const float *dL_ddepth, const float *dL_dnormal,
                                          const float *dL_dalpha, float *g_pos_logit,
                                          float *g_quat, float *g_log_scale, int accumulate,
                                          void *stream)
{
    if (!ctx) return SPLAT_ERR_INVALID_ARG;
    int r = check_gaussians(ctx, g);
    if (r) return r;
    if (!ctx->rendered || g->n != ctx->last_n) return SPLAT_ERR_STATE;
    if (!g_pos_logit || !g_quat || !g_log_scale) return SPLAT_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    r = backward_core(ctx, g, dL_ddepth, dL_dnormal, dL_dalpha, st);
    if (r) return r;
    CK(splat::launch_param_grads(reinterpret_cast<const float4 *>(g->pos_logit),
                                 reinterpret_cast<const float4 *>(g->quat_wxyz),
                                 reinterpret_cast<const float2 *>(g->log_scale), ctx->d_wgrad, g->n,
                                 reinterpret_cast<float4 *>(g_pos_logit),
                                 reinterpret_cast<float4 *>(g_quat),
                                 reinterpret_cast<float2 *>(g_log_scale), accumulate, st));
    ctx->launches += 1;
    return SPLAT_OK;
}

SPLAT_API int splat_render(splat_ctx *ctx, const splat_gaussians *g,
                           const double T_world_sensor[16], const splat_lidar_intrinsics *intr,
                           float *depth, float *normal, float *alpha, void *stream)
{
    int r = splat_set_views(ctx, 1, T_world_sensor, intr);
    if (r) return r;
    return splat_render_views(ctx, g, depth, normal, alpha, stream);
}

SPLAT_API int splat_render_backward(splat_ctx *ctx, const splat_gaussians *g,
                                    const float *dL_ddepth, const float *dL_dnormal,
                                    const float *dL_dalpha, float *g_pos_logit, float *g_quat,
                                    float *g_log_scale, int accumulate, void *stream)
{
    return splat_render_views_backward(ctx, g, dL_ddepth, dL_dnormal, dL_dalpha, g_pos_logit,
                                       g_quat, g_log_scale, accumulate, stream);
}

SPLAT_API int splat_backproject(splat_ctx *ctx, const float *depth, const float *alpha,
                                float o_min, float *points, void *stream)
{
    if (!ctx || !depth || !alpha || !points || !(o_min > 0.0f)) return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(splat::launch_backproject(ctx->d_views, ctx->n_views, ctx->n_pixels, depth, alpha, o_min,
                                 points, st));
    return SPLAT_OK;
}

SPLAT_API int splat_photometric(splat_ctx *ctx, int32_t view, const float *depth,
                                const float *alpha, const float *query_depth, const float *T_qm,
                                float o_min, float huber_delta, double *normal_eqs,
                                float *per_pixel, void *stream)
{
    if (!ctx || !depth || !alpha || !query_depth || !T_qm || !normal_eqs || !(o_min > 0.0f) ||
        !(huber_delta > 0.0f))
        return SPLAT_ERR_INVALID_ARG;
    if (view < 0 || view >= ctx->n_views) return ctx->n_views < 1 ? SPLAT_ERR_STATE
                                                                   : SPLAT_ERR_INVALID_ARG;
    CK(splat::launch_photometric(ctx->views[view], depth, alpha, query_depth, T_qm, o_min,
                                 huber_delta, normal_eqs, per_pixel, ctx->sms,
                                 static_cast<cudaStream_t>(stream)));
    ctx->launches += 1;
    return SPLAT_OK;
}

SPLAT_API int splat_densify(splat_ctx *ctx, const float *target_depth, const float *depth,
                            const float *alpha, const splat_densify_config *cfg, int64_t n_new,
                            float *pos_logit, float *quat, float *log_scale, int64_t n_old,
                            int64_t capacity, void *stream)
{
    if (!ctx || !target_depth || !cfg || !pos_logit || !quat || !log_scale || n_new < 0 ||
        n_old < 0 || n_new > (int64_t{1} << 24) || n_old + n_new > capacity)
        return SPLAT_ERR_INVALID_ARG;
    if (cfg->refine && (!depth || !alpha)) return SPLAT_ERR_INVALID_ARG;
    if (!(cfg->w0 >= 0.0f) || !(cfg->w_cap > 0.0f && cfg->w_cap <= 16.0f) ||
        !(cfg->scale_k > 0.0f) || !(cfg->opacity > 0.0f && cfg->opacity < 1.0f) ||
        !std::isfinite(cfg->lambda_do) || !std::isfinite(cfg->lambda_de))
        return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    // the integer draw needs n_pixels * max weight * n_new < 2^63 (max weight 16 * 256)
    if (ctx->n_pixels > 0 && n_new > 0 &&
        static_cast<double>(ctx->n_pixels) * 4096.0 * static_cast<double>(n_new) >= 9.0e18)
        return SPLAT_ERR_INVALID_ARG;
    splat::GrowArgs a{};
    a.views = ctx->d_views;
    a.n_views = ctx->n_views;
    a.n_pixels = ctx->n_pixels;
    a.t_depth = target_depth;
    a.depth = depth;
    a.alpha = alpha;
    a.refine = cfg->refine ? 1 : 0;
    a.lambda_do = cfg->lambda_do;
    a.lambda_de = cfg->lambda_de;
    a.w0 = cfg->w0;
    a.w_cap = cfg->w_cap;
    a.scale_k = cfg->scale_k;
    a.logit = static_cast<float>(std::log(static_cast<double>(cfg->opacity) /
                                          (1.0 - static_cast<double>(cfg->opacity))));
    a.empty_logit = -30.0f;
    a.seed_lo = static_cast<uint32_t>(cfg->seed);
    a.seed_hi = static_cast<uint32_t>(cfg->seed >> 32);
    a.call = ctx->d_counters + 6;
    a.q = reinterpret_cast<uint32_t *>(ctx->d_gimg);
    a.block_sums = ctx->d_grow_sums;
    a.pos_logit = reinterpret_cast<float4 *>(pos_logit) + n_old;
    a.quat = reinterpret_cast<float4 *>(quat) + n_old;
    a.log_scale = reinterpret_cast<float2 *>(log_scale) + n_old;
    a.n_d = n_new;
    CK(splat::launch_grow(a, static_cast<cudaStream_t>(stream)));
    if (n_new > 0) ctx->launches += 3;
    return SPLAT_OK;
}

SPLAT_API int splat_loss(const float *depth, const float *normal, const float *alpha,
                         const float *target_depth, const float *target_normal,
                         int64_t n_pixels, const splat_loss_config *cfg, float *dL_ddepth,
                         float *dL_dnormal, float *dL_dalpha, double *loss_out, void *stream)
{
    if (!depth || !normal || !alpha || !target_depth || !target_normal || !cfg || !dL_ddepth ||
        !dL_dnormal || !dL_dalpha || !loss_out || n_pixels < 0 ||
        cfg->normal_mode != SPLAT_NORMALS_TARGET)
        return SPLAT_ERR_INVALID_ARG;
    CK(splat::launch_loss(depth, normal, alpha, target_depth, target_normal, n_pixels,
                          cfg->lambda_n, cfg->lambda_o, cfg->o_eps, cfg->rho_exp, dL_ddepth, dL_dnormal,
                          dL_dalpha, loss_out, static_cast<cudaStream_t>(stream)));
    return SPLAT_OK;
}

static bool loss_cfg_ok(const splat_loss_config *cfg, const float *target_normal)
{
    if (cfg->normal_mode == SPLAT_NORMALS_TARGET) return target_normal != nullptr;
    return cfg->normal_mode == SPLAT_NORMALS_RANGE_MAP;
}

SPLAT_API int splat_view_loss(splat_ctx *ctx, const float *depth, const float *normal,
                              const float *alpha, const float *target_depth,
                              const float *target_normal, const splat_loss_config *cfg,
                              float *dL_ddepth, float *dL_dnormal, float *dL_dalpha,
                              double *loss_out, void *stream)
{
    if (!ctx || !depth || !normal || !alpha || !target_depth || !cfg || !dL_ddepth ||
        !dL_dnormal || !dL_dalpha || !loss_out || !loss_cfg_ok(cfg, target_normal))
        return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    CK(splat::launch_loss(depth, normal, alpha, target_depth, target_normal, ctx->n_pixels,
                          cfg->lambda_n, cfg->lambda_o, cfg->o_eps, cfg->rho_exp, dL_ddepth, dL_dnormal,
                          dL_dalpha, loss_out, static_cast<cudaStream_t>(stream), ctx->d_views,
                          ctx->n_views, nullptr, cfg->normal_mode));
    return SPLAT_OK;
}

SPLAT_API int splat_adam_step(float *pos_logit, float *quat, float *log_scale,
                              const float *g_pos_logit, const float *g_quat,
                              const float *g_log_scale, float *m_pos_logit, float *m_quat,
                              float *m_log_scale, float *v_pos_logit, float *v_quat,
                              float *v_log_scale, int32_t *step, int64_t n,
                              const splat_adam_config *cfg, void *stream)
{
    if (!pos_logit || !quat || !log_scale || !g_pos_logit || !g_quat || !g_log_scale ||
        !m_pos_logit || !m_quat || !m_log_scale || !v_pos_logit || !v_quat || !v_log_scale ||
        !step || !cfg || n < 0)
        return SPLAT_ERR_INVALID_ARG;
    splat::AdamArgs a{};
    a.pos_logit = reinterpret_cast<float4 *>(pos_logit);
    a.quat = reinterpret_cast<float4 *>(quat);
    a.log_scale = reinterpret_cast<float2 *>(log_scale);
    a.m_pl = reinterpret_cast<float4 *>(m_pos_logit);
    a.m_q = reinterpret_cast<float4 *>(m_quat);
    a.m_ls = reinterpret_cast<float2 *>(m_log_scale);
    a.v_pl = reinterpret_cast<float4 *>(v_pos_logit);
    a.v_q = reinterpret_cast<float4 *>(v_quat);
    a.v_ls = reinterpret_cast<float2 *>(v_log_scale);
    a.step = step;
    a.n = n;
    a.lr_pos = cfg->lr_pos;
    a.lr_opacity = cfg->lr_opacity;
    a.lr_rot = cfg->lr_rot;
    a.lr_scale = cfg->lr_scale;
    a.beta1 = cfg->beta1;
    a.beta2 = cfg->beta2;
    a.eps = cfg->eps;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(splat::launch_adam(a, reinterpret_cast<const float4 *>(g_pos_logit),
                          reinterpret_cast<const float4 *>(g_quat),
                          reinterpret_cast<const float2 *>(g_log_scale), st));
    CK(splat::launch_step_inc(step, st));
    return SPLAT_OK;
}

SPLAT_API int splat_refine_step(splat_ctx *ctx, float *pos_logit, float *quat, float *log_scale,
                                int64_t n, const float *target_depth, const float *target_normal,
                                const splat_loss_config *loss_cfg,
                                const splat_adam_config *adam_cfg, float *m_pos_logit,
                                float *m_quat, float *m_log_scale, float *v_pos_logit,
                                float *v_quat, float *v_log_scale, int32_t *step,
                                double *loss_out, void *stream)
{
    if (!ctx || !target_depth || !loss_cfg || !adam_cfg || !m_pos_logit || !m_quat ||
        !m_log_scale || !v_pos_logit || !v_quat || !v_log_scale || !step || !loss_out ||
        !loss_cfg_ok(loss_cfg, target_normal))
        return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    splat_gaussians g{pos_logit, quat, log_scale, n};
    int r = check_gaussians(ctx, &g);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t P = ctx->n_pixels;
    float *depth = ctx->d_img, *normal = ctx->d_img + P, *alpha = ctx->d_img + 4 * P;
    float *gd = ctx->d_gimg, *gn = ctx->d_gimg + P, *ga = ctx->d_gimg + 4 * P;
    r = render_core(ctx, &g, depth, normal, alpha, st);
    if (r) return r;
    CK(cudaMemsetAsync(loss_out, 0, sizeof(double), st));
    CK(splat::launch_loss(depth, normal, alpha, target_depth, target_normal, P, loss_cfg->lambda_n,
                          loss_cfg->lambda_o, loss_cfg->o_eps, loss_cfg->rho_exp, gd, gn, ga,
                          loss_out, st,
                          ctx->d_views, ctx->n_views,
                          ctx->samp_draws > 0 ? ctx->d_active : nullptr,
                          loss_cfg->normal_mode));
    const bool prof = ctx->profiling && !capturing(st);
    if (prof) {
        CK(cudaEventRecord(ctx->stage_ev[6], st));
        ctx->stage_rec[6] = true;
    }
    r = backward_core(ctx, &g, gd, gn, ga, st);
    if (r) return r;
    splat::AdamArgs a{};
    a.pos_logit = reinterpret_cast<float4 *>(pos_logit);
    a.quat = reinterpret_cast<float4 *>(quat);
    a.log_scale = reinterpret_cast<float2 *>(log_scale);
    a.m_pl = reinterpret_cast<float4 *>(m_pos_logit);
    a.m_q = reinterpret_cast<float4 *>(m_quat);
    a.m_ls = reinterpret_cast<float2 *>(m_log_scale);
    a.v_pl = reinterpret_cast<float4 *>(v_pos_logit);
    a.v_q = reinterpret_cast<float4 *>(v_quat);
    a.v_ls = reinterpret_cast<float2 *>(v_log_scale);
    a.step = step;
    a.n = n;
    a.lr_pos = adam_cfg->lr_pos;
    a.lr_opacity = adam_cfg->lr_opacity;
    a.lr_rot = adam_cfg->lr_rot;
    a.lr_scale = adam_cfg->lr_scale;
    a.beta1 = adam_cfg->beta1;
    a.beta2 = adam_cfg->beta2;
    a.eps = adam_cfg->eps;
    a.lambda_s = loss_cfg->lambda_s;
    a.tau_s = loss_cfg->tau_s;
    a.loss_out = loss_out;
    CK(splat::launch_adam_fused(a, ctx->d_wgrad, st));
    if (prof) {
        CK(cudaEventRecord(ctx->stage_ev[7], st));
        ctx->stage_rec[7] = true;
    }
    CK(splat::launch_step_inc(step, st));
    ctx->launches += 3;   // loss, fused Adam, step counter
    return SPLAT_OK;
}

SPLAT_API int splat_set_view_sampling(splat_ctx *ctx, int draws, double p_newest, uint64_t seed)
{
    if (!ctx || draws < 0) return SPLAT_ERR_INVALID_ARG;
    if (draws == 0) {
        ctx->samp_draws = 0;
        return SPLAT_OK;
    }
    if (!(p_newest > 0.0 && p_newest <= 1.0)) return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    // truncated geometric law over keyframe age, cumulative, as integer thresholds (FP64, the
    // products and sums in age order)
    const int K = ctx->n_views;
    std::vector<double> P(static_cast<size_t>(K));
    double w = p_newest;
    for (int a = 0; a < K; ++a) {
        P[a] = w;
        w = w * (1.0 - p_newest);
    }
    double Z = 0.0;
    for (int a = 0; a < K; ++a) Z = Z + P[a];
    std::vector<uint32_t> thr(static_cast<size_t>(splat::kMaxViews), 0u);
    double c = 0.0;
    for (int a = 0; a + 1 < K; ++a) {
        c = c + P[a];
        const double v = std::floor((c / Z) * 4294967296.0);
        thr[a] = v >= 4294967295.0 ? 0xFFFFFFFFu : static_cast<uint32_t>(v);
    }
    CK(cudaMemcpy(ctx->d_samp_thr, thr.data(), sizeof(uint32_t) * thr.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->d_counters + 7, 0, sizeof(uint32_t)));
    ctx->samp_draws = draws;
    ctx->samp_seed = seed;
    return SPLAT_OK;
}

SPLAT_API int splat_get_active_views(splat_ctx *ctx, uint8_t *flags)
{
    if (!ctx || !flags) return SPLAT_ERR_INVALID_ARG;
    if (ctx->n_views < 1) return SPLAT_ERR_STATE;
    CK(cudaDeviceSynchronize());
    if (ctx->samp_draws > 0) {
        CK(cudaMemcpy(flags, ctx->d_active, static_cast<size_t>(ctx->n_views),
                      cudaMemcpyDeviceToHost));
    } else {
        for (int v = 0; v < ctx->n_views; ++v) flags[v] = 1;
    }
    return SPLAT_OK;
}

SPLAT_API int splat_set_pose_gradient(splat_ctx *ctx, int enable)
{
    if (!ctx) return SPLAT_ERR_INVALID_ARG;
    ctx->want_pose = enable != 0;
    return SPLAT_OK;
}

SPLAT_API int splat_pose_gradient(splat_ctx *ctx, float *g_pose, void *stream)
{
    if (!ctx || !g_pose) return SPLAT_ERR_INVALID_ARG;
    if (!ctx->have_pose) return SPLAT_ERR_STATE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(g_pose, ctx->d_pose, sizeof(float) * 6 * static_cast<size_t>(ctx->n_views),
                       cudaMemcpyDeviceToDevice, st));
    return SPLAT_OK;
}

SPLAT_API int splat_get_status(splat_ctx *ctx, uint32_t *flags)
{
    if (!ctx || !flags) return SPLAT_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(flags, ctx->d_counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->d_counters + 1, 0, sizeof(uint32_t)));
    return SPLAT_OK;
}

SPLAT_API int splat_get_stats(splat_ctx *ctx, splat_stats *out)
{
    if (!ctx || !out) return SPLAT_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    uint32_t c[5] = {0, 0, 0, 0, 0};
    unsigned long long ev[2] = {0, 0};
    CK(cudaMemcpy(c, ctx->d_counters, sizeof c, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ev, ctx->d_evals, sizeof ev, cudaMemcpyDeviceToHost));
    out->n_pairs = c[0];
    out->n_touching = c[4];
    out->fwd_evals = static_cast<int64_t>(ev[0]);
    out->bwd_evals = static_cast<int64_t>(ev[1]);
    out->n_pixels = ctx->n_pixels;
    out->n_tiles = ctx->n_tiles;
    out->kernel_launches = ctx->launches;
    return SPLAT_OK;
}

SPLAT_API int splat_set_profiling(splat_ctx *ctx, int enable)
{
    if (!ctx) return SPLAT_ERR_INVALID_ARG;
    ctx->profiling = enable != 0;
    ctx->rec_fwd = ctx->rec_bwd = false;
    for (bool &b : ctx->stage_rec) b = false;
    return SPLAT_OK;
}

SPLAT_API int splat_kernel_times(splat_ctx *ctx, float *fwd_ms, float *bwd_ms)
{
    if (!ctx || !fwd_ms || !bwd_ms) return SPLAT_ERR_INVALID_ARG;
    *fwd_ms = -1.0f;
    *bwd_ms = -1.0f;
    if (ctx->rec_fwd) {
        CK(cudaEventSynchronize(ctx->ev[1]));
        CK(cudaEventElapsedTime(fwd_ms, ctx->ev[0], ctx->ev[1]));
    }
    if (ctx->rec_bwd) {
        CK(cudaEventSynchronize(ctx->ev[3]));
        CK(cudaEventElapsedTime(bwd_ms, ctx->ev[2], ctx->ev[3]));
    }
    return SPLAT_OK;
}

SPLAT_API int splat_stage_times(splat_ctx *ctx, float *ms)
{
    if (!ctx || !ms) return SPLAT_ERR_INVALID_ARG;
    // stage k of the render runs between stage events k and k + 1; the loss between the end of
    // the forward compositing and event 6, the fused Adam between the end of the backward and 7
    struct Span {
        cudaEvent_t a, b;
        bool ok;
    };
    const Span spans[7] = {
        {ctx->stage_ev[0], ctx->stage_ev[1], ctx->stage_rec[0] && ctx->stage_rec[1]},
        {ctx->stage_ev[1], ctx->stage_ev[2], ctx->stage_rec[1] && ctx->stage_rec[2]},
        {ctx->stage_ev[2], ctx->stage_ev[3], ctx->stage_rec[2] && ctx->stage_rec[3]},
        {ctx->stage_ev[3], ctx->stage_ev[4], ctx->stage_rec[3] && ctx->stage_rec[4]},
        {ctx->stage_ev[4], ctx->stage_ev[5], ctx->stage_rec[4] && ctx->stage_rec[5]},
        {ctx->ev[1], ctx->stage_ev[6], ctx->rec_fwd && ctx->stage_rec[6]},
        {ctx->ev[3], ctx->stage_ev[7], ctx->rec_bwd && ctx->stage_rec[7]},
    };
    for (int k = 0; k < 7; ++k) {
        ms[k] = -1.0f;
        if (!spans[k].ok) continue;
        CK(cudaEventSynchronize(spans[k].b));
        CK(cudaEventElapsedTime(&ms[k], spans[k].a, spans[k].b));
    }
    return SPLAT_OK;
}

SPLAT_API int64_t splat_debug_copy(splat_ctx *ctx, int32_t which, void *dst, int64_t bytes)
{
    if (!ctx || !dst || bytes < 0) return -1;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    uint32_t m = 0;
    if (cudaMemcpy(&m, ctx->d_counters, sizeof m, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    const void *src = nullptr;
    int64_t need = 0;
    switch (which) {
    case 0: src = ctx->sorted_keys; need = int64_t{4} * m; break;
    case 1: src = ctx->sorted_vals; need = int64_t{4} * m; break;
    case 2: src = ctx->d_ranges; need = int64_t{8} * ctx->n_tiles; break;
    case 3: src = ctx->d_recs; need = int64_t{16} * ctx->last_n * ctx->n_views; break;
    case 4: src = ctx->d_tfinal; need = int64_t{4} * ctx->n_pixels; break;
    case 5: src = ctx->d_nlast; need = int64_t{4} * ctx->n_pixels; break;
    default: return -1;
    }
    if (!ctx->rendered || !src) return -1;
    if (need > bytes) return -1;
    if (need > 0 && cudaMemcpy(dst, src, static_cast<size_t>(need), cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    return need;
}

}  // extern "C"
