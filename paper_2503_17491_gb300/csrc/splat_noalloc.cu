// splat_render_noalloc: the forward render of one view without a context and without any
// allocation, for callers that cannot allocate device memory themselves -- for example code
// that runs after its process has handed all device memory to another allocator, or that must
// not call cudaMalloc once it is running.
//
// Every buffer the render pipeline needs (projection records, sort buffers and histograms, tile
// lists, tile tables, per-pixel auxiliaries, counters) lives in one file-scope __device__ array,
// g_noalloc_scratch, sized for the limits below.  The host-side tables are built in file-scope
// host arrays.  Nothing here calls cudaMalloc, cudaFree, malloc or new.
//
// Limits: at most kMaxGaussians primitives, kMaxRows image rows, kMaxPixels pixels, kMaxTiles
// tiles and kMaxPairs (tile, primitive) pairs; larger requests return SPLAT_ERR_INVALID_ARG
// (sizes) or SPLAT_ERR_CAPACITY (pairs, found on the device).
//
// Every call shares the one array (and the host tables): calls must not overlap, neither on the
// GPU nor from several host threads.  The first call on a device is the set-up call: CUDA loads
// the library's code on first use (lazy module loading), which is when the array and the kernels
// it launches take their device memory, and the call looks up the array's device address
// (cudaGetSymbolAddress) with that device current, once per device.  That call must come before
// the device's memory is handed to another allocator and outside any stream capture.

#include <cmath>
#include <cstring>

#include "splat_internal.cuh"

using splat::PairRec;
using splat::PixFrame;
using splat::TileInfo;
using splat::ViewDesc;

namespace {

constexpr int64_t kMaxGaussians = 16384;
constexpr int kMaxRows = 256;
constexpr int64_t kMaxPixels = 65536;
constexpr int kMaxTiles = 4096;
constexpr int64_t kMaxPairs = 262144;
constexpr int kMaxTileRows = kMaxRows / 4 + 1;   // tile_h >= 4
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t{255}; }

// byte offsets inside the scratch array
constexpr size_t kOffRecs = 0;
constexpr size_t kOffDkeys = align256(kOffRecs + sizeof(PairRec) * kMaxGaussians);
constexpr size_t kOffDvals = align256(kOffDkeys + 4 * kMaxGaussians);
constexpr size_t kOffDkeys2 = align256(kOffDvals + 4 * kMaxGaussians);
constexpr size_t kOffDvals2 = align256(kOffDkeys2 + 4 * kMaxGaussians);
constexpr size_t kOffTrect = align256(kOffDvals2 + 4 * kMaxGaussians);
constexpr size_t kOffSrect = align256(kOffTrect + 8 * kMaxGaussians);
constexpr size_t kOffPrect = align256(kOffSrect + 8 * kMaxGaussians);
constexpr size_t kOffPrim = align256(kOffPrect + 8 * kMaxGaussians);
constexpr size_t kOffTkeys = align256(kOffPrim + 3 * sizeof(float4) * kMaxGaussians);
constexpr size_t kOffTvals = align256(kOffTkeys + 4 * kMaxPairs);
constexpr size_t kOffTkeys2 = align256(kOffTvals + 4 * kMaxPairs);
constexpr size_t kOffTvals2 = align256(kOffTkeys2 + 4 * kMaxPairs);
constexpr size_t kOffBlockSums = align256(kOffTvals2 + 4 * kMaxPairs);
constexpr size_t kOffHist = align256(kOffBlockSums + 4 * splat::kScanGrid);
constexpr size_t kOffRanges = align256(kOffHist + 4 * size_t{splat::kHistWords});
constexpr size_t kOffOrder = align256(kOffRanges + 8 * size_t{kMaxTiles});
constexpr size_t kOffTiles = align256(kOffOrder + 4 * size_t{kMaxTiles});
constexpr size_t kOffPix = align256(kOffTiles + sizeof(TileInfo) * kMaxTiles);
constexpr size_t kOffView = align256(kOffPix + sizeof(PixFrame) * size_t{kMaxTileRows} * 256);
constexpr size_t kOffTfinal = align256(kOffView + sizeof(ViewDesc));
constexpr size_t kOffNlast = align256(kOffTfinal + 4 * kMaxPixels);
constexpr size_t kOffCounters = align256(kOffNlast + 4 * kMaxPixels);
constexpr size_t kOffEvals = align256(kOffCounters + 4 * 8);
constexpr size_t kScratchBytes = align256(kOffEvals + 8 * 2);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// host-side tables, filled per call
ViewDesc g_view;
PixFrame g_pix[kMaxTileRows * 256];
TileInfo g_tiles[kMaxTiles];

// per-device address of g_noalloc_scratch (0 until looked up)
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

void split(double x, float &hi, float &lo)
{
    hi = static_cast<float>(x);
    lo = static_cast<float>(x - static_cast<double>(hi));
}

int bits_for(int64_t n)
{
    int b = 0;
    while ((int64_t{1} << b) < n) ++b;
    return ((b + 7) / 8) * 8;
}

// view tables of one view in the host arrays (same definitions as view registration)
int build_tables(const double *T, const splat_lidar_intrinsics &in, int th, int tw,
                 int64_t *n_tiles)
{
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(T[k])) return SPLAT_ERR_INVALID_ARG;
    if (T[12] != 0.0 || T[13] != 0.0 || T[14] != 0.0 || T[15] != 1.0) return SPLAT_ERR_INVALID_ARG;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += T[4 * k + i] * T[4 * k + j];
            if (std::fabs(s - (i == j ? 1.0 : 0.0)) > 1e-6) return SPLAT_ERR_INVALID_ARG;
        }
    const double det = T[0] * (T[5] * T[10] - T[6] * T[9]) - T[1] * (T[4] * T[10] - T[6] * T[8]) +
                       T[2] * (T[4] * T[9] - T[5] * T[8]);
    if (det < 0.5) return SPLAT_ERR_INVALID_ARG;
    if (in.rows < 2 || in.cols < 2 || in.rows > kMaxRows ||
        int64_t{in.rows} * in.cols > kMaxPixels)
        return SPLAT_ERR_INVALID_ARG;
    if (!(std::isfinite(in.elev_min) && std::isfinite(in.elev_max) &&
          in.elev_min < in.elev_max && in.elev_min > -1.5707f && in.elev_max < 1.5707f))
        return SPLAT_ERR_INVALID_ARG;
    const int tiles_r = (in.rows + th - 1) / th, tiles_c = (in.cols + tw - 1) / tw;
    if (int64_t{tiles_r} * tiles_c > kMaxTiles || tiles_r > kMaxTileRows) return SPLAT_ERR_INVALID_ARG;

    ViewDesc &vd = g_view;
    std::memset(&vd, 0, sizeof vd);
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
    vd.tiles_r = tiles_r;
    vd.tiles_c = tiles_c;
    vd.tile_offset = 0;
    vd.pixel_offset = 0;
    vd.table_offset = 0;
    vd.pix_offset = 0;
    for (int tr = 0; tr < tiles_r; ++tr) {
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
                PixFrame &f = g_pix[tr * th * tw + lr * tw + lc];
                std::memset(&f, 0, sizeof f);
                for (int k = 0; k < 3; ++k) {
                    split(hx[k], f.hx[k], f.hx_lo[k]);
                    split(hy[k], f.hy[k], f.hy_lo[k]);
                    f.v[k] = static_cast<float>(vv[k]);
                }
            }
        for (int tc = 0; tc < tiles_c; ++tc) {
            const double g0 = M_PI - 2.0 * M_PI * (tc * tw + 0.5 * (tw - 1) + 0.5) / in.cols;
            const double sg = std::sin(g0), cg = std::cos(g0);
            const double Q[9] = {c0 * cg, c0 * sg, s0, sg, -cg, 0.0, -s0 * cg, -s0 * sg, c0};
            TileInfo &ti = g_tiles[tr * tiles_c + tc];
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
            ti.view = 0;
            ti.tr = tr;
            ti.tc = tc;
            ti.cols = in.cols;
            ti.valid_r = in.rows - tr * th < th ? in.rows - tr * th : th;
            ti.valid_c = in.cols - tc * tw < tw ? in.cols - tc * tw : tw;
            ti.pix_base = tr * th * tw;
            ti.out_base = static_cast<int64_t>(tr) * th * in.cols + static_cast<int64_t>(tc) * tw;
        }
    }
    *n_tiles = int64_t{tiles_r} * tiles_c;
    return SPLAT_OK;
}

bool supported_tile(int th, int tw)
{
    return (th == 16 && tw == 16) || (th == 8 && tw == 32) || (th == 32 && tw == 8) ||
           (th == 4 && tw == 64);
}

#define NA_CK(call)                                                 \
    do {                                                            \
        const cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return splat::cuda_fail(e_, #call);  \
    } while (0)

}  // namespace

extern "C" SPLAT_API int splat_render_noalloc(const splat_gaussians *g,
                                              const double T_world_sensor[16],
                                              const splat_lidar_intrinsics *intr,
                                              const splat_render_config *cfg_in, float *depth,
                                              float *normal, float *alpha, void *stream)
{
    if (!g || !T_world_sensor || !intr || !depth || !normal || !alpha) return SPLAT_ERR_INVALID_ARG;
    if (g->n < 0 || g->n > kMaxGaussians) return SPLAT_ERR_INVALID_ARG;
    if (g->n > 0 && (!g->pos_logit || !g->quat_wxyz || !g->log_scale)) return SPLAT_ERR_INVALID_ARG;
    splat_render_config cfg;
    if (cfg_in) {
        cfg = *cfg_in;
    } else {
        splat_default_config(&cfg);
    }
    if (!supported_tile(cfg.tile_h, cfg.tile_w) || cfg.work_cap != 0) return SPLAT_ERR_UNSUPPORTED;
    int64_t n_tiles = 0;
    int r = build_tables(T_world_sensor, *intr, cfg.tile_h, cfg.tile_w, &n_tiles);
    if (r) return r;

    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SPLAT_ERR_INVALID_ARG;
    if (!g_scratch_addr[dev]) {   // once per device, with that device current
        void *p = nullptr;
        NA_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    unsigned char *base = g_scratch_addr[dev];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int th = cfg.tile_h, tw = cfg.tile_w;
    const int64_t n = g->n;
    const int64_t P = int64_t{intr->rows} * intr->cols;

    PairRec *recs = reinterpret_cast<PairRec *>(base + kOffRecs);
    uint32_t *dkeys = reinterpret_cast<uint32_t *>(base + kOffDkeys);
    uint32_t *dvals = reinterpret_cast<uint32_t *>(base + kOffDvals);
    uint32_t *dkeys2 = reinterpret_cast<uint32_t *>(base + kOffDkeys2);
    uint32_t *dvals2 = reinterpret_cast<uint32_t *>(base + kOffDvals2);
    uint64_t *trect = reinterpret_cast<uint64_t *>(base + kOffTrect);
    uint64_t *srect = reinterpret_cast<uint64_t *>(base + kOffSrect);
    uint64_t *prect = reinterpret_cast<uint64_t *>(base + kOffPrect);
    uint32_t *tkeys = reinterpret_cast<uint32_t *>(base + kOffTkeys);
    uint32_t *tvals = reinterpret_cast<uint32_t *>(base + kOffTvals);
    uint32_t *tkeys2 = reinterpret_cast<uint32_t *>(base + kOffTkeys2);
    uint32_t *tvals2 = reinterpret_cast<uint32_t *>(base + kOffTvals2);
    float4 *prim = reinterpret_cast<float4 *>(base + kOffPrim);
    uint32_t *block_sums = reinterpret_cast<uint32_t *>(base + kOffBlockSums);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + kOffHist);
    uint2 *ranges = reinterpret_cast<uint2 *>(base + kOffRanges);
    uint32_t *order = reinterpret_cast<uint32_t *>(base + kOffOrder);
    TileInfo *tiles = reinterpret_cast<TileInfo *>(base + kOffTiles);
    PixFrame *pix = reinterpret_cast<PixFrame *>(base + kOffPix);
    ViewDesc *view = reinterpret_cast<ViewDesc *>(base + kOffView);
    float *tfinal = reinterpret_cast<float *>(base + kOffTfinal);
    int32_t *nlast = reinterpret_cast<int32_t *>(base + kOffNlast);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(base + kOffCounters);
    unsigned long long *evals = reinterpret_cast<unsigned long long *>(base + kOffEvals);

    // the tables of this call, and every counter that must start at zero (the array keeps the
    // previous call's contents)
    NA_CK(cudaMemcpyAsync(view, &g_view, sizeof(ViewDesc), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(tiles, g_tiles, sizeof(TileInfo) * n_tiles, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(pix, g_pix, sizeof(PixFrame) * g_view.tiles_r * th * tw,
                          cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(cnt, 0, 4 * 8, st));
    NA_CK(cudaMemsetAsync(evals, 0, 8 * 2, st));

    NA_CK(splat::launch_project(reinterpret_cast<const float4 *>(g->pos_logit),
                                reinterpret_cast<const float4 *>(g->quat_wxyz),
                                reinterpret_cast<const float2 *>(g->log_scale), n, view, 1,
                                cfg.sigma_cut, cfg.alpha_min, th, tw, cfg.flip_normals, recs, dkeys,
                                dvals, trect, prect, prim, cnt + 1, cnt + 4, st));
    uint32_t *dk, *dv;
    NA_CK(splat::radix_sort_pairs(dkeys, dvals, dkeys2, dvals2, nullptr, n, 32, hist, &dk, &dv, st,
                                  nullptr, trect, srect));
    NA_CK(splat::launch_emit(dv, srect, n, cnt + 4, view, n, block_sums, tkeys, tvals, kMaxPairs,
                             cnt, cnt + 1, st));
    uint32_t *tk, *tv;
    NA_CK(splat::radix_sort_pairs(tkeys, tvals, tkeys2, tvals2, cnt, kMaxPairs, bits_for(n_tiles),
                                  hist, &tk, &tv, st));
    uint32_t *rects = tv == tvals ? tvals2 : tvals;   // the tile sort's free buffers
    uint8_t *blocks = reinterpret_cast<uint8_t *>(tk == tkeys ? tkeys2 : tkeys);
    NA_CK(splat::launch_ranges(tk, tv, prect, tiles, th, tw, cnt, kMaxPairs, ranges, n_tiles, rects,
                               blocks, st));
    NA_CK(splat::launch_order_tiles(ranges, n_tiles, order, st));

    splat::RenderArgs a{};
    a.pos_logit = reinterpret_cast<const float4 *>(g->pos_logit);
    a.prim = prim;
    a.n = n;
    a.tiles = tiles;
    a.pixframes = pix;
    a.ranges = ranges;
    a.tile_order = order;
    a.sorted_vals = tv;
    a.entry_rect = rects;
    a.entry_blocks = blocks;
    a.status = cnt + 1;   // no contributor records (forward only)
    a.n_tiles = n_tiles;
    a.n_items = n_tiles * (splat::kBlock / 32);
    a.alpha_min = cfg.alpha_min;
    a.alpha_max = cfg.alpha_max;
    a.t_min = cfg.t_min;
    a.sigma = cfg.sigma_cut;
    a.depth = depth;
    a.normal = normal;
    a.alpha = alpha;
    a.n_pixels = P;
    a.t_final = tfinal;
    a.n_last = nlast;
    a.queue = cnt + 2;
    a.evals = evals;
    int sms = 0;
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * splat::render_occupancy(th, tw, false);
    NA_CK(splat::launch_render_fwd(a, th, tw, grid, st));

    // the status word was produced on the device: wait for it and report it
    uint32_t status = 0;
    NA_CK(cudaMemcpyAsync(&status, cnt + 1, sizeof status, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (status & SPLAT_STATUS_CAPACITY) return SPLAT_ERR_CAPACITY;
    if (status & SPLAT_STATUS_NONFINITE) return SPLAT_ERR_NONFINITE;
    return SPLAT_OK;
}
