// Internal definitions shared by the translation units of libsplatloam (not part of the ABI).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/splatloam.h"

namespace splat {

constexpr int kMaxViews = 64;
constexpr int kBlock = 256;          // threads per render CTA = pixels per tile

// ---------------------------------------------------------------------------------------------
// per-view descriptor (device)
// ---------------------------------------------------------------------------------------------
struct ViewDesc {
    // T^c_w as float pairs (hi = nearest float of the FP64 value, lo = nearest float of the rest)
    float R_hi[9], R_lo[9];       // row-major
    float t_hi[3], t_lo[3];
    int32_t rows, cols;
    float elev_min, elev_max;
    float kr;                     // binary32 (rows - 1) / (elev_max - elev_min): contract rows
    float dgamma;                 // 2 pi / cols  (nearest float)
    float dtheta;                 // (elev_max - elev_min) / (rows - 1)  (nearest float)
    int32_t tiles_r, tiles_c;     // tile rows / columns of this view
    int64_t tile_offset;          // first global tile id of the view
    int64_t pixel_offset;         // first pixel of the view in the packed buffers
    int32_t table_offset;         // into the frame table: tiles_r rows then tiles_c columns
    int32_t pix_offset;           // into the pixel-frame table: tiles_r x 256 entries
    // cones two rows (and a milliradian) beyond the top and bottom rows: z = t |xy|, with
    // l = sqrt(1 + t^2) the Lipschitz constant of z - t |xy| (l = inf: no cone)
    float cull_t_top, cull_l_top, cull_t_bot, cull_l_bot;
};

// Pixel-centre ray of pixel (r, c) of a view (Sec. 3.1), binary32.
__device__ __forceinline__ float3 pixel_ray(const ViewDesc &vd, int r, int c)
{
    const float g = 3.14159265358979f - vd.dgamma * (static_cast<float>(c) + 0.5f);
    const float th = vd.rows > 1 ? vd.elev_max - vd.dtheta * static_cast<float>(r) : vd.elev_max;
    float sg, cg, st, ct;
    sincosf(g, &sg, &cg);
    sincosf(th, &st, &ct);
    return make_float3(ct * cg, ct * sg, st);
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011), from its definition: a round maps
// (c0, c1, c2, c3) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
// is bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += W0;
            k.y += W1;
        }
    }
    return c;
}

// Keyframe sampling (Sec. 3.3): draws j < draws of refinement step *step take the first word x of
// Philox-4x32-10((j, step, 0, 0), (seed lo, seed hi)); the drawn view is n_views - 1 - #{a :
// x >= thr[a]} (thr: n_views - 1 integer thresholds of the cumulative law); active[v] = 1 for a
// view drawn at least once, 0 otherwise; *step then advances by one.
cudaError_t launch_sample_views(int n_views, int draws, const uint32_t *thr, uint32_t seed_lo,
                                uint32_t seed_hi, uint32_t *step, uint8_t *active,
                                cudaStream_t st);

// Back-projection of the packed range images of the registered views to world-frame points
// (3 x n_pixels planar, NaN where O < o_min).
cudaError_t launch_backproject(const ViewDesc *views, int n_views, int64_t n_pixels,
                               const float *depth, const float *alpha, float o_min, float *points,
                               cudaStream_t st);

// Map growth (Sec. 3.3.1, 3.3.2): mask, range-gradient weights and a systematic draw of n_d
// pixels over the packed pixels of the views; slot j of the new primitives takes the pixel that
// holds sample j first, or is written empty.
constexpr int kGrowMaxGrid = 1024;
struct GrowArgs {
    const ViewDesc *views;
    int n_views;
    int64_t n_pixels;
    const float *t_depth, *depth, *alpha;   // depth, alpha: used when refine != 0
    int refine;
    float lambda_do, lambda_de, w0, w_cap, scale_k, logit, empty_logit;
    uint32_t seed_lo, seed_hi;
    uint32_t *call;                         // device counter of draws, advanced per call
    uint32_t *q;                            // scratch, n_pixels
    unsigned long long *block_sums;         // scratch, kGrowMaxGrid + 2
    float4 *pos_logit, *quat;               // the n_d new slots
    float2 *log_scale;
    int64_t n_d;
    int grid;                               // set by launch_grow
    int64_t chunk;
};
cudaError_t launch_grow(GrowArgs a, cudaStream_t st);

// Photometric residual of one view against a query range image and its Gauss-Newton normal
// equations (Sec. 3.3.3): out[29] = H upper triangle (21, row-major), g (6), Huber cost, count;
// per_pixel (nullable) = 8 x P planar: r, w, J (6).  T: device binary32 3 x 4 render -> query.
cudaError_t launch_photometric(const ViewDesc &vd, const float *depth, const float *alpha,
                               const float *qdepth, const float *T, float o_min, float delta,
                               double *out, float *per_pixel, int sms, cudaStream_t st);

// the culling cones of a view (host)
inline void set_cull_cones(ViewDesc &vd, double emin, double emax, double dtheta)
{
    const double m = 2.0 * dtheta + 1e-3;
    const double top = emax + m, bot = emin - m, lim = 1.5;   // well inside +-pi/2
    vd.cull_t_top = top < lim ? static_cast<float>(std::tan(top)) : 0.0f;
    vd.cull_l_top = top < lim ? static_cast<float>(std::sqrt(1.0 + std::tan(top) * std::tan(top)) *
                                                   1.0001)
                              : INFINITY;
    vd.cull_t_bot = bot > -lim ? static_cast<float>(std::tan(bot)) : 0.0f;
    vd.cull_l_bot = bot > -lim ? static_cast<float>(std::sqrt(1.0 + std::tan(bot) * std::tan(bot)) *
                                                    1.0001)
                               : INFINITY;
}

// Frame table entry (float pairs of FP64 sin / cos): per tile row sin/cos of the reference
// elevation theta0, per tile column sin/cos of the reference azimuth gamma0.
struct SinCos2 {
    float s_hi, s_lo, c_hi, c_lo;
};

// Pixel ray planes of one pixel in its tile's frame (FP64 values as float pairs): h_x, h_y
// (hi parts and the remainders) and the ray direction v (hi only).  One entry per (view, tile
// row, pixel of the tile), 64 bytes.
struct PixFrame {
    float hx[3], hy[3], v[3];
    float hx_lo[3], hy_lo[3];
    float pad;
};
static_assert(sizeof(PixFrame) == 64, "PixFrame is 64 bytes");

// Per-tile frame and addressing, computed on the host in FP64 when the views are registered.
// The tile frame Q has rows e1 = v(theta0, gamma0) (the ray through the tile centre),
// e2 = h_x(gamma0), e3 = h_y(theta0, gamma0); M = Q R^c_w and u = Q t^c_w as float pairs,
// R^c_w rounded (normals are produced in the sensor frame).  192 bytes.
struct TileInfo {
    float M_hi[9], M_lo[9];
    float u_hi[3], u_lo[3];
    float R[9];
    int32_t view, tr, tc, cols;      // cols: the view's width (row stride and cyclic period)
    int32_t valid_r, valid_c;        // pixels of this tile inside the image
    int32_t pix_base;                // first PixFrame entry of this tile row
    int64_t out_base;                // packed index of the tile's top-left pixel
    int32_t pad[6];
};
static_assert(sizeof(TileInfo) == 192, "TileInfo is 192 bytes");

// Per (view, primitive) projection record, 16 bytes.
struct PairRec {
    int16_t r0, r1;   // pixel rows [r0, r1]
    int16_t c0, nc;   // cyclic pixel columns [c0, c0 + nc) mod cols
    float kappa;      // binary32 centre range |b_c|
    uint32_t cf;      // bits 0-29: tiles touched; bit 30: normal flipped; bit 31: invalid input
};
static_assert(sizeof(PairRec) == 16, "PairRec is 16 bytes");

enum : uint32_t { kCountMask = 0x3FFFFFFFu, kPairFlip = 1u << 30, kPairInvalid = 1u << 31 };

// ---------------------------------------------------------------------------------------------
// tile geometry shared by the binning and the render kernels
// ---------------------------------------------------------------------------------------------

// A pair's pixel rectangle and normal-flip bit in one word: r0 | flip << 15, r1, c0, nc, 16 bits
// each (rows and columns are below 2^15)
__host__ __device__ inline uint64_t pack_pixel_rect(const PairRec &rec)
{
    const uint32_t r0 = static_cast<uint16_t>(rec.r0) | ((rec.cf & kPairFlip) ? 0x8000u : 0u);
    return static_cast<uint64_t>(r0) | static_cast<uint64_t>(static_cast<uint16_t>(rec.r1)) << 16 |
           static_cast<uint64_t>(static_cast<uint16_t>(rec.c0)) << 32 |
           static_cast<uint64_t>(static_cast<uint16_t>(rec.nc)) << 48;
}

__host__ __device__ inline PairRec unpack_pixel_rect(uint64_t w)
{
    PairRec rec;
    rec.r0 = static_cast<int16_t>(w & 0x7FFFu);
    rec.r1 = static_cast<int16_t>((w >> 16) & 0xFFFFu);
    rec.c0 = static_cast<int16_t>((w >> 32) & 0xFFFFu);
    rec.nc = static_cast<int16_t>(w >> 48);
    rec.kappa = 0.0f;
    rec.cf = (w & 0x8000u) ? kPairFlip : 0u;
    return rec;
}

// A pair's tile rectangle in one word: first tile row, tile rows, first tile column, tile columns
// (cyclic modulo the view's tile columns), 16 bits each; every field is below 2^13 for images
// of at most 32,767 rows and columns and tiles of at least 4 pixels a side.
__host__ __device__ inline uint64_t pack_tile_rect(int tr0, int ntr, int tc0, int ntc)
{
    return static_cast<uint64_t>(static_cast<uint16_t>(tr0)) |
           static_cast<uint64_t>(static_cast<uint16_t>(ntr)) << 16 |
           static_cast<uint64_t>(static_cast<uint16_t>(tc0)) << 32 |
           static_cast<uint64_t>(static_cast<uint16_t>(ntc)) << 48;
}

// ---------------------------------------------------------------------------------------------
// float-pair ("double-float") arithmetic, used where the sensor-frame centre of a primitive
// must keep more than 24 bits (the lateral offset of a far splat from a ray).
// ---------------------------------------------------------------------------------------------
struct f2 {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    f2 r;
    two_sum(p, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    f2 r;
    two_sum(s, e, r.h, r.l);
    return r;
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{-a.h, -a.l}; }

// Sum_j M_j x_j + u in float-pair arithmetic, rounded to one float (x exact floats).
__device__ __forceinline__ float f2_dot3_add(f2 m0, f2 m1, f2 m2, float x0, float x1, float x2,
                                             f2 u)
{
    float p0 = __fmul_rn(m0.h, x0), e0 = __fmaf_rn(m0.h, x0, -p0);
    float p1 = __fmul_rn(m1.h, x1), e1 = __fmaf_rn(m1.h, x1, -p1);
    float p2 = __fmul_rn(m2.h, x2), e2 = __fmaf_rn(m2.h, x2, -p2);
    float s1, t1, s2, t2, s3, t3;
    two_sum(p0, p1, s1, t1);
    two_sum(s1, p2, s2, t2);
    two_sum(s2, u.h, s3, t3);
    float err = __fadd_rn(__fadd_rn(e0, e1), e2);
    err = __fadd_rn(err, __fadd_rn(__fadd_rn(t1, t2), t3));
    err = __fmaf_rn(m0.l, x0, err);
    err = __fmaf_rn(m1.l, x1, err);
    err = __fmaf_rn(m2.l, x2, err);
    err = __fadd_rn(err, u.l);
    return __fadd_rn(s3, err);
}

// The same sum returned as a normalised float pair (hi = the rounded sum, lo = the rest).
__device__ __forceinline__ f2 f2_dot3_add2(f2 m0, f2 m1, f2 m2, float x0, float x1, float x2,
                                           f2 u)
{
    float p0 = __fmul_rn(m0.h, x0), e0 = __fmaf_rn(m0.h, x0, -p0);
    float p1 = __fmul_rn(m1.h, x1), e1 = __fmaf_rn(m1.h, x1, -p1);
    float p2 = __fmul_rn(m2.h, x2), e2 = __fmaf_rn(m2.h, x2, -p2);
    float s1, t1, s2, t2, s3, t3;
    two_sum(p0, p1, s1, t1);
    two_sum(s1, p2, s2, t2);
    two_sum(s2, u.h, s3, t3);
    float err = __fadd_rn(__fadd_rn(e0, e1), e2);
    err = __fadd_rn(err, __fadd_rn(__fadd_rn(t1, t2), t3));
    err = __fmaf_rn(m0.l, x0, err);
    err = __fmaf_rn(m1.l, x1, err);
    err = __fmaf_rn(m2.l, x2, err);
    err = __fadd_rn(err, u.l);
    f2 r;
    two_sum(s3, err, r.h, r.l);
    return r;
}

// K7 for one primitive: world-frame accumulators (dL/dmu, dL/do | dL/dt_a, dL/dlog s_a |
// dL/dt_b, dL/dlog s_b | dL/dt_n) -> gradients of (mu, logit), of the unnormalised quaternion
// (through R(q/|q|)) and of the log-scales.
__device__ __forceinline__ void chain_params(const float4 pl, const float4 q, const float4 *wg,
                                             float4 &g_pl, float4 &g_q, float2 &g_ls)
{
    const float4 a0 = wg[0], a1 = wg[1], a2 = wg[2], a3 = wg[3];
    const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    const float rn = rsqrtf(qn2);
    const float w = q.x * rn, x = q.y * rn, y = q.z * rn, z = q.w * rn;
    // G[r][c] = dL/dR[r][c]; column c of R is t_a, t_b, t_n
    const float G00 = a1.x, G10 = a1.y, G20 = a1.z;
    const float G01 = a2.x, G11 = a2.y, G21 = a2.z;
    const float G02 = a3.x, G12 = a3.y, G22 = a3.z;
    const float gw = 2.0f * (z * (G10 - G01) + y * (G02 - G20) + x * (G21 - G12));
    const float gx = 2.0f * (y * (G01 + G10) + z * (G02 + G20) + w * (G21 - G12)) -
                     4.0f * x * (G11 + G22);
    const float gy = 2.0f * (x * (G01 + G10) + w * (G02 - G20) + z * (G12 + G21)) -
                     4.0f * y * (G00 + G22);
    const float gz = 2.0f * (w * (G10 - G01) + x * (G02 + G20) + y * (G12 + G21)) -
                     4.0f * z * (G00 + G11);
    const float dotq = w * gw + x * gx + y * gy + z * gz;
    g_q = make_float4((gw - w * dotq) * rn, (gx - x * dotq) * rn, (gy - y * dotq) * rn,
                      (gz - z * dotq) * rn);
    const float o = 1.0f / (1.0f + __expf(-pl.w));
    g_pl = make_float4(a0.x, a0.y, a0.z, a0.w * o * (1.0f - o));
    g_ls = make_float2(a1.w, a2.w);
}

// ---------------------------------------------------------------------------------------------
// kernel launchers (defined in the .cu files)
// ---------------------------------------------------------------------------------------------
struct Workspace;   // host-side bookkeeping, defined in splat_abi.cu

// trect[p]: the pair's tile rectangle as one word (see pack_tile_rect), 0 when it touches none;
// prect[p]: its pixel rectangle and normal-flip bit (pack_pixel_rect)
// Record the text of a failed CUDA call for splat_last_cuda_error (thread-local) and return
// SPLAT_ERR_CUDA.
int cuda_fail(cudaError_t e, const char *what);

cudaError_t launch_project(const float4 *pos_logit, const float4 *quat, const float2 *log_scale,
                           int64_t n, const ViewDesc *views, int n_views, float sigma,
                           float alpha_min, int tile_h, int tile_w, int flip_normals,
                           PairRec *recs, uint32_t *dkeys, uint32_t *dvals, uint64_t *trect,
                           uint64_t *prect, float4 *prim, uint32_t *status, uint32_t *n_valid,
                           cudaStream_t st, const uint8_t *active = nullptr);

// stable LSD radix sort of (uint32 key, uint32 value) pairs on key bits [0, bits);
// the count is read on the device from *d_count (clamped to max_n); result lands in
// (keys_out, vals_out).  tmp_hist holds kHistWords uint32.
constexpr int kSortGrid = 608;    // 4 CTAs per SM (152 SMs)
constexpr int kSortTile = 2048;   // keys per CTA tile (256 threads x 8)
constexpr int kHistWords = kSortGrid * 256 + 256;   // per-CTA digit counts + digit totals
// With d_count_kept non-null the first pass also drops every item whose key is 0xFFFFFFFF (which
// would sort last) and the later passes sort the d_count_kept items left, which the caller has
// counted beforehand.
// With aux_out non-null the last pass also writes aux_out[i] = aux_in[value of sorted item i]:
// a copy of per-value data in sorted order, so that the stages after the sort read it in order.
cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                             const uint32_t *d_count, int64_t max_n, int bits, uint32_t *tmp_hist,
                             uint32_t **keys_out, uint32_t **vals_out, cudaStream_t st,
                             const uint32_t *d_count_kept = nullptr,
                             const uint64_t *aux_in = nullptr, uint64_t *aux_out = nullptr);

// offsets of every sorted pair, emission of (global tile, pair id) entries, total pair count
// emission grid: CTAs over the sorted pairs (measured on GB300: 1024 -> 4096 CTAs took the
// three emission kernels from 0.142 to 0.131 ms on 4 M pairs); the CTA-sum scan runs in one CTA
// of 1024 threads, kScanGrid / 1024 sums per thread
constexpr int kScanGrid = 4096;
// tile-ranges grid (grid-stride over the list entries): 6 CTAs per SM measured fastest
// (0.089 ms on 6.1 M entries, against 0.113 ms with 16 per SM)
constexpr int kRangesGrid = 912;
// n_valid: device count of the leading sorted pairs that touch a tile (the rest touch none)
// sorted_trect[j]: the tile rectangle of sorted pair j (the range sort's copy of trect)
cudaError_t launch_emit(const uint32_t *sorted_pair_ids, const uint64_t *sorted_trect,
                        int64_t n_pairs_total, const uint32_t *n_valid, const ViewDesc *views,
                        int64_t n_per_view, uint32_t *block_sums, uint32_t *tile_keys,
                        uint32_t *tile_vals, int64_t max_pairs, uint32_t *d_count,
                        uint32_t *status, cudaStream_t st);

// Pixel rectangle of a (view, primitive) record inside tile (tr, tc) of a tile_h x tile_w
// tiling, packed as 4 bytes (r_lo, r_hi, c_lo, c_hi) with the record's normal-flip bit in bit 31;
// the record's columns are cyclic modulo the image width cols.  0xFF (r_lo > r_hi) when empty.
constexpr uint32_t kRectFlip = 0x80000000u;

__device__ __forceinline__ uint32_t tile_local_rect(const PairRec &rec, int tr, int tc, int cols,
                                                    int tile_h, int tile_w)
{
    const int rb = tr * tile_h, cb = tc * tile_w;
    int r_lo = rec.r0 - rb, r_hi = rec.r1 - rb;
    r_lo = r_lo < 0 ? 0 : r_lo;
    r_hi = r_hi > tile_h - 1 ? tile_h - 1 : r_hi;
    if (r_lo > r_hi) return 0xFFu;
    const int W = cols, nc = rec.nc;
    int c_lo, c_hi;
    if (nc >= W) {
        c_lo = 0;
        c_hi = tile_w - 1;
    } else {
        int d = cb - rec.c0;     // tile start relative to the range start, in [0, W)
        d += d < 0 ? W : 0;
        int e = rec.c0 - cb;     // range start relative to the tile start, in [0, W)
        e += e < 0 ? W : 0;
        const bool start_in = d < nc;
        const bool begins_here = e < tile_w;
        if (start_in && begins_here && d != 0) {   // both ends of a wrapping range meet here
            c_lo = 0;
            c_hi = tile_w - 1;
        } else if (start_in) {
            c_lo = 0;
            c_hi = nc - 1 - d;
            c_hi = c_hi > tile_w - 1 ? tile_w - 1 : c_hi;
        } else if (begins_here) {
            c_lo = e;
            c_hi = e + nc - 1;
            c_hi = c_hi > tile_w - 1 ? tile_w - 1 : c_hi;
        } else {
            return 0xFFu;
        }
    }
    return static_cast<uint32_t>(r_lo) | (static_cast<uint32_t>(r_hi) << 8) |
           (static_cast<uint32_t>(c_lo) << 16) | (static_cast<uint32_t>(c_hi) << 24) |
           ((rec.cf & kPairFlip) ? kRectFlip : 0u);
}

// Which of a tile's 4 x 8 pixel blocks (bit (row block) * tile_w / 8 + column block) a rectangle
// inside the tile (tile_local_rect) meets.
__device__ __forceinline__ uint32_t rect_blocks(uint32_t rect, int tile_h, int tile_w)
{
    const int r_lo = rect & 0xFF, r_hi = (rect >> 8) & 0xFF;
    const int c_lo = (rect >> 16) & 0x3F, c_hi = (rect >> 24) & 0x3F;
    if (r_lo > r_hi || r_hi >= tile_h) return 0u;
    const int wc = tile_w / 8;
    const uint32_t cols = ((2u << (c_hi >> 3)) - 1u) & ~((1u << (c_lo >> 3)) - 1u);
    uint32_t m = 0u;
    for (int rb = r_lo >> 2; rb <= r_hi >> 2; ++rb) m |= cols << (rb * wc);
    return m;
}

// K4: [start, end) per tile from the sorted tile ids, and every list entry's pixel rectangle
// inside its tile (tile_local_rect) in entry_rect and the 4 x 8 blocks it meets (rect_blocks) in
// entry_blocks
cudaError_t launch_ranges(const uint32_t *tile_keys, const uint32_t *tile_vals,
                          const uint64_t *prect, const TileInfo *tiles, int tile_h, int tile_w,
                          const uint32_t *d_count, int64_t max_pairs, uint2 *ranges,
                          int64_t n_tiles, uint32_t *entry_rect, uint8_t *entry_blocks,
                          cudaStream_t st);

// tiles ordered by decreasing log2 of their list length (order inside a bucket unspecified)
cudaError_t launch_order_tiles(const uint2 *ranges, int64_t n_tiles, uint32_t *order,
                               cudaStream_t st);

struct RenderArgs {
    const float4 *pos_logit;      // per primitive: centre (the opacity logit is not read)
    // per primitive, written by the projection: (s_a t_a, o), (s_b t_b, 0), (t_n, 0) -- the
    // scaled tangent axes, the normal and the opacity in the world frame
    const float4 *prim;
    int64_t n;                    // primitives per view (pair id = view * n + i)
    const TileInfo *tiles;        // global tile -> frame and addressing
    const PixFrame *pixframes;
    const uint2 *ranges;          // global tile -> [start, end)
    const uint32_t *tile_order;   // tiles in decreasing order of list length (work order)
    const uint32_t *sorted_vals;  // pair ids in (tile, range, id) order
    const uint32_t *entry_rect;   // per list entry: pixel rectangle inside its tile, flip bit
    const uint8_t *entry_blocks;  // per list entry: the 4 x 8 blocks of its tile it meets
    int64_t n_tiles;
    int64_t n_items;              // n_tiles x blocks per tile
    float alpha_min, alpha_max, t_min, sigma;
    // forward outputs (packed pixels)
    float *depth, *normal, *alpha;
    int64_t n_pixels;
    float *t_final;
    int32_t *n_last;
    // backward inputs / outputs
    const float *g_depth, *g_normal, *g_alpha;
    float4 *wgrad;                // per primitive 4 x float4 (world-frame accumulators)
    float *pose_grad;             // per view (dL/drho, dL/domega), or null
    uint32_t *queue;              // work counter (zeroed before each launch)
    // contributor records (forward writes, backward reads; see splat_render.cu)
    uint2 *rec;                   // pool of 32-record chunks, or null (no records)
    uint32_t *rec_prev;           // per chunk: the item's previous chunk
    uint32_t *rec_alloc;          // chunks taken (zeroed before the forward)
    uint32_t rec_cap;             // chunks in the pool
    uint32_t *rec_head, *rec_fill;   // per work item: last chunk and its fill
    uint32_t *status;             // status bits
    unsigned long long *evals;    // evaluation counter
};

cudaError_t launch_render_fwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st);
cudaError_t launch_render_bwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st);
int render_occupancy(int tile_h, int tile_w, bool backward);

cudaError_t launch_param_grads(const float4 *pos_logit, const float4 *quat, const float2 *log_scale,
                               const float4 *wgrad, int64_t n, float4 *g_pos_logit, float4 *g_quat,
                               float2 *g_log_scale, int accumulate, cudaStream_t st);

// active (nullable): pixels of views with active[v] == 0 count as invalid (views: the registered
// views, for the pixel -> view lookup).  normal_mode 0: normal term against t_normal; 1:
// self-regularised against the normals of the rendered range map (needs views; t_normal unused)
cudaError_t launch_loss(const float *depth, const float *normal, const float *alpha,
                        const float *t_depth, const float *t_normal, int64_t n_pixels,
                        float lambda_n, float lambda_o, float o_eps, float rho_exp,
                        float *g_depth, float *g_normal, float *g_alpha, double *loss_out,
                        cudaStream_t st, const ViewDesc *views = nullptr, int n_views = 0,
                        const uint8_t *active = nullptr, int normal_mode = 0);

struct AdamArgs {
    float4 *pos_logit;
    float4 *quat;
    float2 *log_scale;
    float4 *m_pl, *m_q;
    float2 *m_ls;
    float4 *v_pl, *v_q;
    float2 *v_ls;
    int32_t *step;
    int64_t n;
    float lr_pos, lr_opacity, lr_rot, lr_scale, beta1, beta2, eps;
    // scale term (fused form only): lambda_s max(0, max(s_a, s_b) - tau_s), added to *loss_out
    float lambda_s, tau_s;
    double *loss_out;
};

// Adam from explicit parameter gradients
cudaError_t launch_adam(const AdamArgs &a, const float4 *g_pl, const float4 *g_q,
                        const float2 *g_ls, cudaStream_t st);
// Adam with the chain rule from the world-frame accumulators fused in
cudaError_t launch_adam_fused(const AdamArgs &a, const float4 *wgrad, cudaStream_t st);
cudaError_t launch_step_inc(int32_t *step, cudaStream_t st);

}  // namespace splat
