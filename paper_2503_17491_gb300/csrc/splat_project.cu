// K1: per-primitive projection for every registered view -- the range key, the sign that turns
// the normal towards the sensor, and the conservative spherical bounding box of the region of the
// 3-sigma box where the primitive can reach alpha_min, with its tile rectangle (Sec. 3.2.1 tiles and range sort; Sec. 3.2.3 bounding
// box computation; Supp. B).
//
// Everything in this file takes integer decisions (which tiles, which order, which sign), so it
// follows a fixed binary32 contract: every value is produced by the same sequence of correctly
// rounded IEEE operations on every machine.  The file is compiled with -fmad=false so that no
// a*b+c is fused; fused multiply-adds appear only where written as fmaf.  The arctangent and
// exponential and logarithm used by the contract are evaluated from their series (see
// contract_atan2, contract_exp, contract_log), never through a math library.
//
// One thread per primitive reads its 40 bytes once (coalesced float4/float2 loads) and loops
// over the views; each (view, primitive) record is 16 bytes, plus one 8-byte word with the
// pair's tile rectangle that the range sort lays out in range order for the emission.  The
// range-sort keys and pair ids are written here too, so the sort starts from this kernel's
// output.  Each primitive also gets the 48 bytes the compositing kernels stage for it -- its
// scaled tangent axes, normal and opacity in the world frame -- so that they need not redo the
// quaternion and exponentials for every (block, list entry).

#include <cmath>

#include "splat_internal.cuh"

namespace splat {
namespace {

constexpr float kPi = 3.14159274f;      // nearest binary32 values
constexpr float kHalfPi = 1.57079637f;
constexpr float kTwoPi = 6.28318548f;
constexpr float kQuarterPi = 0.785398163f;
constexpr float kTanPi8 = 0.414213562f;
constexpr float kPixelMargin = 0.01f;   // pixel units, both axes

// atan2 from the arctangent series: reduce to t = min/max in [0, 1], fold t > tan(pi/8) with
// atan t = pi/4 + atan((t - 1)/(t + 1)), then z - z^3/3 + ... + z^17/17 on |z| <= tan(pi/8).
__device__ float contract_atan2(float y, float x)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float hi = ax > ay ? ax : ay;
    const float lo = ax > ay ? ay : ax;
    if (hi == 0.0f) return 0.0f;
    const float t = lo / hi;
    float z, base;
    if (t > kTanPi8) {
        z = (t - 1.0f) / (t + 1.0f);
        base = kQuarterPi;
    } else {
        z = t;
        base = 0.0f;
    }
    const float z2 = z * z;
    float p = 0.0588235294f;
    p = fmaf(p, z2, -0.0666666667f);
    p = fmaf(p, z2, 0.0769230769f);
    p = fmaf(p, z2, -0.0909090909f);
    p = fmaf(p, z2, 0.111111111f);
    p = fmaf(p, z2, -0.142857143f);
    p = fmaf(p, z2, 0.2f);
    p = fmaf(p, z2, -0.333333333f);
    p = fmaf(p, z2, 1.0f);
    float a = fmaf(z, p, base);
    if (ay > ax) a = kHalfPi - a;
    if (x < 0.0f) a = kPi - a;
    if (y < 0.0f) a = -a;
    return a;
}

// exp from a Cody-Waite split of ln 2 (2839/4096 plus its binary32 remainder) and the
// exponential series through r^7/7!; 2^k is assembled in the exponent field.
__device__ float contract_exp(float x)
{
    x = x > 80.0f ? 80.0f : x;
    x = x < -80.0f ? -80.0f : x;
    const float k = rintf(x * 1.44269504f);
    const float r = (x - k * 0.693115234375f) - k * 3.19461849e-05f;
    float p = 1.98412698e-04f;
    p = fmaf(p, r, 1.38888889e-03f);
    p = fmaf(p, r, 8.33333333e-03f);
    p = fmaf(p, r, 4.16666667e-02f);
    p = fmaf(p, r, 0.166666667f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    const int ki = static_cast<int>(k);
    return p * __uint_as_float(static_cast<uint32_t>(ki + 127) << 23);
}

// ln for the contract, x >= 1: x = 2^e m with m folded into [1/sqrt2, sqrt2), then
// ln m = 2 atanh z, z = (m - 1)/(m + 1), from the series 2(z + z^3/3 + ... + z^9/9).
__device__ float contract_log(float x)
{
    const uint32_t u = __float_as_uint(x);
    int e = static_cast<int>((u >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((u & 0x7FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) {
        m = m * 0.5f;
        e = e + 1;
    }
    const float z = (m - 1.0f) / (m + 1.0f);
    const float z2 = z * z;
    float p = 0.111111111f;
    p = fmaf(p, z2, 0.142857143f);
    p = fmaf(p, z2, 0.2f);
    p = fmaf(p, z2, 0.333333333f);
    p = fmaf(p, z2, 1.0f);
    return fmaf(static_cast<float>(e), 0.693147182f, 2.0f * z * p);
}

struct v3 {
    float x, y, z;
};

// R v with R row-major, each row summed as ((a + b) + c)
__device__ __forceinline__ v3 rot(const float *R, v3 v)
{
    return v3{(R[0] * v.x + R[1] * v.y) + R[2] * v.z, (R[3] * v.x + R[4] * v.y) + R[5] * v.z,
              (R[6] * v.x + R[7] * v.y) + R[8] * v.z};
}

// keep the higher and the lower of the points seen so far, by elevation atan2(z, r), r >= 0:
// z r' > z' r says that (z, r) lies above (z', r'); the first of equal points stays
__device__ __forceinline__ void elev_candidate(float z, float r, float &zh, float &rh, float &zl,
                                               float &rl, bool &have)
{
    if (!have) {
        zh = z; rh = r; zl = z; rl = r;
        have = true;
        return;
    }
    if (z * rh > zh * r) { zh = z; rh = r; }
    if (z * rl < zl * r) { zl = z; rl = r; }
}

// The view-independent part: the reach radius r_o, the half-side a and the octagon's cut c (in
// units of a) of a primitive with opacity o; false when o stays below alpha_min everywhere.
struct Octagon {
    float a, k, c;
};

__device__ bool contract_octagon(float o, float alpha_min, float sigma, Octagon &oct)
{
    float x = o / alpha_min;
    if (x < 0.999f) return false;
    if (x < 1.0f) x = 1.0f;
    const float ro = sqrtf(2.0f * contract_log(x)) * 1.001f + 0.002f;
    const float a = ro < sigma ? ro : sigma;
    const float k = (1.41421356f * ro) / a;
    // the octagon (|u|, |w| <= 1, |u| + |w| <= k in units of a); when the diamond misses the
    // square's corners (k >= 2) the cut c = 1 repeats each corner, and the repeated vertices give
    // zero-length edges that add nothing
    oct.a = a;
    oct.k = k;
    oct.c = k < 2.0f ? k - 1.0f : 1.0f;
    return true;
}

// Spherical bounding box of the splat-space region where the primitive can contribute: the
// 3-sigma box |s|_inf <= sigma intersected with the disk where o G(s) >= alpha_min, i.e.
// |s| <= r_o = sqrt(2 ln(o / alpha_min)), bounded by |s|_inf <= a = min(sigma, r_o) and the
// diamond |s_a| + |s_b| <= sqrt2 r_o (an octagon when it cuts the corners), r_o widened by
// 0.1 % + 0.002.  The polygon maps to P = b_c + s_a b_alpha + s_b b_beta.  Azimuth: every column
// when the z axis pierces the polygon's xy-shadow, else the extreme vertex azimuths relative to
// the centre direction.  Elevation: the extreme of the vertices and each edge's interior extremum
// (where z / |xy| is stationary along the edge), and the pole the z axis reaches.  Returns the tile count and
// fills the record's pixel rectangle.
__device__ uint32_t contract_bbox(v3 ba, v3 bb, v3 bc, const Octagon &oct, const ViewDesc &vd,
                                  int th_shift, int tw_shift, PairRec &rec, uint64_t &trect)
{
    const float a = oct.a, k = oct.k, c = oct.c;
    const v3 A{a * ba.x, a * ba.y, a * ba.z};
    const v3 B{a * bb.x, a * bb.y, a * bb.z};
    const v3 C = bc;
    const float u[8] = {1.0f, 1.0f, c, -c, -1.0f, -1.0f, -c, c};
    const float w[8] = {-c, c, 1.0f, 1.0f, c, -c, -1.0f, -1.0f};
    v3 P[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        P[i] = v3{(C.x + u[i] * A.x) + w[i] * B.x, (C.y + u[i] * A.y) + w[i] * B.y,
                  (C.z + u[i] * A.z) + w[i] * B.z};

    // does the z axis cross the polygon's xy-shadow?  c + u A + w B = 0 with |u|, |w| <= 1 and
    // |u| + |w| <= k
    const float det = A.x * B.y - A.y * B.x;
    const float cxb = C.x * B.y - C.y * B.x;
    const float axc = A.x * C.y - A.y * C.x;
    const float la = fabsf(A.x) + fabsf(A.y), lb = fabsf(B.x) + fabsf(B.y);
    const float lc = fabsf(C.x) + fabsf(C.y);
    const float tol = 1e-5f * ((la + lb) * ((lc + la) + lb));
    const float adet = fabsf(det);
    const bool axis_in = (fabsf(cxb) <= adet + tol) && (fabsf(axc) <= adet + tol) &&
                         (fabsf(cxb) + fabsf(axc) <= k * adet + 2.0f * tol);
    bool north = false, south = false;
    if (axis_in) {
        if (adet > tol) {
            const float uu = -cxb / det, ww = -axc / det;
            const float zh = (C.z + uu * A.z) + ww * B.z;
            const float tz = 1e-5f * ((fabsf(C.z) + fabsf(A.z)) + fabsf(B.z));
            north = zh > -tz;
            south = zh < tz;
        } else {
            north = south = true;
        }
    }

    // elevation: the highest and the lowest of the vertices and of the edges' interior extrema,
    // ordered by z / |xy| without a division (z_i r_j against z_j r_i); one arctangent each
    float zh = 0.0f, rh = 0.0f, zl = 0.0f, rl = 0.0f;
    bool have = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const v3 p = P[i], q = P[(i + 1) & 7];
        elev_candidate(p.z, sqrtf(p.x * p.x + p.y * p.y), zh, rh, zl, rl, have);
        const v3 d{q.x - p.x, q.y - p.y, q.z - p.z};
        const float pd = p.x * d.x + p.y * d.y;
        const float pp = p.x * p.x + p.y * p.y;
        const float dd = d.x * d.x + d.y * d.y;
        const float num = p.z * pd - d.z * pp;
        const float den = d.z * pd - p.z * dd;
        // the quotient can round into (0, 1) only when num and den are non-zero with one sign
        // and |num| < |den| (a quotient >= 1 rounds to >= 1): testing that first skips the
        // division for most edges and changes no result
        if (den != 0.0f && num != 0.0f && (num > 0.0f) == (den > 0.0f) &&
            fabsf(num) < fabsf(den)) {
            const float lam = num / den;
            if (lam > 0.0f && lam < 1.0f) {
                const v3 X{p.x + lam * d.x, p.y + lam * d.y, p.z + lam * d.z};
                elev_candidate(X.z, sqrtf(X.x * X.x + X.y * X.y), zh, rh, zl, rl, have);
            }
        }
    }
    float el_hi = contract_atan2(zh, rh), el_lo = contract_atan2(zl, rl);
    if (north) el_hi = kHalfPi;
    if (south) el_lo = -kHalfPi;

    const int H = vd.rows, W = vd.cols;
    const float vhi = (vd.elev_max - el_hi) * vd.kr - kPixelMargin;
    const float vlo = (vd.elev_max - el_lo) * vd.kr + kPixelMargin;
    int r0 = static_cast<int>(ceilf(vhi));
    int r1 = static_cast<int>(floorf(vlo));
    r0 = r0 < 0 ? 0 : r0;
    r1 = r1 > H - 1 ? H - 1 : r1;
    if (r0 > r1) return 0u;

    int c0, nc;
    if (axis_in) {
        c0 = 0;
        nc = W;
    } else {
        // the polygon's xy-shadow misses the origin, so it spans less than pi in azimuth: the
        // extreme vertices follow from the signs of cross products, one arctangent each,
        // relative to the centre direction
        const float gc = contract_atan2(C.y, C.x);
        float xmin = P[0].x, ymin = P[0].y, xmax = P[0].x, ymax = P[0].y;
#pragma unroll
        for (int i = 1; i < 8; ++i) {
            if (xmax * P[i].y - ymax * P[i].x > 0.0f) { xmax = P[i].x; ymax = P[i].y; }
            if (xmin * P[i].y - ymin * P[i].x < 0.0f) { xmin = P[i].x; ymin = P[i].y; }
        }
        const float dmax = contract_atan2(C.x * ymax - C.y * xmax, C.x * xmax + C.y * ymax);
        const float dmin = contract_atan2(C.x * ymin - C.y * xmin, C.x * xmin + C.y * ymin);
        const float glo = gc + dmin, ghi = gc + dmax;
        const float kc = static_cast<float>(W) / kTwoPi;
        const float uf = ((kPi - ghi) * kc - 0.5f) - kPixelMargin;
        const float ul = ((kPi - glo) * kc - 0.5f) + kPixelMargin;
        const int cf = static_cast<int>(ceilf(uf));
        const int cl = static_cast<int>(floorf(ul));
        if (cf > cl) return 0u;
        nc = cl - cf + 1;
        if (nc >= W) {
            c0 = 0;
            nc = W;
        } else {
            const int rem = cf % W;   // in (-W, W)
            c0 = rem < 0 ? rem + W : rem;
        }
    }
    // tile columns of the pixel columns c0 .. c0 + nc - 1 (mod W), wrapping past the last tile;
    // tile sides are powers of two and every index here is non-negative, so shifts divide
    int tc0, ntc;
    if (nc >= W) {
        tc0 = 0;
        ntc = vd.tiles_c;
    } else {
        const int cl = c0 + nc - 1;
        const int a = c0 >> tw_shift;
        const int b = cl < W ? cl >> tw_shift : vd.tiles_c + ((cl - W) >> tw_shift);
        tc0 = a;
        ntc = b - a + 1;
        if (ntc >= vd.tiles_c) {
            tc0 = 0;
            ntc = vd.tiles_c;
        }
    }
    rec.r0 = static_cast<int16_t>(r0);
    rec.r1 = static_cast<int16_t>(r1);
    rec.c0 = static_cast<int16_t>(c0);
    rec.nc = static_cast<int16_t>(nc);
    const int ntr = (r1 >> th_shift) - (r0 >> th_shift) + 1;
    trect = pack_tile_rect(r0 >> th_shift, ntr, tc0, ntc);
    return static_cast<uint32_t>(ntr * ntc);
}

__global__ void __launch_bounds__(256) k_project(
    const float4 *__restrict__ pos_logit, const float4 *__restrict__ quat,
    const float2 *__restrict__ log_scale, int64_t n, const ViewDesc *__restrict__ views,
    int n_views, float sigma, float alpha_min, int tile_h, int tile_w, int flip_normals,
    PairRec *__restrict__ recs, uint32_t *__restrict__ dkeys, uint32_t *__restrict__ dvals,
    uint64_t *__restrict__ trect, uint64_t *__restrict__ prect, float4 *__restrict__ prim,
    uint32_t *__restrict__ status, uint32_t *__restrict__ n_valid,
    const uint8_t *__restrict__ active)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int th_shift = __ffs(tile_h) - 1, tw_shift = __ffs(tile_w) - 1;   // powers of two
    const float4 pl = pos_logit[i];
    const float4 q4 = quat[i];
    const float2 ls = log_scale[i];

    bool ok = isfinite(pl.x) && isfinite(pl.y) && isfinite(pl.z) && isfinite(pl.w) &&
              isfinite(q4.x) && isfinite(q4.y) && isfinite(q4.z) && isfinite(q4.w) &&
              isfinite(ls.x) && isfinite(ls.y);
    // C1: normalised quaternion and scales
    float w = q4.x, x = q4.y, y = q4.z, z = q4.w;
    const float qq = ((w * w + x * x) + y * y) + z * z;
    ok = ok && qq > 0.0f && isfinite(qq);
    v3 ta{}, tb{}, tn{};
    float sa = 0.0f, sb = 0.0f, oc = 0.0f;
    Octagon oct{};
    bool opaque = false;   // the opacity reaches alpha_min somewhere
    if (ok) {
        const float r = sqrtf(qq);
        w = w / r;
        x = x / r;
        y = y / r;
        z = z / r;
        // C2: rotation columns
        ta = v3{1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y + w * z), 2.0f * (x * z - w * y)};
        tb = v3{2.0f * (x * y - w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z + w * x)};
        tn = v3{2.0f * (x * z + w * y), 2.0f * (y * z - w * x), 1.0f - 2.0f * (x * x + y * y)};
        sa = contract_exp(ls.x);
        sb = contract_exp(ls.y);
        oc = 1.0f / (1.0f + contract_exp(-pl.w));
        opaque = contract_octagon(oc, alpha_min, sigma, oct);
    } else {
        atomicOr(status, SPLAT_STATUS_NONFINITE);
    }
    // what the compositing kernels stage for every (block, list entry) of this primitive
    prim[3 * i] = make_float4(sa * ta.x, sa * ta.y, sa * ta.z, oc);
    prim[3 * i + 1] = make_float4(sb * tb.x, sb * tb.y, sb * tb.z, 0.0f);
    prim[3 * i + 2] = make_float4(tn.x, tn.y, tn.z, 0.0f);
    const v3 mu{pl.x, pl.y, pl.z};

    uint32_t nv = 0;   // pairs of this primitive that touch a tile
    for (int v = 0; v < n_views; ++v) {
        const ViewDesc &vd = views[v];
        const int64_t p = static_cast<int64_t>(v) * n + i;
        PairRec rec;
        rec.r0 = rec.r1 = rec.c0 = rec.nc = 0;
        rec.kappa = 0.0f;
        rec.cf = ok ? 0u : kPairInvalid;
        uint64_t tr = 0;
        if (ok) {
            // C3: sensor frame with the binary32 T^c_w
            const v3 ra = rot(vd.R_hi, ta), rb = rot(vd.R_hi, tb), rm = rot(vd.R_hi, mu);
            const v3 ba{sa * ra.x, sa * ra.y, sa * ra.z};
            const v3 bb{sb * rb.x, sb * rb.y, sb * rb.z};
            const v3 bc{rm.x + vd.t_hi[0], rm.y + vd.t_hi[1], rm.z + vd.t_hi[2]};
            const v3 nr = rot(vd.R_hi, tn);
            const float dot = (nr.x * bc.x + nr.y * bc.y) + nr.z * bc.z;
            if (flip_normals && dot > 0.0f) rec.cf |= kPairFlip;
            rec.kappa = sqrtf((bc.x * bc.x + bc.y * bc.y) + bc.z * bc.z);
            // A pair whose whole 3-sigma box lies beyond the view's culling cones (two rows past
            // the top or bottom row) and away from the z axis reaches no row: every point of
            // the box is within R = sigma (s_a + s_b) of b_c, and z - t |xy| changes by at most
            // l R over that ball; staying clear of the axis also keeps the polygon's pole tests
            // false.  This skips the polygon for such pairs and changes no result.
            const float rxy = sqrtf(bc.x * bc.x + bc.y * bc.y);
            const float reach = sigma * (sa + sb) * 1.01f;
            const bool clear = rxy * 0.99f - reach > 1e-3f;
            const bool above = bc.z - vd.cull_t_top * rxy > reach * vd.cull_l_top;
            const bool below = vd.cull_t_bot * rxy - bc.z > reach * vd.cull_l_bot;
            // C4: bounding box (views not sampled for this step take no pairs)
            if (opaque && !(clear && (above || below)) && !(active && !active[v]))
                rec.cf |= contract_bbox(ba, bb, bc, oct, vd, th_shift, tw_shift, rec, tr);
        }
        recs[p] = rec;
        trect[p] = (rec.cf & kCountMask) ? tr : 0ull;
        prect[p] = pack_pixel_rect(rec);
        dkeys[p] = (rec.cf & kCountMask) ? __float_as_uint(rec.kappa) : 0xFFFFFFFFu;
        dvals[p] = static_cast<uint32_t>(p);
        nv += (rec.cf & kCountMask) ? 1u : 0u;
    }
    // the number of pairs that touch a tile: after the range sort they lead (the others carry
    // the key 0xFFFFFFFF), so the emission stops there
    const unsigned am = __activemask();
    const unsigned s = __reduce_add_sync(am, nv);
    if ((threadIdx.x & 31) == __ffs(am) - 1 && s) atomicAdd(n_valid, s);
}

}  // namespace

cudaError_t launch_project(const float4 *pos_logit, const float4 *quat, const float2 *log_scale,
                           int64_t n, const ViewDesc *views, int n_views, float sigma,
                           float alpha_min, int tile_h, int tile_w, int flip_normals,
                           PairRec *recs, uint32_t *dkeys, uint32_t *dvals, uint64_t *trect,
                           uint64_t *prect, float4 *prim, uint32_t *status, uint32_t *n_valid,
                           cudaStream_t st, const uint8_t *active)
{
    if (n <= 0) return cudaSuccess;
    const unsigned grid = static_cast<unsigned>((n + 255) / 256);
    k_project<<<grid, 256, 0, st>>>(pos_logit, quat, log_scale, n, views, n_views, sigma,
                                    alpha_min, tile_h, tile_w, flip_normals, recs, dkeys, dvals,
                                    trect, prect, prim, status, n_valid, active);
    return cudaGetLastError();
}

}  // namespace splat
