// K5/K6 (+K10): per-tile front-to-back compositing and its back-to-front adjoint, as persistent
// kernels over a work queue of (view, tile) items, and K7, the chain rule from the per-primitive
// accumulators to the parameters.
//
// One CTA of 256 threads renders one tile of tile_h x tile_w = 256 pixels, one pixel per
// thread.  The tile's primitives (its slice of the sorted list, Sec. 3.2.1) are staged into
// shared memory 256 at a time -- each thread stages one primitive -- and every pixel then runs
// through the batch.
//
// Numerics.  Each pixel ray is intersected with a splat as two planes h_x, h_y through the
// sensor (Sec. 3.2.2, Eq. planes_to_splat; Supp. D.1): h_a = (h_x.b_a, h_x.b_b, h_x.b_c),
// h_b likewise with h_y, p = h_a x h_b, s_hat = (p_x, p_y) / p_z.  The products h.b_c are lateral
// offsets of the splat centre from the ray: a few centimetres out of up to 100 m of range, which
// binary32 sensor-frame vectors cannot resolve (an f32 ulp at 64-128 m is 7.6e-6 m).  So every
// tile gets its own orthonormal frame Q = (e1, e2, e3) -- e1 the ray through the tile centre, e2
// and e3 its two planes -- and a primitive is staged as Q b in that frame, with Q R^c_w and
// Q t^c_w kept as float pairs and the centre Q b_c formed in float-pair arithmetic before it is
// rounded.  Inside the tile frame every pixel ray is within half a tile of e1, so h.b_c is a
// difference of numbers of a few metres, not of a hundred.  The pixel planes in the tile frame
// come from exact small angle offsets (integer pixel offsets times 2 pi / W and the row
// spacing), so no large angle is ever rounded.
//
// The range is d = nu . v (nu lies on the ray, so this equals |nu| without a square root) and
// a hit counts only when d > 0 (in front of the sensor).  The cutoffs follow the 3DGS
// conventions (alpha clamp, alpha_min, stop before T < t_min) plus the 3-sigma box test
// max |s_hat| <= sigma, written as max(|p_x|, |p_y|) <= sigma |p_z| so that misses need no
// division.  A per-(tile, primitive) pixel rectangle from the bounding box skips most misses
// with two integer compares.
//
// Forward and backward evaluate a (pixel, primitive) pair with the same explicitly rounded
// operations (no contraction choices left to the compiler), so the backward replays exactly
// the contributor set of the forward.  The backward recovers T_k = T_{k+1} / (1 - alpha_k) from
// the final transmittance, keeps the suffix sums B_{d,k}, B_{n,k}, B_{o,k} of Supp. D.2, sums
// each primitive's 13 per-pixel terms across the warp with shuffles, then across the CTA in
// shared memory, rotates them back to the world frame once per (tile, primitive) and issues
// four float4 atomics into a per-primitive accumulator (view independent, so gradients of many
// views add up directly).

#include "splat_internal.cuh"

namespace splat {
namespace {

struct __align__(16) Staged {
    float4 a;   // b_alpha' (tile frame), o
    float4 b;   // b_beta' (tile frame), packed pixel rectangle (bits)
    float4 c;   // c' = Q b_c (tile frame), alpha clamp flag unused
    float4 n;   // normal (sensor frame)
};

struct TileFrame {
    f2 M[9];        // Q R^c_w, row-major
    f2 u[3];        // Q t^c_w
    float Mh[9];    // hi parts
    float Rh[9];    // R^c_w hi parts (normals stay in the sensor frame)
    int view;
    int tr, tc;
    int pad_;
};

struct Pix {
    float hx0, hx1, hx2;
    float hy0, hy1, hy2;
    float v0, v1, v2;
};

__device__ __forceinline__ float dot3e(float a0, float a1, float a2, float b0, float b1, float b2)
{
    return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

// tile frame: rows e1 = v(theta0, gamma0), e2 = h_x(gamma0), e3 = h_y(theta0, gamma0)
__device__ void build_frame(const ViewDesc &vd, const SinCos2 *frames, int tr, int tc, int tid,
                            TileFrame &tf)
{
    const SinCos2 rowf = frames[vd.table_offset + tr];
    const SinCos2 colf = frames[vd.table_offset + vd.tiles_r + tc];
    const f2 st{rowf.s_hi, rowf.s_lo}, ct{rowf.c_hi, rowf.c_lo};
    const f2 sg{colf.s_hi, colf.s_lo}, cg{colf.c_hi, colf.c_lo};
    if (tid < 12) {
        const int k = tid < 9 ? tid / 3 : tid - 9;   // row of Q
        f2 q[3];
        if (k == 0) {
            q[0] = f2_mul(ct, cg);
            q[1] = f2_mul(ct, sg);
            q[2] = st;
        } else if (k == 1) {
            q[0] = sg;
            q[1] = f2_neg(cg);
            q[2] = f2{0.0f, 0.0f};
        } else {
            q[0] = f2_neg(f2_mul(st, cg));
            q[1] = f2_neg(f2_mul(st, sg));
            q[2] = ct;
        }
        if (tid < 9) {
            const int j = tid % 3;
            f2 acc{0.0f, 0.0f};
#pragma unroll
            for (int m = 0; m < 3; ++m)
                acc = f2_add(acc, f2_mul(q[m], f2{vd.R_hi[3 * m + j], vd.R_lo[3 * m + j]}));
            tf.M[tid] = acc;
            tf.Mh[tid] = acc.h + acc.l;
        } else {
            f2 acc{0.0f, 0.0f};
#pragma unroll
            for (int m = 0; m < 3; ++m)
                acc = f2_add(acc, f2_mul(q[m], f2{vd.t_hi[m], vd.t_lo[m]}));
            tf.u[k] = acc;
        }
    } else if (tid < 21) {
        tf.Rh[tid - 12] = vd.R_hi[tid - 12];
    }
}

template <int TH, int TW>
__device__ __forceinline__ Pix pixel_frame(const ViewDesc &vd, const SinCos2 *frames, int tr,
                                           int lr, int lc)
{
    const SinCos2 rowf = frames[vd.table_offset + tr];
    const float s0 = rowf.s_hi, c0 = rowf.c_hi;
    const float dlc = static_cast<float>(lc) - 0.5f * static_cast<float>(TW - 1);
    const float dlr = static_cast<float>(lr) - 0.5f * static_cast<float>(TH - 1);
    const float dg = -vd.dgamma * dlc;   // gamma - gamma0
    const float dt = -vd.dtheta * dlr;   // theta - theta0
    float sg, cg, sdt, cdt;
    sincosf(dg, &sg, &cg);
    sincosf(dt, &sdt, &cdt);
    const float sh = sinf(0.5f * dg);
    const float omc = 2.0f * sh * sh;      // 1 - cos(dg) without cancellation
    const float sth = s0 * cdt + c0 * sdt; // sin(theta)
    const float cth = c0 * cdt - s0 * sdt; // cos(theta)
    Pix p;
    p.hx0 = c0 * sg;
    p.hx1 = cg;
    p.hx2 = -s0 * sg;
    p.hy0 = -sdt + c0 * sth * omc;
    p.hy1 = sth * sg;
    p.hy2 = cdt - s0 * sth * omc;
    p.v0 = cdt - c0 * cth * omc;
    p.v1 = -cth * sg;
    p.v2 = sdt + s0 * cth * omc;
    return p;
}

// pixel rectangle of a primitive inside the tile, packed as 4 bytes (r_lo, r_hi, c_lo, c_hi)
template <int TH, int TW>
__device__ __forceinline__ uint32_t local_rect(const PairRec &rec, const ViewDesc &vd, int tr,
                                               int tc)
{
    const int rb = tr * TH, cb = tc * TW;
    int r_lo = rec.r0 - rb, r_hi = rec.r1 - rb;
    r_lo = r_lo < 0 ? 0 : r_lo;
    r_hi = r_hi > TH - 1 ? TH - 1 : r_hi;
    if (r_lo > r_hi) return 0xFFu;   // empty: r_lo = 255 > r_hi = 0
    const int W = vd.cols, nc = rec.nc;
    int c_lo, c_hi;
    if (nc >= W) {
        c_lo = 0;
        c_hi = TW - 1;
    } else {
        const int d = ((cb - rec.c0) % W + W) % W;      // tile start relative to the range start
        const int e = ((rec.c0 - cb) % W + W) % W;      // range start relative to the tile start
        const bool start_in = d < nc;
        const bool begins_here = e < TW;
        if (start_in && begins_here && d != 0) {   // both ends of a wrapping range meet here
            c_lo = 0;
            c_hi = TW - 1;
        } else if (start_in) {
            c_lo = 0;
            c_hi = nc - 1 - d;
            c_hi = c_hi > TW - 1 ? TW - 1 : c_hi;
        } else if (begins_here) {
            c_lo = e;
            c_hi = e + nc - 1;
            c_hi = c_hi > TW - 1 ? TW - 1 : c_hi;
        } else {
            return 0xFFu;
        }
    }
    return static_cast<uint32_t>(r_lo) | (static_cast<uint32_t>(r_hi) << 8) |
           (static_cast<uint32_t>(c_lo) << 16) | (static_cast<uint32_t>(c_hi) << 24);
}

__device__ __forceinline__ bool in_rect(uint32_t rect, int lr, int lc)
{
    const int r_lo = rect & 0xFF, r_hi = (rect >> 8) & 0xFF;
    const int c_lo = (rect >> 16) & 0xFF, c_hi = rect >> 24;
    return lr >= r_lo && lr <= r_hi && lc >= c_lo && lc <= c_hi;
}

struct Prim {
    int64_t i;
    float sa, sb;
    bool flip;
};

// stage pair id p of the current tile into the tile frame
__device__ __forceinline__ void stage(const RenderArgs &A, const TileFrame &tf, uint32_t p,
                                      const PairRec &rec, uint32_t rect, Staged &out, Prim &pr)
{
    const int64_t i = static_cast<int64_t>(p) - static_cast<int64_t>(tf.view) * A.n;
    const float4 pl = A.pos_logit[i];
    const float4 q = A.quat[i];
    const float2 ls = A.log_scale[i];
    const float rn = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * rn, x = q.y * rn, y = q.z * rn, z = q.w * rn;
    const float ta0 = 1.0f - 2.0f * (y * y + z * z), ta1 = 2.0f * (x * y + w * z),
                ta2 = 2.0f * (x * z - w * y);
    const float tb0 = 2.0f * (x * y - w * z), tb1 = 1.0f - 2.0f * (x * x + z * z),
                tb2 = 2.0f * (y * z + w * x);
    const float tn0 = 2.0f * (x * z + w * y), tn1 = 2.0f * (y * z - w * x),
                tn2 = 1.0f - 2.0f * (x * x + y * y);
    const float sa = __expf(ls.x), sb = __expf(ls.y);
    const float o = 1.0f / (1.0f + __expf(-pl.w));
    const float *M = tf.Mh;
    out.a = make_float4(sa * (M[0] * ta0 + M[1] * ta1 + M[2] * ta2),
                        sa * (M[3] * ta0 + M[4] * ta1 + M[5] * ta2),
                        sa * (M[6] * ta0 + M[7] * ta1 + M[8] * ta2), o);
    out.b = make_float4(sb * (M[0] * tb0 + M[1] * tb1 + M[2] * tb2),
                        sb * (M[3] * tb0 + M[4] * tb1 + M[5] * tb2),
                        sb * (M[6] * tb0 + M[7] * tb1 + M[8] * tb2), __uint_as_float(rect));
    out.c = make_float4(f2_dot3_add(tf.M[0], tf.M[1], tf.M[2], pl.x, pl.y, pl.z, tf.u[0]),
                        f2_dot3_add(tf.M[3], tf.M[4], tf.M[5], pl.x, pl.y, pl.z, tf.u[1]),
                        f2_dot3_add(tf.M[6], tf.M[7], tf.M[8], pl.x, pl.y, pl.z, tf.u[2]), 0.0f);
    const float *R = tf.Rh;
    const float fs = (rec.cf & kPairFlip) ? -1.0f : 1.0f;
    out.n = make_float4(fs * (R[0] * tn0 + R[1] * tn1 + R[2] * tn2),
                        fs * (R[3] * tn0 + R[4] * tn1 + R[5] * tn2),
                        fs * (R[6] * tn0 + R[7] * tn1 + R[8] * tn2), 0.0f);
    pr.i = i;
    pr.sa = sa;
    pr.sb = sb;
    pr.flip = (rec.cf & kPairFlip) != 0;
}

struct Hit {
    float ha0, ha1, ha2, hb0, hb1, hb2;
    float pz, px, py, inv, sa, sb, G, a, d;
    bool clamped;
};

// the per-pair test and geometry, identical in forward and backward
__device__ __forceinline__ bool evaluate(const Staged &s, const Pix &px, float sigma,
                                         float amin, float amax, Hit &h)
{
    h.ha0 = dot3e(px.hx0, px.hx1, px.hx2, s.a.x, s.a.y, s.a.z);
    h.ha1 = dot3e(px.hx0, px.hx1, px.hx2, s.b.x, s.b.y, s.b.z);
    h.ha2 = dot3e(px.hx0, px.hx1, px.hx2, s.c.x, s.c.y, s.c.z);
    h.hb0 = dot3e(px.hy0, px.hy1, px.hy2, s.a.x, s.a.y, s.a.z);
    h.hb1 = dot3e(px.hy0, px.hy1, px.hy2, s.b.x, s.b.y, s.b.z);
    h.hb2 = dot3e(px.hy0, px.hy1, px.hy2, s.c.x, s.c.y, s.c.z);
    h.pz = __fmaf_rn(h.ha0, h.hb1, -__fmul_rn(h.ha1, h.hb0));
    h.px = __fmaf_rn(h.ha1, h.hb2, -__fmul_rn(h.ha2, h.hb1));
    h.py = __fmaf_rn(h.ha2, h.hb0, -__fmul_rn(h.ha0, h.hb2));
    const float apz = fabsf(h.pz);
    if (!(apz > 0.0f) || !(fmaxf(fabsf(h.px), fabsf(h.py)) <= __fmul_rn(sigma, apz))) return false;
    h.inv = __frcp_rn(h.pz);
    h.sa = __fmul_rn(h.px, h.inv);
    h.sb = __fmul_rn(h.py, h.inv);
    const float r2 = __fmaf_rn(h.sa, h.sa, __fmul_rn(h.sb, h.sb));
    h.G = __expf(__fmul_rn(-0.5f, r2));
    const float oG = __fmul_rn(s.a.w, h.G);
    h.clamped = oG > amax;
    h.a = h.clamped ? amax : oG;
    if (h.a < amin) return false;
    const float nu0 = __fmaf_rn(h.sa, s.a.x, __fmaf_rn(h.sb, s.b.x, s.c.x));
    const float nu1 = __fmaf_rn(h.sa, s.a.y, __fmaf_rn(h.sb, s.b.y, s.c.y));
    const float nu2 = __fmaf_rn(h.sa, s.a.z, __fmaf_rn(h.sb, s.b.z, s.c.z));
    h.d = dot3e(nu0, nu1, nu2, px.v0, px.v1, px.v2);
    return h.d > 0.0f;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long *s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBlock / 32; ++w) t += s_red[w];
    return t;
}

// ---------------------------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------------------------
template <int TH, int TW>
__global__ void __launch_bounds__(kBlock, 3) k_render_fwd(const RenderArgs A)
{
    static_assert(TH * TW == kBlock, "one pixel per thread");
    __shared__ Staged s_st[kBlock];
    __shared__ TileFrame s_tf;
    __shared__ int64_t s_tile;
    __shared__ unsigned long long s_red[kBlock / 32];
    const int tid = threadIdx.x;
    const int lr = tid / TW, lc = tid % TW;
    unsigned long long evals = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(A.queue, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= A.n_tiles) break;
        const int v = A.tile_view[tile];
        const ViewDesc &vd = A.views[v];
        const int lt = static_cast<int>(tile - vd.tile_offset);
        const int tr = lt / vd.tiles_c, tc = lt - tr * vd.tiles_c;
        build_frame(vd, A.frames, tr, tc, tid, s_tf);
        if (tid == 0) {
            s_tf.view = v;
            s_tf.tr = tr;
            s_tf.tc = tc;
        }
        const int r = tr * TH + lr, c = tc * TW + lc;
        const bool inside = r < vd.rows && c < vd.cols;
        const Pix px = pixel_frame<TH, TW>(vd, A.frames, tr, lr, lc);
        const uint2 rg = A.ranges[tile];
        const int len = static_cast<int>(rg.y - rg.x);
        float T = 1.0f, D = 0.0f, N0 = 0.0f, N1 = 0.0f, N2 = 0.0f, O = 0.0f;
        int last = 0;
        bool done = !inside;
        __syncthreads();   // frame ready

        for (int bs = 0; bs < len; bs += kBlock) {
            if (__syncthreads_count(done ? 0 : 1) == 0) break;
            if (bs + tid < len) {
                const uint32_t p = A.sorted_vals[rg.x + bs + tid];
                const PairRec rec = A.recs[p];
                Prim pr;
                stage(A, s_tf, p, rec, local_rect<TH, TW>(rec, vd, tr, tc), s_st[tid], pr);
            }
            __syncthreads();
            if (!done) {
                const int nb = len - bs < kBlock ? len - bs : kBlock;
                for (int k = 0; k < nb; ++k) {
                    const Staged &s = s_st[k];
                    if (!in_rect(__float_as_uint(s.b.w), lr, lc)) continue;
                    ++evals;
                    Hit h;
                    if (!evaluate(s, px, A.sigma, A.alpha_min, A.alpha_max, h)) continue;
                    const float tt = __fmul_rn(T, __fsub_rn(1.0f, h.a));
                    if (tt < A.t_min) {
                        done = true;
                        break;
                    }
                    const float w = __fmul_rn(h.a, T);
                    D = __fmaf_rn(w, h.d, D);
                    const float4 nn = s.n;
                    N0 = __fmaf_rn(w, nn.x, N0);
                    N1 = __fmaf_rn(w, nn.y, N1);
                    N2 = __fmaf_rn(w, nn.z, N2);
                    O = __fadd_rn(O, w);
                    T = tt;
                    last = bs + k + 1;
                }
            }
        }
        if (inside) {
            const int64_t pix = vd.pixel_offset + static_cast<int64_t>(r) * vd.cols + c;
            A.depth[pix] = D;
            A.normal[pix] = N0;
            A.normal[A.n_pixels + pix] = N1;
            A.normal[2 * A.n_pixels + pix] = N2;
            A.alpha[pix] = O;
            A.t_final[pix] = T;
            A.n_last[pix] = last;
        }
    }
    const unsigned long long tot = block_sum_u64(evals, s_red);
    if (tid == 0 && tot) atomicAdd(A.evals, tot);
}

// ---------------------------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------------------------
constexpr int kAcc = 16;   // per staged primitive: g_ba'(3) g_bb'(3) g_c'(3) g_n(3) g_o, pad

template <int TH, int TW>
__global__ void __launch_bounds__(kBlock, 2) k_render_bwd(const RenderArgs A)
{
    __shared__ Staged s_st[kBlock];
    __shared__ float s_acc[kBlock][kAcc];
    __shared__ TileFrame s_tf;
    __shared__ int64_t s_tile;
    __shared__ int s_maxlast;
    __shared__ unsigned long long s_red[kBlock / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    const int lr = tid / TW, lc = tid % TW;
    unsigned long long evals = 0;

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            s_tile = atomicAdd(A.queue, 1u);
            s_maxlast = 0;
        }
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= A.n_tiles) break;
        const int v = A.tile_view[tile];
        const ViewDesc &vd = A.views[v];
        const int lt = static_cast<int>(tile - vd.tile_offset);
        const int tr = lt / vd.tiles_c, tc = lt - tr * vd.tiles_c;
        build_frame(vd, A.frames, tr, tc, tid, s_tf);
        if (tid == 0) {
            s_tf.view = v;
            s_tf.tr = tr;
            s_tf.tc = tc;
        }
        const int r = tr * TH + lr, c = tc * TW + lc;
        const bool inside = r < vd.rows && c < vd.cols;
        const Pix px = pixel_frame<TH, TW>(vd, A.frames, tr, lr, lc);
        const uint2 rg = A.ranges[tile];
        float T = 1.0f, gD = 0.0f, gN0 = 0.0f, gN1 = 0.0f, gN2 = 0.0f, gO = 0.0f;
        int nl = 0;
        if (inside) {
            const int64_t pix = vd.pixel_offset + static_cast<int64_t>(r) * vd.cols + c;
            T = A.t_final[pix];
            nl = A.n_last[pix];
            if (A.g_depth) gD = A.g_depth[pix];
            if (A.g_normal) {
                gN0 = A.g_normal[pix];
                gN1 = A.g_normal[A.n_pixels + pix];
                gN2 = A.g_normal[2 * A.n_pixels + pix];
            }
            if (A.g_alpha) gO = A.g_alpha[pix];
            if (nl > 0) atomicMax(&s_maxlast, nl);
        }
        float Bd = 0.0f, Bo = 0.0f, Bn0 = 0.0f, Bn1 = 0.0f, Bn2 = 0.0f;
        __syncthreads();   // frame and s_maxlast ready
        const int maxlast = s_maxlast;

        for (int be = maxlast; be > 0; be -= kBlock) {
            const int bs = be - kBlock > 0 ? be - kBlock : 0;
            __syncthreads();
            Prim pr;
            pr.i = -1;
            if (bs + tid < be) {
                const uint32_t p = A.sorted_vals[rg.x + bs + tid];
                const PairRec rec = A.recs[p];
                stage(A, s_tf, p, rec, local_rect<TH, TW>(rec, vd, tr, tc), s_st[tid], pr);
            }
#pragma unroll
            for (int j = 0; j < kAcc; ++j) s_acc[tid][j] = 0.0f;
            __syncthreads();
            for (int k = be - 1; k >= bs; --k) {
                const Staged &s = s_st[k - bs];
                float g[13];
#pragma unroll
                for (int j = 0; j < 13; ++j) g[j] = 0.0f;
                bool contrib = false;
                if (k < nl && in_rect(__float_as_uint(s.b.w), lr, lc)) {
                    ++evals;
                    Hit h;
                    if (evaluate(s, px, A.sigma, A.alpha_min, A.alpha_max, h)) {
                        contrib = true;
                        const float om = __fsub_rn(1.0f, h.a);
                        const float Tk = __fdiv_rn(T, om);
                        const float w = __fmul_rn(h.a, Tk);
                        const float inv_om = __frcp_rn(om);
                        const float4 nn = s.n;
                        // dL/dalpha_k = sum_ch g_ch (x_k A_k - B_ch,k / (1 - alpha_k))
                        float gA = gD * (h.d * Tk - Bd * inv_om);
                        gA += gO * (Tk - Bo * inv_om);
                        gA += gN0 * (nn.x * Tk - Bn0 * inv_om);
                        gA += gN1 * (nn.y * Tk - Bn1 * inv_om);
                        gA += gN2 * (nn.z * Tk - Bn2 * inv_om);
                        Bd += w * h.d;
                        Bo += w;
                        Bn0 += w * nn.x;
                        Bn1 += w * nn.y;
                        Bn2 += w * nn.z;
                        T = Tk;
                        const float gd = gD * w;          // dL/dd_k
                        g[9] = gN0 * w;                    // dL/dn_k
                        g[10] = gN1 * w;
                        g[11] = gN2 * w;
                        const float gAe = h.clamped ? 0.0f : gA;
                        g[12] = gAe * h.G;                 // dL/do
                        // dL/ds_hat: density term and range term (d = nu . v)
                        const float vba = px.v0 * s.a.x + px.v1 * s.a.y + px.v2 * s.a.z;
                        const float vbb = px.v0 * s.b.x + px.v1 * s.b.y + px.v2 * s.b.z;
                        const float gsa = -gAe * h.a * h.sa + gd * vba;
                        const float gsb = -gAe * h.a * h.sb + gd * vbb;
                        // dL/dp_hat with s_hat = (p_x, p_y) / p_z
                        const float gp0 = gsa * h.inv, gp1 = gsb * h.inv;
                        const float gp2 = -(h.sa * gsa + h.sb * gsb) * h.inv;
                        // rho_a = g_p x h_a = dL/dh_b ; rho_b = g_p x h_b = -dL/dh_a
                        const float ra0 = gp1 * h.ha2 - gp2 * h.ha1;
                        const float ra1 = gp2 * h.ha0 - gp0 * h.ha2;
                        const float ra2 = gp0 * h.ha1 - gp1 * h.ha0;
                        const float rb0 = gp1 * h.hb2 - gp2 * h.hb1;
                        const float rb1 = gp2 * h.hb0 - gp0 * h.hb2;
                        const float rb2 = gp0 * h.hb1 - gp1 * h.hb0;
                        const float t0 = gd * h.sa, t1 = gd * h.sb;
                        g[0] = -rb0 * px.hx0 + ra0 * px.hy0 + t0 * px.v0;
                        g[1] = -rb0 * px.hx1 + ra0 * px.hy1 + t0 * px.v1;
                        g[2] = -rb0 * px.hx2 + ra0 * px.hy2 + t0 * px.v2;
                        g[3] = -rb1 * px.hx0 + ra1 * px.hy0 + t1 * px.v0;
                        g[4] = -rb1 * px.hx1 + ra1 * px.hy1 + t1 * px.v1;
                        g[5] = -rb1 * px.hx2 + ra1 * px.hy2 + t1 * px.v2;
                        g[6] = -rb2 * px.hx0 + ra2 * px.hy0 + gd * px.v0;
                        g[7] = -rb2 * px.hx1 + ra2 * px.hy1 + gd * px.v1;
                        g[8] = -rb2 * px.hx2 + ra2 * px.hy2 + gd * px.v2;
                    }
                }
                if (__any_sync(0xFFFFFFFFu, contrib)) {
#pragma unroll
                    for (int j = 0; j < 13; ++j) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1)
                            g[j] += __shfl_xor_sync(0xFFFFFFFFu, g[j], o);
                    }
                    if (lane == 0) {
#pragma unroll
                        for (int j = 0; j < 13; ++j) atomicAdd(&s_acc[k - bs][j], g[j]);
                    }
                }
            }
            __syncthreads();
            if (pr.i >= 0) {
                const float *a = s_acc[tid];
                bool any = false;
#pragma unroll
                for (int j = 0; j < 13; ++j) any |= a[j] != 0.0f;
                if (any) {
                    const float *M = s_tf.Mh;
                    const float *R = s_tf.Rh;
                    const Staged &s = s_st[tid];
                    // world frame: M^T g' (M = Q R^c_w), normals: R^c_w^T g_n
                    float gmu[3], gta[3], gtb[3], gtn[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        gmu[j] = M[j] * a[6] + M[3 + j] * a[7] + M[6 + j] * a[8];
                        gta[j] = pr.sa * (M[j] * a[0] + M[3 + j] * a[1] + M[6 + j] * a[2]);
                        gtb[j] = pr.sb * (M[j] * a[3] + M[3 + j] * a[4] + M[6 + j] * a[5]);
                        gtn[j] = R[j] * a[9] + R[3 + j] * a[10] + R[6 + j] * a[11];
                        if (pr.flip) gtn[j] = -gtn[j];
                    }
                    const float gls_a = a[0] * s.a.x + a[1] * s.a.y + a[2] * s.a.z;
                    const float gls_b = a[3] * s.b.x + a[4] * s.b.y + a[5] * s.b.z;
                    float4 *dst = A.wgrad + 4 * pr.i;
                    atomicAdd(dst + 0, make_float4(gmu[0], gmu[1], gmu[2], a[12]));
                    atomicAdd(dst + 1, make_float4(gta[0], gta[1], gta[2], gls_a));
                    atomicAdd(dst + 2, make_float4(gtb[0], gtb[1], gtb[2], gls_b));
                    atomicAdd(dst + 3, make_float4(gtn[0], gtn[1], gtn[2], 0.0f));
                }
            }
        }
    }
    const unsigned long long tot = block_sum_u64(evals, s_red);
    if (tid == 0 && tot) atomicAdd(A.evals, tot);
}

// ---------------------------------------------------------------------------------------------
// K7: world-frame accumulators -> parameter gradients
// ---------------------------------------------------------------------------------------------
__global__ void k_param_grads(const float4 *__restrict__ pos_logit, const float4 *__restrict__ quat,
                              const float4 *__restrict__ wgrad, int64_t n,
                              float4 *__restrict__ g_pl, float4 *__restrict__ g_q,
                              float2 *__restrict__ g_ls, int accumulate)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a, b;
    float2 c;
    chain_params(pos_logit[i], quat[i], wgrad + 4 * i, a, b, c);
    if (accumulate) {
        const float4 a0 = g_pl[i], b0 = g_q[i];
        const float2 c0 = g_ls[i];
        a = make_float4(a.x + a0.x, a.y + a0.y, a.z + a0.z, a.w + a0.w);
        b = make_float4(b.x + b0.x, b.y + b0.y, b.z + b0.z, b.w + b0.w);
        c = make_float2(c.x + c0.x, c.y + c0.y);
    }
    g_pl[i] = a;
    g_q[i] = b;
    g_ls[i] = c;
}

template <typename K>
cudaError_t dispatch(int th, int tw, K k)
{
    if (th == 16 && tw == 16) return k(std::integral_constant<int, 16>{}, std::integral_constant<int, 16>{});
    if (th == 8 && tw == 32) return k(std::integral_constant<int, 8>{}, std::integral_constant<int, 32>{});
    if (th == 32 && tw == 8) return k(std::integral_constant<int, 32>{}, std::integral_constant<int, 8>{});
    if (th == 4 && tw == 64) return k(std::integral_constant<int, 4>{}, std::integral_constant<int, 64>{});
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_render_fwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st)
{
    return dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        k_render_fwd<decltype(TH)::value, decltype(TW)::value><<<grid, kBlock, 0, st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_render_bwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st)
{
    return dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        k_render_bwd<decltype(TH)::value, decltype(TW)::value><<<grid, kBlock, 0, st>>>(a);
        return cudaGetLastError();
    });
}

int render_occupancy(int tile_h, int tile_w, bool backward)
{
    int blocks = 0;
    dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        constexpr int h = decltype(TH)::value, w = decltype(TW)::value;
        if (backward)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_bwd<h, w>, kBlock, 0);
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_fwd<h, w>, kBlock, 0);
    });
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_param_grads(const float4 *pos_logit, const float4 *quat, const float2 *log_scale,
                               const float4 *wgrad, int64_t n, float4 *g_pos_logit, float4 *g_quat,
                               float2 *g_log_scale, int accumulate, cudaStream_t st)
{
    (void)log_scale;
    if (n <= 0) return cudaSuccess;
    k_param_grads<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
        pos_logit, quat, wgrad, n, g_pos_logit, g_quat, g_log_scale, accumulate);
    return cudaGetLastError();
}

}  // namespace splat
