// K5/K6 (+K10): front-to-back compositing and its back-to-front adjoint as persistent kernels
// over a work queue, and K7, the chain rule from the per-primitive accumulators to the
// parameters.
//
// Work decomposition.  A work item is one 4 x 8 pixel block of one tile (a tile is
// tile_h x tile_w = 256 pixels, i.e. 8 blocks), taken by one warp; the queue holds the blocks of
// every tile of every registered view, so many keyframes of uneven sizes share one launch, and
// hands tiles out longest list first so that the last items are short.  Warps never wait for
// one another.  A warp walks its tile's slice of the sorted list (Sec. 3.2.1) 32 entries at a
// time -- every lane reads one entry's projection record and tests whether the primitive's pixel
// rectangle meets the warp's block -- and stages the entries that do, 32 at a time, into shared
// memory.  A staged batch is then evaluated pair-parallel: the (primitive, pixel) candidates --
// every pixel of the block inside a staged primitive's rectangle that is still live -- are
// numbered primitive-major (a prefix sum of the per-primitive counts; each primitive's lane
// writes its candidates into a shared list), and each round gives one candidate to every lane,
// so the intersection math runs on all 32 lanes whatever the primitives' footprints.
// Each pixel's lane then composites that round's hits on it in list order (front to back in the
// forward, back to front in the backward), fetching them from the candidate lanes by shuffle.
// The forward has a second schedule for batches whose candidates spread evenly over the block's
// pixels: every lane takes its own pixel's candidates (a 32 x 32 bit transpose of the staged
// primitives' pixel masks) and evaluates and blends them one per step in its registers, with no
// hand-over; each batch takes whichever schedule its candidate counts make cheaper.  Both blend
// every pixel's hits in list order with the same operations, so the choice changes no result.
// A warp leaves its block as soon as all its pixels are saturated.
//
// Numerics.  Each pixel ray is intersected with a splat as two planes h_x, h_y through the
// sensor (Sec. 3.2.2, Eq. planes_to_splat; Supp. D.1): h_a = (h_x.b_a, h_x.b_b, h_x.b_c),
// h_b likewise with h_y, p = h_a x h_b, s_hat = (p_x, p_y) / p_z.  The products h.b_c are lateral
// offsets of the splat centre from the pixel planes: centimetres out of up to 100 m of range,
// which binary32 sensor-frame vectors cannot resolve.  So every tile has its own orthonormal
// frame Q = (e1, e2, e3) -- e1 the ray through the tile centre, e2 and e3 its two planes -- and
// a primitive is staged as Q b, with the centre Q b_c kept as a float pair; Q R^c_w, Q t^c_w and
// the pixel planes in that frame come from tables computed in FP64 on the host (float pairs).
// In h_x.b_c and h_y.b_c two products cancel; each pair is summed exactly inside one fused
// multiply-add with the rounding error of the other product and the operands' low parts added
// back (dot_pair), so grazing rays at range keep their accuracy.  (A cheaper binary32 pre-test
// that skipped this for clear misses paid off only while all lanes of a warp evaluated one
// primitive: with 32 different pairs per warp some lane always passes it.)
//
// The range is d = nu . v (nu lies on the ray, so this equals |nu| without a square root) and
// a hit counts only when d > 0 (in front of the sensor).  Cutoffs: alpha clamped at alpha_max,
// skipped below alpha_min, stop before T < t_min, and max |s_hat| <= sigma written as
// max(|p_x|, |p_y|) <= sigma |p_z| so that misses need no division.
//
// Forward and backward evaluate a pair with the same explicitly rounded operations.  The forward
// records, per work item, the staged primitives that contributed with the mask of the pixels they
// contributed to (contributor records, below); the backward walks those records back to front, so
// it evaluates exactly the forward's contributing pairs and no others.  The backward recovers
// T_k = T_{k+1} / (1 - alpha_k) from the final transmittance and keeps the suffix sums B_{d,k},
// B_{n,k}, B_{o,k} of Supp. D.2 (as one sum over the channels) in the pixel's lane.  Within a
// round every hit is an affine map of the pixel's (T, sum) state, so each hit lane composes the
// maps of the pixel's earlier hits of the round by pointer jumping, reads the pixel's state once,
// and forms its own dL/dalpha_k and blending weight and the pair's 13 geometric terms.  The
// backward numbers candidates in groups of four lanes that share one primitive (a primitive's
// pixels fill whole groups), so the terms are summed inside the group by two exchanges, then
// across the consecutive groups of one primitive by a segmented suffix sum, and the primitive's
// first group adds them into its shared-memory accumulator without atomics (shared float atomics
// where the lanes of a primitive meet measured 3x slower).  After the batch, the
// lane that staged a primitive rotates its sums back to the world frame and issues four float4
// atomics into a per-primitive accumulator (view independent, so gradients of many views add up
// directly).

#include "splat_internal.cuh"

namespace splat {
namespace {

constexpr int kWarps = kBlock / 32;  // warps per CTA (independent)
constexpr int kBlocksPerTile = kBlock / 32;
constexpr int kAcc = 13;             // per staged primitive: g_ba'(3) g_bb'(3) g_c'(3) g_n(3) g_o
constexpr uint32_t kFull = 0xFFFFFFFFu;
// Relative cost of the forward's two schedules of a staged batch (measured on the 12-keyframe
// render): one pixel-parallel step (every lane evaluates and blends one candidate of its own
// pixel) against one pair-parallel round (32 candidates, then the hand-over of the hits to their
// pixels' lanes); the batch takes the pixel-parallel schedule when
// max_pixel_candidates * kPixelStepCost <= rounds * kRoundCost.
constexpr int kPixelStepCost = 9, kRoundCost = 20;

// A staged primitive, as four float4 rows and one float (structure of arrays, so that lanes
// reading different primitives spread over the banks):
//   a: b_alpha' (tile frame), o        b: b_beta' (tile frame), packed pixel rectangle (bits)
//   c: c' = Q b_c, hi part (tile frame); w: low part of c'_x
//   n: normal (sensor frame); w: low part of c'_y            czl: low part of c'_z
struct SlotRef {
    const float4 &a, &b, &c, &n;
    const float &czl;
};

// a pixel's planes and ray in the tile frame; the low parts kept are those of the components
// that enter the exact pair of each plane (h_x: 0 and 1, h_y: 0 and 2)
struct Pix {
    float hx0, hx1, hx2;
    float hy0, hy1, hy2;
    float v0, v1, v2;
    float hxl0, hxl1;
    float hyl0, hyl2;
};

__device__ __forceinline__ float dot3e(float a0, float a1, float a2, float b0, float b1, float b2)
{
    return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

// h . c' with h and c' as float pairs, the plane h of a pixel and c' the splat centre, both in
// the tile frame.  Two of the three products are large (range x the pixel's angular offset from
// the tile centre, and the centre's lateral offset from the tile's plane) and cancel to the
// centre's offset from the pixel's plane, centimetres out of up to 100 m: for h_x they are
// products 0 and 1, for h_y products 0 and 2.  The pair is summed inside one fused multiply-add,
// fma(h_a, c_a, fl(h_b c_b)), which forms h_a c_a exactly and rounds only the small sum; the
// rounding error of fl(h_b c_b) (one more fma), the low parts of both operands of the pair and
// the third, small product are added in binary32.
__device__ __forceinline__ float dot_pair(float ha, float ca, float hb, float cb, float hal,
                                          float cal, float hbl, float cbl, float hc, float cc)
{
    const float pb = __fmul_rn(hb, cb);
    const float eb = __fmaf_rn(hb, cb, -pb);
    const float sum = __fmaf_rn(ha, ca, pb);
    float err = __fmaf_rn(ha, cal, eb);
    err = __fmaf_rn(hb, cbl, err);
    err = __fmaf_rn(hal, ca, err);
    err = __fmaf_rn(hbl, cb, err);
    err = __fmaf_rn(hc, cc, err);
    return __fadd_rn(sum, err);
}

__device__ __forceinline__ Pix load_pix(const PixFrame *table, int index)
{
    const float4 *e = reinterpret_cast<const float4 *>(table + index);
    const float4 a = e[0], b = e[1], c = e[2], d = e[3];
    Pix p;
    p.hx0 = a.x; p.hx1 = a.y; p.hx2 = a.z;
    p.hy0 = a.w; p.hy1 = b.x; p.hy2 = b.y;
    p.v0 = b.z; p.v1 = b.w; p.v2 = c.x;
    p.hxl0 = c.y; p.hxl1 = c.z;
    p.hyl0 = d.x; p.hyl2 = d.z;
    return p;
}

// pixel mask of a rectangle over the 4 x 8 block with top-left (br, bc): bit 8 r + c for the
// block's row r and column c
__device__ __forceinline__ uint32_t pixel_mask(uint32_t rect, int br, int bc)
{
    const int r_lo = rect & 0xFF, r_hi = (rect >> 8) & 0xFF;
    const int c_lo = (rect >> 16) & 0xFF, c_hi = rect >> 24;
    const int ra = max(r_lo - br, 0), rb = min(r_hi - br, 3);
    const int ca = max(c_lo - bc, 0), cb = min(c_hi - bc, 7);
    if (ra > rb || ca > cb) return 0u;
    const uint32_t cols = ((2u << cb) - 1u) & ~((1u << ca) - 1u);
    const uint32_t rows = (0xFFFFFFFFu >> (8 * (3 - rb))) & (0xFFFFFFFFu << (8 * ra));
    return (cols * 0x01010101u) & rows;
}

// mask of the lanes t whose value key_t equals this lane's index (5 ballots over the key bits)
__device__ __forceinline__ uint32_t lanes_keyed_to_me(bool valid, int key, int lane)
{
    uint32_t m = __ballot_sync(kFull, valid);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t b = __ballot_sync(kFull, (key >> k) & 1);
        m &= ((lane >> k) & 1) ? b : ~b;
    }
    return m;
}

// inclusive warp prefix sum
__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// 32 x 32 bit transpose over the warp: lane j holds row j (bit l = column l); afterwards lane l
// holds column l (bit j = bit l of row j).  Five butterfly stages each swap the off-diagonal
// blocks of the level: the lane with bit s clear keeps the columns with bit s clear and takes its
// partner's, the other lane the reverse.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    constexpr uint32_t kHigh[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu,
                                   0xAAAAAAAAu};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int s = 16 >> k;
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & kHigh[k]) | ((y & kHigh[k]) >> s))
                       : ((x & ~kHigh[k]) | ((y & ~kHigh[k]) << s));
    }
    return x;
}

// Per-warp shared state: the staged batch (structure of arrays), the block's pixel frames
// (structure of arrays, four float4 per pixel), and the queue of list entries that meet the
// block and wait to be staged (appended in walk order 32 at a time).
struct WarpBatch {
    float4 a[32], b[32], c[32], n[32];
    float czl[32];        // low part of c'_z
    uint32_t pos[32];     // list position of the staged entry (backward: bit 31 = flipped)
    uint32_t prim[32];    // primitive index
    float4 p0[32], p1[32], p2[32];
    float p3[32];
    // the batch's candidates in numbering order: slot << 5 | pixel, bit 15 = a candidate (the
    // backward's padding entries of a group carry their slot without it)
    uint16_t cand[1024];
    uint32_t hits[32];    // forward: the block's pixels each slot contributed to
};

constexpr uint16_t kCandValid = 0x8000u;

// write the candidates of slot `lane` (pixel mask m) at entries [first, first + span): the set
// bits of m in increasing order, then padding entries that carry the slot only
__device__ __forceinline__ void list_candidates(uint16_t *cand, uint32_t m, int first, int span,
                                                int lane)
{
    int j = first;
    while (m) {
        const int px = __ffs(m) - 1;
        m &= m - 1u;
        cand[j++] = static_cast<uint16_t>(kCandValid | (lane << 5) | px);
    }
    for (; j < first + span; ++j) cand[j] = static_cast<uint16_t>(lane << 5);
}

// entries of the tile's list that meet the warp's block, waiting to be staged: fewer than 32
// left over from the last chunk plus up to 128 from the next
constexpr int kQueue = 160;
struct WarpQueue {
    uint32_t p[kQueue];      // pair id
    uint32_t rect[kQueue];   // pixel rectangle inside the tile
    uint32_t pos[kQueue];    // list position, bit 31: normal flipped
};

__device__ __forceinline__ SlotRef slot_at(const WarpBatch &w, int s)
{
    return SlotRef{w.a[s], w.b[s], w.c[s], w.n[s], w.czl[s]};
}

__device__ __forceinline__ void put_pix(WarpBatch &w, int lane, const Pix &p)
{
    w.p0[lane] = make_float4(p.hx0, p.hx1, p.hx2, p.hy0);
    w.p1[lane] = make_float4(p.hy1, p.hy2, p.v0, p.v1);
    w.p2[lane] = make_float4(p.v2, p.hxl0, p.hxl1, p.hyl0);
    w.p3[lane] = p.hyl2;
}

__device__ __forceinline__ Pix get_pix(const WarpBatch &w, int l)
{
    const float4 a = w.p0[l], b = w.p1[l], c = w.p2[l];
    const float d = w.p3[l];
    Pix p;
    p.hx0 = a.x; p.hx1 = a.y; p.hx2 = a.z;
    p.hy0 = a.w; p.hy1 = b.x; p.hy2 = b.y;
    p.v0 = b.z; p.v1 = b.w; p.v2 = c.x;
    p.hxl0 = c.y; p.hxl1 = c.z;
    p.hyl0 = c.w; p.hyl2 = d;
    return p;
}

// stage pair id p of the tile into slot s, in the tile frame; returns the primitive index
__device__ __forceinline__ uint32_t stage(const RenderArgs &A, const TileInfo &ti, uint32_t p,
                                          bool flip, uint32_t rect, WarpBatch &w, int s)
{
    const int64_t i = static_cast<int64_t>(p) - static_cast<int64_t>(ti.view) * A.n;
    const float4 pl = A.pos_logit[i];
    const float4 ea = A.prim[3 * i], eb = A.prim[3 * i + 1], en = A.prim[3 * i + 2];
    const float *M = ti.M_hi;
    w.a[s] = make_float4(M[0] * ea.x + M[1] * ea.y + M[2] * ea.z,
                         M[3] * ea.x + M[4] * ea.y + M[5] * ea.z,
                         M[6] * ea.x + M[7] * ea.y + M[8] * ea.z, ea.w);
    w.b[s] = make_float4(M[0] * eb.x + M[1] * eb.y + M[2] * eb.z,
                         M[3] * eb.x + M[4] * eb.y + M[5] * eb.z,
                         M[6] * eb.x + M[7] * eb.y + M[8] * eb.z, __uint_as_float(rect));
    f2 c[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        c[r] = f2_dot3_add2(f2{ti.M_hi[3 * r], ti.M_lo[3 * r]},
                            f2{ti.M_hi[3 * r + 1], ti.M_lo[3 * r + 1]},
                            f2{ti.M_hi[3 * r + 2], ti.M_lo[3 * r + 2]}, pl.x, pl.y, pl.z,
                            f2{ti.u_hi[r], ti.u_lo[r]});
    const float *R = ti.R;
    const float fs = flip ? -1.0f : 1.0f;
    w.c[s] = make_float4(c[0].h, c[1].h, c[2].h, c[0].l);
    w.n[s] = make_float4(fs * (R[0] * en.x + R[1] * en.y + R[2] * en.z),
                         fs * (R[3] * en.x + R[4] * en.y + R[5] * en.z),
                         fs * (R[6] * en.x + R[7] * en.y + R[8] * en.z), c[1].l);
    w.czl[s] = c[2].l;
    return static_cast<uint32_t>(i);
}

struct Hit {
    float ha0, ha1, ha2, hb0, hb1, hb2;
    float pz, px, py, inv, sa, sb, G, a, d;
    bool clamped;
};

// the per-pair test and geometry, identical in forward and backward
__device__ __forceinline__ bool evaluate(const SlotRef &s, const Pix &px, float sigma,
                                         float amin, float amax, Hit &h)
{
    h.ha0 = dot3e(px.hx0, px.hx1, px.hx2, s.a.x, s.a.y, s.a.z);
    h.ha1 = dot3e(px.hx0, px.hx1, px.hx2, s.b.x, s.b.y, s.b.z);
    h.hb0 = dot3e(px.hy0, px.hy1, px.hy2, s.a.x, s.a.y, s.a.z);
    h.hb1 = dot3e(px.hy0, px.hy1, px.hy2, s.b.x, s.b.y, s.b.z);
    // offsets of the centre from the two pixel planes, the cancelling pair summed exactly
    h.ha2 = dot_pair(px.hx0, s.c.x, px.hx1, s.c.y, px.hxl0, s.c.w, px.hxl1, s.n.w, px.hx2, s.c.z);
    h.hb2 = dot_pair(px.hy0, s.c.x, px.hy2, s.c.z, px.hyl0, s.c.w, px.hyl2, s.czl, px.hy1, s.c.y);
    h.pz = __fmaf_rn(h.ha0, h.hb1, -__fmul_rn(h.ha1, h.hb0));
    h.px = __fmaf_rn(h.ha1, h.hb2, -__fmul_rn(h.ha2, h.hb1));
    h.py = __fmaf_rn(h.ha2, h.hb0, -__fmul_rn(h.ha0, h.hb2));
    const float apz = fabsf(h.pz);
    if (!(apz > 0.0f) || !(fmaxf(fabsf(h.px), fabsf(h.py)) <= __fmul_rn(sigma, apz)))
        return false;
    h.inv = __fdividef(1.0f, h.pz);
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

// add a per-lane counter to a global total: one atomic per warp, no block barrier
__device__ __forceinline__ void warp_count(unsigned long long v, unsigned long long *total)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// the next work item of this warp (lane 0 takes it from the queue)
__device__ __forceinline__ uint32_t next_item(uint32_t *queue, int lane)
{
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(queue, 1u);
    return __shfl_sync(kFull, it, 0);
}

// copy the tile's 192-byte record into the warp's shared slot
__device__ __forceinline__ void load_tile(const TileInfo *tiles, int64_t tile, TileInfo &dst,
                                         int lane)
{
    const float4 *src = reinterpret_cast<const float4 *>(tiles + tile);
    float4 *d = reinterpret_cast<float4 *>(&dst);
    if (lane < 12) d[lane] = src[lane];
    __syncwarp();
}

struct BlockPix {
    int br, bc, lr, lc;
    bool inside;
    int64_t out;     // packed pixel index
    int pf;          // pixel-frame entry
};

template <int TH, int TW>
__device__ __forceinline__ BlockPix block_pixel(const TileInfo &ti, int blk, int lane)
{
    constexpr int WC = TW / 8;
    BlockPix b;
    b.br = (blk / WC) * 4;
    b.bc = (blk % WC) * 8;
    b.lr = b.br + (lane >> 3);
    b.lc = b.bc + (lane & 7);
    b.inside = b.lr < ti.valid_r && b.lc < ti.valid_c;
    b.out = ti.out_base + static_cast<int64_t>(b.lr) * ti.cols + b.lc;
    b.pf = ti.pix_base + b.lr * TW + b.lc;
    return b;
}

// Candidate numbering of a staged batch: lane b holds its primitive's live-pixel mask m, the
// count before it (off) and, after the call, the batch total K (uniform).
struct Numbering {
    uint32_t m;
    int off, K;
};

__device__ __forceinline__ Numbering number_candidates(uint32_t m, int lane)
{
    Numbering nb;
    nb.m = m;
    const int n = __popc(m);
    const int incl = warp_incl_scan(n, lane);
    nb.off = incl - n;
    nb.K = __shfl_sync(kFull, incl, 31);
    return nb;
}

// The backward numbers groups of four candidates instead: a primitive's pixels fill
// ceil(n / 4) whole groups (off and K count groups), so that the four lanes of an aligned lane
// group always belong to one primitive and its terms can be summed inside the group.
__device__ __forceinline__ Numbering number_groups(uint32_t m, int lane)
{
    Numbering nb;
    nb.m = m;
    const int n = (__popc(m) + 3) >> 2;
    const int incl = warp_incl_scan(n, lane);
    nb.off = incl - n;
    nb.K = __shfl_sync(kFull, incl, 31);
    return nb;
}

// Contributor records.  The forward appends, per work item and in list order, one record per
// staged primitive that contributed to a pixel of the block: (pair id | normal-flip bit 31,
// mask of the block's pixels it contributed to).  Records go to chunks of 32 taken from a pool by
// an atomic counter; each chunk links to the item's previous one, and the item keeps its last
// chunk and that chunk's fill.  The backward walks an item's chunks from the last, each chunk
// (read back to front) being one batch, so it evaluates exactly the pairs that contributed.
constexpr uint32_t kNoChunk = 0xFFFFFFFFu;

// append the records of the lanes with `have` (in lane order) to the item's chain
__device__ __forceinline__ void append_records(const RenderArgs &A, bool have, uint2 r, int lane,
                                               uint32_t &chain, int &fill)
{
    const uint32_t bal = __ballot_sync(kFull, have);
    const int nh = __popc(bal);
    if (nh == 0 || fill < 0) return;
    const int rank = __popc(bal & ((1u << lane) - 1u));
    const int room = chain == kNoChunk ? 0 : 32 - fill;
    if (nh <= room) {
        if (have) A.rec[static_cast<int64_t>(chain) * 32 + fill + rank] = r;
        fill += nh;
        return;
    }
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(A.rec_alloc, 1u);
    c = __shfl_sync(kFull, c, 0);
    if (c >= A.rec_cap) {   // pool exhausted: the backward of this item would be incomplete
        if (lane == 0) atomicOr(A.status, SPLAT_STATUS_CAPACITY);
        fill = -1;
        return;
    }
    if (lane == 0) A.rec_prev[c] = chain;
    if (have) {
        if (rank < room)
            A.rec[static_cast<int64_t>(chain) * 32 + fill + rank] = r;
        else
            A.rec[static_cast<int64_t>(c) * 32 + (rank - room)] = r;
    }
    chain = c;
    fill = nh - room;
}

// ---------------------------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------------------------
struct FwdShared {
    WarpBatch w[kWarps];
    TileInfo ti[kWarps];
    WarpQueue q[kWarps];
};

template <int TH, int TW>
__global__ void __launch_bounds__(kBlock, 3) k_render_fwd(const RenderArgs A)
{
    static_assert(TH * TW == kBlock && TH % 4 == 0 && TW % 8 == 0, "4x8 warp blocks");
    extern __shared__ __align__(16) unsigned char s_raw[];
    FwdShared &sh = *reinterpret_cast<FwdShared *>(s_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpBatch &w = sh.w[warp];
    TileInfo &ti = sh.ti[warp];
    WarpQueue &q = sh.q[warp];
    unsigned long long evals = 0;

    for (;;) {
        const uint32_t item = next_item(A.queue, lane);
        if (item >= A.n_items) break;
        const int64_t tile = A.tile_order[item / kBlocksPerTile];
        const int blk = item % kBlocksPerTile;
        __syncwarp();
        load_tile(A.tiles, tile, ti, lane);
        const BlockPix bp = block_pixel<TH, TW>(ti, blk, lane);
        put_pix(w, lane, load_pix(A.pixframes, bp.inside ? bp.pf : ti.pix_base));
        const uint2 rg = A.ranges[tile];
        float T = 1.0f, D = 0.0f, N0 = 0.0f, N1 = 0.0f, N2 = 0.0f, O = 0.0f;
        int last = 0;
        bool done = !bp.inside;
        uint32_t chain = kNoChunk;   // this item's last record chunk
        int fill = 0;                 // records in it

        // blend a hit (alpha a, range d, staged slot bs) into this pixel, front to back
        auto blend = [&](float a, float d, int bs) {
            const float tt = __fmul_rn(T, __fsub_rn(1.0f, a));
            if (tt < A.t_min) {
                done = true;
                return;
            }
            const float wgt = __fmul_rn(a, T);
            D = __fmaf_rn(wgt, d, D);
            const float4 nn = w.n[bs];
            N0 = __fmaf_rn(wgt, nn.x, N0);
            N1 = __fmaf_rn(wgt, nn.y, N1);
            N2 = __fmaf_rn(wgt, nn.z, N2);
            O = __fadd_rn(O, wgt);
            T = tt;
            last = static_cast<int>(w.pos[bs]) + 1;
            atomicOr(&w.hits[bs], 1u << lane);
        };

        // stage queue entries [off, off + cnt) and composite them in one of two schedules
        auto composite = [&](int cnt, int off) {
            uint32_t m = 0u;
            w.hits[lane] = 0u;
            const int qi = off + lane;
            if (lane < cnt) {
                stage(A, ti, q.p[qi], (q.pos[qi] >> 31) != 0, q.rect[qi], w, lane);
                w.pos[lane] = q.pos[qi] & 0x7FFFFFFFu;
                m = pixel_mask(q.rect[qi], bp.br, bp.bc);
            }
            m &= __ballot_sync(kFull, !done);
            // this pixel's candidates: the slots whose mask holds it
            uint32_t mine = transpose32(m, lane);
            const int steps_px = static_cast<int>(
                __reduce_max_sync(kFull, static_cast<unsigned>(__popc(mine))));
            const int K = static_cast<int>(
                __reduce_add_sync(kFull, static_cast<unsigned>(__popc(m))));
            evals += __popc(mine);
            __syncwarp();
            if (steps_px * kPixelStepCost <= ((K + 31) >> 5) * kRoundCost) {
                // pixel-parallel: each lane evaluates its own pixel's candidates in slot (= list)
                // order and blends them in its registers
                const Pix px = get_pix(w, lane);
                while (__any_sync(kFull, mine != 0u)) {
                    if (mine != 0u) {
                        const int j = __ffs(mine) - 1;
                        mine &= mine - 1u;
                        Hit h;
                        if (evaluate(slot_at(w, j), px, A.sigma, A.alpha_min, A.alpha_max, h)) {
                            blend(h.a, h.d, j);
                            if (done) mine = 0u;
                        }
                    }
                }
            } else {
                // pair-parallel: one candidate per lane and round, numbered primitive-major
                const Numbering nb = number_candidates(m, lane);
                list_candidates(w.cand, m, nb.off, __popc(m), lane);
                __syncwarp();
                for (int r0 = 0; r0 < nb.K; r0 += 32) {
                    const int t = r0 + lane;
                    const uint32_t e = t < nb.K ? w.cand[t] : 0u;
                    const bool valid = (e & kCandValid) != 0u;
                    const int b = (e >> 5) & 31, l = e & 31;
                    Hit h;
                    h.a = h.d = 0.0f;
                    bool hit = false;
                    if (valid)
                        hit = evaluate(slot_at(w, b), get_pix(w, l), A.sigma, A.alpha_min,
                                       A.alpha_max, h);
                    // this pixel's hits of the round, in list order, fetched from their lanes
                    // two at a time (both fetches are issued before the first is blended)
                    uint32_t hm = lanes_keyed_to_me(hit, l, lane);
                    while (__any_sync(kFull, hm != 0u)) {
                        const bool have1 = hm != 0u;
                        const int src1 = have1 ? __ffs(hm) - 1 : lane;
                        hm &= hm - 1u;
                        const bool have2 = hm != 0u;
                        const int src2 = have2 ? __ffs(hm) - 1 : lane;
                        hm &= hm - 1u;
                        const float a1 = __shfl_sync(kFull, h.a, src1);
                        const float d1 = __shfl_sync(kFull, h.d, src1);
                        const int b1 = __shfl_sync(kFull, b, src1);
                        const float a2 = __shfl_sync(kFull, h.a, src2);
                        const float d2 = __shfl_sync(kFull, h.d, src2);
                        const int b2 = __shfl_sync(kFull, b, src2);
                        if (have1 && !done) blend(a1, d1, b1);
                        if (have2 && !done) blend(a2, d2, b2);
                    }
                    if (__all_sync(kFull, done)) break;
                }
            }
            __syncwarp();
            // contributor records of the batch (slots with at least one contribution), in list
            // order, for the backward
            if (A.rec) {
                const uint32_t hm = lane < cnt ? w.hits[lane] : 0u;
                const uint2 r = lane < cnt ? make_uint2(q.p[qi] | (q.pos[qi] & 0x80000000u), hm)
                                           : make_uint2(0u, 0u);
                append_records(A, hm != 0u, r, lane, chain, fill);
            }
        };

        // Walk the tile's list 128 entries at a time from the 4-aligned entry at or below its
        // start: each lane reads the block masks of four consecutive entries as one word (the
        // next chunk's word is loaded ahead), the entries that meet the block are appended to
        // the queue in list order (a warp prefix sum of the lanes' counts), with their pair ids
        // and rectangles read as one 16-byte vector each, and every 32 queued entries are
        // staged and composited.
        const uint32_t *mask_words = reinterpret_cast<const uint32_t *>(A.entry_blocks);
        const uint32_t base = rg.x & ~3u;
        uint32_t mw = 0u;
        if (base + 4u * lane < rg.y) mw = mask_words[(base >> 2) + lane];
        int qn = 0;
        for (uint32_t ch = base; ch < rg.y; ch += 128) {
            if (__all_sync(kFull, done)) break;
            const uint32_t j0 = ch + 4u * lane;
            uint32_t mnext = 0u;
            if (j0 + 128u < rg.y) mnext = mask_words[(j0 + 128u) >> 2];
            uint32_t rel4 = 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t j = j0 + k;
                if (j >= rg.x && j < rg.y && ((mw >> (8 * k + blk)) & 1u)) rel4 |= 1u << k;
            }
            uint4 pv = make_uint4(0u, 0u, 0u, 0u), rv = pv;
            if (rel4) {
                pv = *reinterpret_cast<const uint4 *>(A.sorted_vals + j0);
                rv = *reinterpret_cast<const uint4 *>(A.entry_rect + j0);
            }
            const uint32_t pa[4] = {pv.x, pv.y, pv.z, pv.w};
            const uint32_t ra[4] = {rv.x, rv.y, rv.z, rv.w};
            // once some pixels of the block are saturated, an entry whose rectangle covers only
            // saturated ones is passed over
            const uint32_t live = __ballot_sync(kFull, !done);
            if (live != kFull) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (((rel4 >> k) & 1u) && !(pixel_mask(ra[k] & ~kRectFlip, bp.br, bp.bc) & live))
                        rel4 &= ~(1u << k);
            }
            const int c4 = __popc(rel4);
            const int incl = warp_incl_scan(c4, lane);
            if (rel4) {
                int at = qn + incl - c4;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if ((rel4 >> k) & 1u) {
                        q.p[at] = pa[k];
                        q.rect[at] = ra[k] & ~kRectFlip;
                        q.pos[at] = (j0 + k - rg.x) | ((ra[k] & kRectFlip) ? 0x80000000u : 0u);
                        ++at;
                    }
                }
            }
            qn += __shfl_sync(kFull, incl, 31);
            mw = mnext;
            __syncwarp();
            int head = 0;
            while (qn - head >= 32 && !__all_sync(kFull, done)) {
                composite(32, head);
                head += 32;
            }
            if (head > 0) {   // move the rest (fewer than 32 unless all pixels are done) down
                qn -= head;
                if (qn >= 32) qn = 0;   // every pixel is done: the walk ends at the loop's top
                uint32_t pp = 0u, rr = 0u, ps = 0u;
                if (lane < qn) {
                    pp = q.p[head + lane];
                    rr = q.rect[head + lane];
                    ps = q.pos[head + lane];
                }
                __syncwarp();
                if (lane < qn) {
                    q.p[lane] = pp;
                    q.rect[lane] = rr;
                    q.pos[lane] = ps;
                }
                __syncwarp();
            }
        }
        if (qn > 0 && !__all_sync(kFull, done)) composite(qn, 0);
        if (A.rec && lane == 0) {   // an item whose records overflowed the pool keeps none
            A.rec_head[item] = fill < 0 ? kNoChunk : chain;
            A.rec_fill[item] = fill < 0 ? 0u : static_cast<uint32_t>(fill);
        }
        if (bp.inside) {
            A.depth[bp.out] = D;
            A.normal[bp.out] = N0;
            A.normal[A.n_pixels + bp.out] = N1;
            A.normal[2 * A.n_pixels + bp.out] = N2;
            A.alpha[bp.out] = O;
            A.t_final[bp.out] = T;
            A.n_last[bp.out] = last;
        }
    }
    warp_count(evals, A.evals);
}

// ---------------------------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------------------------
struct BwdShared {
    WarpBatch w[kWarps];
    float acc[kWarps][32][kAcc];
    float pose[kWarps][16];  // the batch's reduced sensor-pose terms (9 used)
    TileInfo ti[kWarps];
};

template <int TH, int TW>
__global__ void __launch_bounds__(kBlock, 3) k_render_bwd(const RenderArgs A)
{
    static_assert(TH * TW == kBlock && TH % 4 == 0 && TW % 8 == 0, "4x8 warp blocks");
    extern __shared__ __align__(16) unsigned char s_raw[];
    BwdShared &sh = *reinterpret_cast<BwdShared *>(s_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpBatch &w = sh.w[warp];
    float(*acc)[kAcc] = sh.acc[warp];
    float *pose_sums = sh.pose[warp];
    TileInfo &ti = sh.ti[warp];
    unsigned long long evals = 0;

    for (;;) {
        const uint32_t item = next_item(A.queue, lane);
        if (item >= A.n_items) break;
        const int64_t tile = A.tile_order[item / kBlocksPerTile];
        const int blk = item % kBlocksPerTile;
        __syncwarp();
        load_tile(A.tiles, tile, ti, lane);
        const BlockPix bp = block_pixel<TH, TW>(ti, blk, lane);
        put_pix(w, lane, load_pix(A.pixframes, bp.inside ? bp.pf : ti.pix_base));
        float T = 1.0f, gD = 0.0f, gN0 = 0.0f, gN1 = 0.0f, gN2 = 0.0f, gO = 0.0f;
        if (bp.inside) {
            T = A.t_final[bp.out];
            if (A.g_depth) gD = A.g_depth[bp.out];
            if (A.g_normal) {
                gN0 = A.g_normal[bp.out];
                gN1 = A.g_normal[A.n_pixels + bp.out];
                gN2 = A.g_normal[2 * A.n_pixels + bp.out];
            }
            if (A.g_alpha) gO = A.g_alpha[bp.out];
        }
        float Y = 0.0f;   // sum over channels of g_ch B_ch (suffix sums of Supp. D.2)

        // stage the batch's records (slot l = record r of lane l: pair id | flip, contributed
        // pixels), replay and differentiate them round by round, then flush each staged
        // primitive's sums (lane b flushes slot b)
        auto adjoint = [&](int cnt, uint2 r) {
            uint32_t m = 0u;
            if (lane < cnt) {
                w.prim[lane] = stage(A, ti, r.x & 0x7FFFFFFFu, (r.x >> 31) != 0, 0u, w, lane);
                w.pos[lane] = r.x & 0x80000000u;
#pragma unroll
                for (int c = 0; c < kAcc; ++c) acc[lane][c] = 0.0f;
                m = r.y;
            }
            const Numbering nb = number_groups(m, lane);
            list_candidates(w.cand, m, 4 * nb.off, 4 * ((__popc(m) + 3) >> 2), lane);
            __syncwarp();
            for (int u0 = 0; u0 < nb.K; u0 += 8) {
                const int t = 4 * u0 + lane;
                const uint32_t e = t < 4 * nb.K ? w.cand[t] : (31u << 5);
                const bool valid = (e & kCandValid) != 0u;
                const int b = (e >> 5) & 31, l = e & 31;
                // the pixel's channel gradients meet the hit's channels in its own lane:
                // X_k = sum_ch g_ch x_ch,k (x = d, 1, n); fetched before the evaluation so that
                // the exchanges overlap it
                const float gDl = __shfl_sync(kFull, gD, l);
                const float gOl = __shfl_sync(kFull, gO, l);
                const float gNl0 = __shfl_sync(kFull, gN0, l);
                const float gNl1 = __shfl_sync(kFull, gN1, l);
                const float gNl2 = __shfl_sync(kFull, gN2, l);
                Hit h;
                h.a = h.d = 0.0f;
                h.clamped = false;
                bool hit = false;
                if (valid) {
                    ++evals;
                    hit = evaluate(slot_at(w, b), get_pix(w, l), A.sigma, A.alpha_min,
                                   A.alpha_max, h);
                }
                float X = 0.0f, inv_om = 0.0f;
                if (hit) {
                    const float4 nn = w.n[b];
                    X = gDl * h.d + gOl + gNl0 * nn.x + gNl1 * nn.y + gNl2 * nn.z;
                    inv_om = __fdividef(1.0f, __fsub_rn(1.0f, h.a));
                }
                // The round's hits on a pixel, back to front in lane order: hit k takes the
                // pixel's (T, Y) -- transmittance and Y = sum_ch g_ch B_ch,k, the suffix sum of
                // Supp. D.2 -- to (T io_k, Y + a_k X_k io_k T), io_k = 1 / (1 - alpha_k): an
                // affine map (s_k, c_k) = (io_k, a_k X_k io_k).  Each hit lane composes the maps
                // of the pixel's earlier hits by pointer jumping along the chain of the pixel's
                // hit lanes, applies them to the pixel's state at the round start, and forms
                // T_k = T io_k, w_k = alpha_k T_k and dL/dalpha_k = T_k X_k - Y io_k itself; the
                // pixel lane then applies the composition of all its hits of the round.
                const uint32_t mine = lanes_keyed_to_me(hit, l, lane);   // pixel lane: its hits
                const uint32_t peers = __shfl_sync(kFull, mine, l);      // hit lane: its pixel's
                const int prev0 = hit ? 31 - __clz(peers & ((1u << lane) - 1u)) : -1;
                float ms = hit ? inv_om : 1.0f, mc = hit ? h.a * X * inv_om : 0.0f;
                int pv = prev0;
                while (__any_sync(kFull, pv >= 0)) {
                    const int src = pv >= 0 ? pv : lane;
                    const float ps = __shfl_sync(kFull, ms, src);
                    const float pc = __shfl_sync(kFull, mc, src);
                    const int pp = __shfl_sync(kFull, pv, src);
                    if (pv >= 0) {
                        mc = pc + ps * mc;
                        ms = ps * ms;
                        pv = pp;
                    }
                }
                const int xsrc = prev0 >= 0 ? prev0 : lane;   // the earlier hits' composition
                const float xs0 = __shfl_sync(kFull, ms, xsrc);
                const float xc0 = __shfl_sync(kFull, mc, xsrc);
                const float xs = prev0 >= 0 ? xs0 : 1.0f, xc = prev0 >= 0 ? xc0 : 0.0f;
                const float Tl = __shfl_sync(kFull, T, l), Yl = __shfl_sync(kFull, Y, l);
                {
                    const int last = mine != 0u ? 31 - __clz(mine) : lane;
                    const float ls = __shfl_sync(kFull, ms, last);
                    const float lc = __shfl_sync(kFull, mc, last);
                    if (mine != 0u) {
                        Y = Y + lc * T;
                        T = ls * T;
                    }
                }
                float g[16];
#pragma unroll
                for (int c = 0; c < kAcc; ++c) g[c] = 0.0f;
                if (hit) {
                    const float Tp = xs * Tl, Yp = Yl + xc * Tl;
                    const float Tk = Tp * inv_om;
                    const float wgt = __fmul_rn(h.a, Tk);
                    const float gAe = h.clamped ? 0.0f : Tk * X - Yp * inv_om;
                    const SlotRef st = slot_at(w, b);
                    const Pix px = get_pix(w, l);
                    const float gd = gDl * wgt;            // dL/dd_k
                    g[9] = gNl0 * wgt;                      // dL/dn_k
                    g[10] = gNl1 * wgt;
                    g[11] = gNl2 * wgt;
                    g[12] = gAe * h.G;                      // dL/do
                    // dL/ds_hat: density term and range term (d = nu . v)
                    const float vba = px.v0 * st.a.x + px.v1 * st.a.y + px.v2 * st.a.z;
                    const float vbb = px.v0 * st.b.x + px.v1 * st.b.y + px.v2 * st.b.z;
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
                // sum the group's four lanes (one primitive) by recursive halving: after the
                // exchange across lane bit 0 a lane keeps 8 of the 16 values, after bit 1 it
                // keeps 4 (indices base .. base + 3); then add up the groups of one primitive
                // (consecutive groups) towards its first group of the round, which alone writes
                const uint32_t hm = __ballot_sync(kFull, hit);
                if (hm != 0u) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        if (c + 8 < kAcc) {
                            const bool up = (lane & 1) != 0;
                            const float send = up ? g[c] : g[c + 8];
                            const float keep = up ? g[c + 8] : g[c];
                            g[c] = keep + __shfl_xor_sync(kFull, send, 1);
                        } else {
                            // no term c + 8: the odd lane's slot stands for a term past the 13th,
                            // whose value is never used, so both lanes take the sum of term c
                            g[c] += __shfl_xor_sync(kFull, g[c], 1);
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const bool up = (lane & 2) != 0;
                        const float send = up ? g[c] : g[c + 4];
                        const float keep = up ? g[c + 4] : g[c];
                        g[c] = keep + __shfl_xor_sync(kFull, send, 2);
                    }
#pragma unroll
                    for (int s = 4; s < 32; s <<= 1) {
                        const int bo = __shfl_down_sync(kFull, b, s);
                        const bool same = lane + s < 32 && bo == b;
                        // a primitive's groups are consecutive: when none reaches s lanes ahead,
                        // none reaches 2s ahead, and the remaining stages would add nothing
                        if (!__any_sync(kFull, same)) break;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float o = __shfl_down_sync(kFull, g[c], s);
                            g[c] += same ? o : 0.0f;
                        }
                    }
                    const int bp4 = __shfl_up_sync(kFull, b, 4);
                    const bool first = lane < 4 || bp4 != b;
                    if (first && ((hm >> (lane & ~3)) != 0u)) {
                        const int base = ((lane & 1) ? 8 : 0) + ((lane & 2) ? 4 : 0);
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (base + c < kAcc) acc[b][base + c] += g[c];
                    }
                }
                __syncwarp();
            }
            if (lane < cnt) {
                const float *a = acc[lane];
                bool any = false;
#pragma unroll
                for (int c = 0; c < kAcc; ++c) any |= a[c] != 0.0f;
                if (any) {
                    const float *M = ti.M_hi;
                    const float *R = ti.R;
                    const SlotRef st = slot_at(w, lane);
                    // the scales are the lengths of the staged axes (M is a rotation)
                    const float sa = sqrtf(st.a.x * st.a.x + st.a.y * st.a.y + st.a.z * st.a.z);
                    const float sb = sqrtf(st.b.x * st.b.x + st.b.y * st.b.y + st.b.z * st.b.z);
                    const bool flip = (w.pos[lane] >> 31) != 0;
                    // world frame: M^T g' (M = Q R^c_w), normals: R^c_w^T g_n
                    float gmu[3], gta[3], gtb[3], gtn[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        gmu[j] = M[j] * a[6] + M[3 + j] * a[7] + M[6 + j] * a[8];
                        gta[j] = sa * (M[j] * a[0] + M[3 + j] * a[1] + M[6 + j] * a[2]);
                        gtb[j] = sb * (M[j] * a[3] + M[3 + j] * a[4] + M[6 + j] * a[5]);
                        gtn[j] = R[j] * a[9] + R[3 + j] * a[10] + R[6 + j] * a[11];
                        if (flip) gtn[j] = -gtn[j];
                    }
                    const float gls_a = a[0] * st.a.x + a[1] * st.a.y + a[2] * st.a.z;
                    const float gls_b = a[3] * st.b.x + a[4] * st.b.y + a[5] * st.b.z;
                    float4 *dst = A.wgrad + 4 * static_cast<int64_t>(w.prim[lane]);
                    atomicAdd(dst + 0, make_float4(gmu[0], gmu[1], gmu[2], a[12]));
                    atomicAdd(dst + 1, make_float4(gta[0], gta[1], gta[2], gls_a));
                    atomicAdd(dst + 2, make_float4(gtb[0], gtb[1], gtb[2], gls_b));
                    atomicAdd(dst + 3, make_float4(gtn[0], gtn[1], gtn[2], 0.0f));
                }
            }
            if (A.pose_grad) {
                // sensor-pose terms of the batch (left perturbation T^c_w <- exp(xi^) T^c_w):
                // rho gets g_bc, omega gets b x g for the centre and both axes (tile frame) and
                // n x g_n (sensor frame); summed over the warp, taken to the sensor frame by
                // Q^T = R^c_w M^T
                float v[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) v[c] = 0.0f;
                if (lane < cnt) {
                    const float *a = acc[lane];
                    const SlotRef st = slot_at(w, lane);
                    v[0] = a[6];
                    v[1] = a[7];
                    v[2] = a[8];
                    v[3] = (st.c.y * a[8] - st.c.z * a[7]) + (st.a.y * a[2] - st.a.z * a[1]) +
                           (st.b.y * a[5] - st.b.z * a[4]);
                    v[4] = (st.c.z * a[6] - st.c.x * a[8]) + (st.a.z * a[0] - st.a.x * a[2]) +
                           (st.b.z * a[3] - st.b.x * a[5]);
                    v[5] = (st.c.x * a[7] - st.c.y * a[6]) + (st.a.x * a[1] - st.a.y * a[0]) +
                           (st.b.x * a[4] - st.b.y * a[3]);
                    v[6] = st.n.y * a[11] - st.n.z * a[10];
                    v[7] = st.n.z * a[9] - st.n.x * a[11];
                    v[8] = st.n.x * a[10] - st.n.y * a[9];
                }
                // recursive halving over the warp: lane l < 16 ends with value reduced_index(l)
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int m = 1 << s, half = 8 >> s;
                    const bool up = (lane & m) != 0;
#pragma unroll
                    for (int k = 0; k < half; ++k) {
                        const float send = up ? v[k] : v[k + half];
                        const float keep = up ? v[k + half] : v[k];
                        v[k] = keep + __shfl_xor_sync(kFull, send, m);
                    }
                }
                const float tot = v[0] + __shfl_xor_sync(kFull, v[0], 16);
                const int idx = ((lane & 1) ? 8 : 0) + ((lane & 2) ? 4 : 0) +
                                ((lane & 4) ? 2 : 0) + ((lane & 8) ? 1 : 0);
                float *scratch = pose_sums;
                if (lane < 16 && idx < 9) scratch[idx] = tot;
                __syncwarp();
                if (lane < 6) {
                    const float *M = ti.M_hi;
                    const float *R = ti.R;
                    // y = M^T x (tile frame -> world-axis coordinates), z_k = (R y)_k
                    const int part = lane < 3 ? 0 : 3, k = lane < 3 ? lane : lane - 3;
                    float y[3];
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        y[j] = M[j] * scratch[part] + M[3 + j] * scratch[part + 1] +
                               M[6 + j] * scratch[part + 2];
                    float z = R[3 * k] * y[0] + R[3 * k + 1] * y[1] + R[3 * k + 2] * y[2];
                    if (part == 3) {
                        // a cross product formed in the tile frame changes sign with det Q
                        // (= det M; the frame (ray, h_x, h_y) is left-handed)
                        const float det = M[0] * (M[4] * M[8] - M[5] * M[7]) -
                                          M[1] * (M[3] * M[8] - M[5] * M[6]) +
                                          M[2] * (M[3] * M[7] - M[4] * M[6]);
                        z = (det < 0.0f ? -z : z) + scratch[6 + k];
                    }
                    atomicAdd(A.pose_grad + 6 * static_cast<int64_t>(ti.view) + lane, z);
                }
            }
            __syncwarp();
        };

        // the item's record chunks, last first; each chunk read back to front is one batch
        uint32_t chunk = A.rec_head[item];
        int cnt = static_cast<int>(A.rec_fill[item]);
        while (chunk != kNoChunk) {
            uint2 r = make_uint2(0u, 0u);
            if (lane < cnt) r = A.rec[static_cast<int64_t>(chunk) * 32 + (cnt - 1 - lane)];
            adjoint(cnt, r);
            chunk = A.rec_prev[chunk];
            cnt = 32;
        }
    }
    warp_count(evals, A.evals);
}

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

// both kernels' shared memory is above the 48 KB static limit: allow it once per instantiation
template <int TH, int TW>
cudaError_t fwd_prepare()
{
    static cudaError_t e = cudaFuncSetAttribute(k_render_fwd<TH, TW>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(sizeof(FwdShared)));
    return e;
}

template <int TH, int TW>
cudaError_t bwd_prepare()
{
    static cudaError_t e = cudaFuncSetAttribute(k_render_bwd<TH, TW>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(sizeof(BwdShared)));
    return e;
}

cudaError_t launch_render_fwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st)
{
    return dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        constexpr int h = decltype(TH)::value, w = decltype(TW)::value;
        const cudaError_t e = fwd_prepare<h, w>();
        if (e != cudaSuccess) return e;
        k_render_fwd<h, w><<<grid, kBlock, sizeof(FwdShared), st>>>(a);
        return cudaGetLastError();
    });
}

cudaError_t launch_render_bwd(const RenderArgs &a, int tile_h, int tile_w, int grid,
                              cudaStream_t st)
{
    return dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        constexpr int h = decltype(TH)::value, w = decltype(TW)::value;
        const cudaError_t e = bwd_prepare<h, w>();
        if (e != cudaSuccess) return e;
        k_render_bwd<h, w><<<grid, kBlock, sizeof(BwdShared), st>>>(a);
        return cudaGetLastError();
    });
}

int render_occupancy(int tile_h, int tile_w, bool backward)
{
    int blocks = 0;
    dispatch(tile_h, tile_w, [&](auto TH, auto TW) {
        constexpr int h = decltype(TH)::value, w = decltype(TW)::value;
        if (backward) {
            const cudaError_t e = bwd_prepare<h, w>();
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_bwd<h, w>,
                                                                 kBlock, sizeof(BwdShared));
        }
        const cudaError_t e = fwd_prepare<h, w>();
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_render_fwd<h, w>, kBlock,
                                                             sizeof(FwdShared));
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
