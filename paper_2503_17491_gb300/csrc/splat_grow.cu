// Map growth (Sec. 3.3.1 local model initialisation, Sec. 3.3.2 densification): a mask over the
// packed pixels of the registered views, a weight per pixel from the range gradients of the
// target range image, one systematic weighted draw of n_d pixels over all views, and a new
// primitive per drawn pixel (back-projected target range, normal towards the sensor).
//
// Three launches, no host synchronisation (capturable):
//   k_grow_weights  per pixel: mask and integer weight q (binary32 arithmetic, no contraction),
//                   stored in a scratch array; per block the u64 sum of its chunk
//   k_grow_top      one block: exclusive scan of the block sums, the total Q and the random
//                   offset o of the draw (Philox), the call counter advanced
//   k_grow_select   per pixel: its exclusive prefix C_i by a block scan, the samples
//                   s_j = floor((j Q + o) / n_d) inside [C_i, C_i + q_i), and the new primitive
//                   in the slot of its first sample (its other slots are written empty)
// The integer draw is exact, so the drawn pixels are identical to any other evaluation of the
// same definition.  HBM-bound: about 4 + 4 + 8 bytes per pixel and 40 bytes per slot.

#include "splat_internal.cuh"

namespace splat {
namespace {

constexpr int kGrowThreads = 256;

__device__ __forceinline__ int view_of(const ViewDesc *__restrict__ views, int n_views, int64_t p)
{
    int v = 0;
    while (v + 1 < n_views && views[v + 1].pixel_offset <= p) ++v;
    return v;
}

// The weight of pixel p (0 off the mask).  Adds and multiplies are the rounded intrinsics so
// that nothing is contracted: w = min((w0 + |g_x|) + |g_y|, w_cap), q = floor(256 w).
__device__ __forceinline__ uint32_t grow_weight(const GrowArgs &a, int64_t p)
{
    const float dt = a.t_depth[p];
    if (!(dt > 0.0f)) return 0u;
    if (a.refine) {
        const bool m_n = a.alpha[p] <= a.lambda_do;
        const bool m_e = fabsf(__fsub_rn(a.depth[p], dt)) >= a.lambda_de;
        if (!(m_n || m_e)) return 0u;
    }
    const ViewDesc &vd = a.views[view_of(a.views, a.n_views, p)];
    const int64_t local = p - vd.pixel_offset;
    const int r = static_cast<int>(local / vd.cols), c = static_cast<int>(local % vd.cols);
    const float dx = a.t_depth[p - c + (c + 1 == vd.cols ? 0 : c + 1)];
    const float gx = dx > 0.0f ? __fsub_rn(dx, dt) : 0.0f;
    float gy = 0.0f;
    if (r + 1 < vd.rows) {
        const float dy = a.t_depth[p + vd.cols];
        gy = dy > 0.0f ? __fsub_rn(dy, dt) : 0.0f;
    }
    const float w = fminf(__fadd_rn(__fadd_rn(a.w0, fabsf(gx)), fabsf(gy)), a.w_cap);
    return static_cast<uint32_t>(floorf(__fmul_rn(w, 256.0f)));
}

// Block-wide exclusive scan of one u64 per thread; returns the thread's prefix, *total the sum.
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long x,
                                                                   unsigned long long *s_warp,
                                                                   unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < kGrowThreads / 32; ++w) {
            const unsigned long long t = s_warp[w];
            s_warp[w] = run;
            run += t;
        }
        s_warp[kGrowThreads / 32] = run;
    }
    __syncthreads();
    const unsigned long long r = s_warp[warp] + inc - x;
    *total = s_warp[kGrowThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kGrowThreads) k_grow_weights(const GrowArgs a)
{
    __shared__ unsigned long long s_warp[kGrowThreads / 32 + 1];
    const int64_t lo = static_cast<int64_t>(blockIdx.x) * a.chunk;
    const int64_t hi = lo + a.chunk < a.n_pixels ? lo + a.chunk : a.n_pixels;
    unsigned long long sum = 0;
    for (int64_t p = lo + threadIdx.x; p < hi; p += kGrowThreads) {
        const uint32_t q = grow_weight(a, p);
        a.q[p] = q;
        sum += q;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kGrowThreads / 32; ++w) t += s_warp[w];
        a.block_sums[blockIdx.x] = t;
    }
}

// block_sums[0, grid): exclusive prefixes afterwards; [grid]: Q; [grid + 1]: o
__global__ void __launch_bounds__(1024) k_grow_top(const GrowArgs a)
{
    __shared__ unsigned long long s[1024];
    const int t = threadIdx.x;
    s[t] = t < a.grid ? a.block_sums[t] : 0ull;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
        const unsigned long long y = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += y;
        __syncthreads();
    }
    if (t < a.grid) a.block_sums[t] = t == 0 ? 0ull : s[t - 1];
    if (t == 0) {
        const unsigned long long Q = s[1023];
        const uint32_t call = *a.call;
        const uint32_t x = philox4x32_10(make_uint4(0u, call, 2u, 0u),
                                         make_uint2(a.seed_lo, a.seed_hi)).x;
        // o = floor(x Q / 2^32) = high word of (x 2^32) Q
        a.block_sums[a.grid] = Q;
        a.block_sums[a.grid + 1] = __umul64hi(static_cast<unsigned long long>(x) << 32, Q);
        *a.call = call + 1u;
    }
}

// #{j < n_d : floor((j Q + o) / n_d) < X} = clamp(ceil((X n_d - o) / Q), 0, n_d)
__device__ __forceinline__ unsigned long long samples_below(unsigned long long X,
                                                            unsigned long long n_d,
                                                            unsigned long long Q,
                                                            unsigned long long o)
{
    const unsigned long long xn = X * n_d;
    if (xn <= o) return 0ull;
    const unsigned long long c = (xn - o + Q - 1ull) / Q;
    return c < n_d ? c : n_d;
}

__device__ __forceinline__ void write_empty(const GrowArgs &a, int64_t j)
{
    a.pos_logit[j] = make_float4(0.0f, 0.0f, 0.0f, a.empty_logit);
    a.quat[j] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    a.log_scale[j] = make_float2(0.0f, 0.0f);
}

// The new primitive of pixel p (Sec. 3.3.1): centre T_ws (d v), normal -R_ws v towards the
// sensor as the shortest-arc rotation from e_z, isotropic scale scale_k d sqrt(dgamma dtheta).
__device__ __forceinline__ void write_primitive(const GrowArgs &a, int64_t j, int64_t p)
{
    const ViewDesc &vd = a.views[view_of(a.views, a.n_views, p)];
    const int64_t local = p - vd.pixel_offset;
    const int r = static_cast<int>(local / vd.cols), c = static_cast<int>(local % vd.cols);
    const float d = a.t_depth[p];
    const float3 v = pixel_ray(vd, r, c);
    const float *R = vd.R_hi;   // T^c_w: p_s = R p_w + t, so p_w = R^T (p_s - t)
    const float sx = d * v.x - vd.t_hi[0], sy = d * v.y - vd.t_hi[1], sz = d * v.z - vd.t_hi[2];
    const float mx = R[0] * sx + R[3] * sy + R[6] * sz;
    const float my = R[1] * sx + R[4] * sy + R[7] * sz;
    const float mz = R[2] * sx + R[5] * sy + R[8] * sz;
    float nx = -(R[0] * v.x + R[3] * v.y + R[6] * v.z);
    float ny = -(R[1] * v.x + R[4] * v.y + R[7] * v.z);
    float nz = -(R[2] * v.x + R[5] * v.y + R[8] * v.z);
    const float inv_n = rsqrtf(nx * nx + ny * ny + nz * nz);
    nx *= inv_n;
    ny *= inv_n;
    nz *= inv_n;
    float4 q;
    if (1.0f + nz < 1e-6f) {
        q = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
    } else {
        const float w = 1.0f + nz;
        const float inv_q = rsqrtf(w * w + ny * ny + nx * nx);
        q = make_float4(w * inv_q, -ny * inv_q, nx * inv_q, 0.0f);
    }
    const float dth = vd.rows > 1 ? vd.dtheta : vd.dgamma;
    const float ls = logf(a.scale_k * d * sqrtf(vd.dgamma * dth));
    a.pos_logit[j] = make_float4(mx, my, mz, a.logit);
    a.quat[j] = q;
    a.log_scale[j] = make_float2(ls, ls);
}

__global__ void __launch_bounds__(kGrowThreads) k_grow_select(const GrowArgs a)
{
    __shared__ unsigned long long s_warp[kGrowThreads / 32 + 1];
    const unsigned long long Q = a.block_sums[a.grid], o = a.block_sums[a.grid + 1];
    const unsigned long long n_d = static_cast<unsigned long long>(a.n_d);
    if (Q == 0ull) {   // nothing masked: every slot empty
        for (int64_t j = static_cast<int64_t>(blockIdx.x) * kGrowThreads + threadIdx.x; j < a.n_d;
             j += static_cast<int64_t>(gridDim.x) * kGrowThreads)
            write_empty(a, j);
        return;
    }
    const int64_t lo = static_cast<int64_t>(blockIdx.x) * a.chunk;
    const int64_t hi = lo + a.chunk < a.n_pixels ? lo + a.chunk : a.n_pixels;
    unsigned long long base = a.block_sums[blockIdx.x];
    for (int64_t p0 = lo; p0 < hi; p0 += kGrowThreads) {   // uniform trip count per block
        const int64_t p = p0 + threadIdx.x;
        const unsigned long long q = p < hi ? a.q[p] : 0u;
        unsigned long long tile_total;
        const unsigned long long C = base + block_exclusive_scan(q, s_warp, &tile_total);
        base += tile_total;
        if (q == 0ull) continue;
        const unsigned long long j0 = samples_below(C, n_d, Q, o);
        const unsigned long long j1 = samples_below(C + q, n_d, Q, o);
        if (j1 > j0) {
            write_primitive(a, static_cast<int64_t>(j0), p);
            for (unsigned long long j = j0 + 1; j < j1; ++j) write_empty(a, static_cast<int64_t>(j));
        }
    }
}

}  // namespace

int grow_grid(int64_t n_pixels)
{
    const int64_t tiles = (n_pixels + kGrowThreads - 1) / kGrowThreads;
    return static_cast<int>(tiles < kGrowMaxGrid ? (tiles > 0 ? tiles : 1) : kGrowMaxGrid);
}

cudaError_t launch_grow(GrowArgs a, cudaStream_t st)
{
    if (a.n_d <= 0) return cudaSuccess;
    a.grid = grow_grid(a.n_pixels);
    const int64_t per = (a.n_pixels + a.grid - 1) / a.grid;
    a.chunk = (per + kGrowThreads - 1) / kGrowThreads * kGrowThreads;
    k_grow_weights<<<a.grid, kGrowThreads, 0, st>>>(a);
    k_grow_top<<<1, 1024, 0, st>>>(a);
    k_grow_select<<<a.grid, kGrowThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace splat
