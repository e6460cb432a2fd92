// K8 (loss) and K9 (Adam, optionally fused with K7).
//
// Loss over the valid pixels M_v (target range > 0, Sec. 3.3.1): the L1 range term of
// Eq. loss_range (rho_d = Dt^rho_exp, 1 by default), the normal term of Eq. loss_normal taken either against the target
// normal or against the normal of the rendered range map (self-regularised), and optionally the
// opacity term of Eq. loss_opacity.  Per-pixel gradients are written
// for the backward; the scalar is reduced per warp in binary32 and per CTA in binary64.
//
// Adam: the paper does not name its optimiser; a bias-corrected Adam with one learning rate per
// parameter group is used.  The fused form applies the parameter chain rule (world-frame
// accumulators -> d/dmu, d/dlogit, d/dq, d/dlog s) inside the update, so no parameter-gradient
// buffer is written or read.  Both are HBM-bound streaming kernels (one primitive per thread,
// 16-byte loads).

#include "splat_internal.cuh"

namespace splat {
namespace {

__device__ __forceinline__ float3 f3sub(float3 a, float3 b)
{
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 f3cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3dot(float3 a, float3 b)
{
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
__device__ __forceinline__ float3 f3scale(float3 a, float s)
{
    return make_float3(a.x * s, a.y * s, a.z * s);
}

// One stencil of the self-regularised normal term (Eq. loss_normal with N(D) from the rendered
// range map, after 2DGS): base pixel u = (r, c), x = (r, c + 1 mod W), y = (r + 1, c);
// P(w) = D(w) v(w); m = (P(x) - P(u)) x (P(y) - P(u)); n_D = -sign(m . v(u)) m / |m| faces the
// sensor.  The term lambda (1 - N(u) . n_D) counts where the targets of u, x and y are valid,
// their rendered ranges are positive and m != 0; the sign is held fixed in the gradient.  Gives
// the value, n_D and dL/dP at x and y (dL/dP(u) = -(gx + gy)).
struct Stencil {
    bool ok;
    float val;
    float3 nd, gx, gy;
};

// The pixel-centre rays of the 3 x 3 neighbourhood of pixel (r, c) (columns wrapped), from one
// sine/cosine pair per row and per column: ray(i, j) is the ray of (r - 1 + i, c - 1 + j), the
// same products pixel_ray forms.
struct Rays3x3 {
    float ct[3], st[3], cg[3], sg[3];
    __device__ __forceinline__ float3 ray(int i, int j) const
    {
        return make_float3(ct[i] * cg[j], ct[i] * sg[j], st[i]);
    }
};

__device__ __forceinline__ Rays3x3 rays_around(const ViewDesc &vd, int r, int c)
{
    Rays3x3 t;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int rr = r - 1 + i;
        const float th = vd.rows > 1 ? vd.elev_max - vd.dtheta * static_cast<float>(rr)
                                     : vd.elev_max;
        sincosf(th, &t.st[i], &t.ct[i]);
        int cc = c - 1 + i;
        cc = cc < 0 ? cc + vd.cols : (cc >= vd.cols ? cc - vd.cols : cc);
        const float g = 3.14159265358979f - vd.dgamma * (static_cast<float>(cc) + 0.5f);
        sincosf(g, &t.sg[i], &t.cg[i]);
    }
    return t;
}

// the stencil with base (r, c) = neighbourhood offset (i, j) of the rays' centre pixel
__device__ __forceinline__ Stencil normal_stencil(const ViewDesc &vd, int r, int c,
                                                  const Rays3x3 &rays, int i, int j,
                                                  const float *__restrict__ depth,
                                                  const float *__restrict__ normal,
                                                  const float *__restrict__ t_depth, int64_t n,
                                                  float lambda_n)
{
    Stencil s;
    s.ok = false;
    if (r < 0 || r + 1 >= vd.rows) return s;
    const int cx = c + 1 == vd.cols ? 0 : c + 1;
    const int64_t iu = vd.pixel_offset + static_cast<int64_t>(r) * vd.cols + c;
    const int64_t ix = iu - c + cx, iy = iu + vd.cols;
    if (!(t_depth[iu] > 0.0f && t_depth[ix] > 0.0f && t_depth[iy] > 0.0f)) return s;
    const float du = depth[iu], dxr = depth[ix], dyr = depth[iy];
    if (!(du > 0.0f && dxr > 0.0f && dyr > 0.0f)) return s;   // a zero range: side undefined
    const float3 vu = rays.ray(i, j), vx = rays.ray(i, j + 1), vy = rays.ray(i + 1, j);
    const float3 pu = f3scale(vu, du);
    const float3 dx = f3sub(f3scale(vx, dxr), pu), dy = f3sub(f3scale(vy, dyr), pu);
    const float3 m = f3cross(dx, dy);
    const float mn = sqrtf(f3dot(m, m));
    if (!(mn > 0.0f)) return s;
    const float sgn = f3dot(m, vu) > 0.0f ? -1.0f : 1.0f;
    const float inv = 1.0f / mn;
    const float3 mh = f3scale(m, inv);
    const float3 N = make_float3(normal[iu], normal[n + iu], normal[2 * n + iu]);
    s.nd = f3scale(mh, sgn);
    s.val = lambda_n * (1.0f - f3dot(N, s.nd));
    const float3 g = f3scale(N, -lambda_n);                         // dL/dn_D
    const float3 gm = f3scale(f3sub(g, f3scale(mh, f3dot(mh, g))), sgn * inv);   // dL/dm
    s.gx = f3cross(dy, gm);
    s.gy = f3cross(gm, dx);
    s.ok = true;
    return s;
}

// normal_mode 0: the normal term against the target normals; 1: the self-regularised term
// (each pixel gathers dL/dD from the three stencils it belongs to, so no atomics are needed).
template <int kNormalMode>
__global__ void __launch_bounds__(256) k_loss(const float *__restrict__ depth,
                                              const float *__restrict__ normal,
                                              const float *__restrict__ alpha,
                                              const float *__restrict__ t_depth,
                                              const float *__restrict__ t_normal, int64_t n,
                                              float lambda_n, float lambda_o, float o_eps,
                                              float rho_exp, float *__restrict__ g_depth,
                                              float *__restrict__ g_normal,
                                              float *__restrict__ g_alpha,
                                              double *__restrict__ loss_out,
                                              const ViewDesc *__restrict__ views, int n_views,
                                              const uint8_t *__restrict__ active)
{
    __shared__ double s_part[8];
    float acc = 0.0f;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float dt = t_depth[p];
        float gd = 0.0f, gn0 = 0.0f, gn1 = 0.0f, gn2 = 0.0f, go = 0.0f;
        int v = 0;
        if (kNormalMode == 1 || active)
            while (v + 1 < n_views && views[v + 1].pixel_offset <= p) ++v;
        const bool view_on = !active || active[v] != 0;   // views not sampled do not count
        if (dt > 0.0f && view_on) {
            const float rho = rho_exp == 0.0f ? 1.0f : powf(dt, rho_exp);   // rho_d = Dt^p
            const float e = depth[p] - dt;
            acc += rho * fabsf(e);
            gd = e > 0.0f ? rho : (e < 0.0f ? -rho : 0.0f);
            if (kNormalMode == 0) {
                const float n0 = t_normal[p], n1 = t_normal[n + p], n2 = t_normal[2 * n + p];
                const float dn = normal[p] * n0 + normal[n + p] * n1 + normal[2 * n + p] * n2;
                acc += lambda_n * (1.0f - dn);
                gn0 = -lambda_n * n0;
                gn1 = -lambda_n * n1;
                gn2 = -lambda_n * n2;
            }
            if (lambda_o != 0.0f) {
                const float o = alpha[p];
                acc += lambda_o * -logf(fmaxf(o, o_eps));
                go = o > o_eps ? -lambda_o / o : 0.0f;
            }
        }
        if (kNormalMode == 1 && view_on && lambda_n != 0.0f) {
            const ViewDesc &vd = views[v];
            const int64_t local = p - vd.pixel_offset;
            const int r = static_cast<int>(local / vd.cols), c = static_cast<int>(local % vd.cols);
            const Rays3x3 rays = rays_around(vd, r, c);
            const float3 vp = rays.ray(1, 1);
            const Stencil s0 = normal_stencil(vd, r, c, rays, 1, 1, depth, normal, t_depth, n,
                                              lambda_n);
            if (s0.ok) {   // p is the stencil's base u
                acc += s0.val;
                gn0 = -lambda_n * s0.nd.x;
                gn1 = -lambda_n * s0.nd.y;
                gn2 = -lambda_n * s0.nd.z;
                gd -= f3dot(make_float3(s0.gx.x + s0.gy.x, s0.gx.y + s0.gy.y, s0.gx.z + s0.gy.z),
                            vp);
            }
            const Stencil s1 = normal_stencil(vd, r, c == 0 ? vd.cols - 1 : c - 1, rays, 1, 0,
                                              depth, normal, t_depth, n, lambda_n);
            if (s1.ok) gd += f3dot(s1.gx, vp);   // p is x of its left neighbour's stencil
            const Stencil s2 = normal_stencil(vd, r - 1, c, rays, 0, 1, depth, normal, t_depth, n,
                                              lambda_n);
            if (s2.ok) gd += f3dot(s2.gy, vp);   // p is y of the stencil above
        }
        g_depth[p] = gd;
        g_normal[p] = gn0;
        g_normal[n + p] = gn1;
        g_normal[2 * n + p] = gn2;
        g_alpha[p] = go;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = static_cast<double>(acc);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += s_part[w];
        atomicAdd(loss_out, t);
    }
}

struct AdamScalars {
    float c1, c2;   // bias corrections 1 - beta^t
};

__device__ __forceinline__ AdamScalars adam_scalars(const AdamArgs &a)
{
    const float t = static_cast<float>(*a.step + 1);
    return AdamScalars{1.0f - powf(a.beta1, t), 1.0f - powf(a.beta2, t)};
}

__device__ __forceinline__ float adam1(float p, float g, float &m, float &v, float lr,
                                       const AdamArgs &a, const AdamScalars &s)
{
    m = a.beta1 * m + (1.0f - a.beta1) * g;
    v = a.beta2 * v + (1.0f - a.beta2) * g * g;
    const float mh = m / s.c1, vh = v / s.c2;
    return p - lr * mh / (sqrtf(vh) + a.eps);
}

__device__ __forceinline__ void adam_prim(const AdamArgs &a, int64_t i, float4 g_pl, float4 g_q,
                                          float2 g_ls, const AdamScalars &s)
{
    float4 p = a.pos_logit[i], m = a.m_pl[i], v = a.v_pl[i];
    p.x = adam1(p.x, g_pl.x, m.x, v.x, a.lr_pos, a, s);
    p.y = adam1(p.y, g_pl.y, m.y, v.y, a.lr_pos, a, s);
    p.z = adam1(p.z, g_pl.z, m.z, v.z, a.lr_pos, a, s);
    p.w = adam1(p.w, g_pl.w, m.w, v.w, a.lr_opacity, a, s);
    a.pos_logit[i] = p;
    a.m_pl[i] = m;
    a.v_pl[i] = v;
    float4 q = a.quat[i], mq = a.m_q[i], vq = a.v_q[i];
    q.x = adam1(q.x, g_q.x, mq.x, vq.x, a.lr_rot, a, s);
    q.y = adam1(q.y, g_q.y, mq.y, vq.y, a.lr_rot, a, s);
    q.z = adam1(q.z, g_q.z, mq.z, vq.z, a.lr_rot, a, s);
    q.w = adam1(q.w, g_q.w, mq.w, vq.w, a.lr_rot, a, s);
    a.quat[i] = q;
    a.m_q[i] = mq;
    a.v_q[i] = vq;
    float2 l = a.log_scale[i], ml = a.m_ls[i], vl = a.v_ls[i];
    l.x = adam1(l.x, g_ls.x, ml.x, vl.x, a.lr_scale, a, s);
    l.y = adam1(l.y, g_ls.y, ml.y, vl.y, a.lr_scale, a, s);
    a.log_scale[i] = l;
    a.m_ls[i] = ml;
    a.v_ls[i] = vl;
}

__global__ void __launch_bounds__(256) k_adam(const AdamArgs a, const float4 *__restrict__ g_pl,
                                              const float4 *__restrict__ g_q,
                                              const float2 *__restrict__ g_ls)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    adam_prim(a, i, g_pl[i], g_q[i], g_ls[i], adam_scalars(a));
}

__global__ void __launch_bounds__(256) k_adam_fused(const AdamArgs a,
                                                    const float4 *__restrict__ wgrad)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float4 gp, gq;
    float2 gl;
    chain_params(a.pos_logit[i], a.quat[i], wgrad + 4 * i, gp, gq, gl);
    if (a.lambda_s != 0.0f) {
        // scale term: growth of the larger scale beyond tau_s (the first axis on a tie);
        // d/dlog s = s
        const float2 ls = a.log_scale[i];
        const float sa = expf(ls.x), sb = expf(ls.y);
        const float sm = fmaxf(sa, sb);
        float pen = 0.0f;
        if (sm > a.tau_s) {
            pen = a.lambda_s * (sm - a.tau_s);
            if (sa >= sb) gl.x += a.lambda_s * sa;
            else gl.y += a.lambda_s * sb;
        }
        double acc = static_cast<double>(pen);
        const unsigned am = __activemask();
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(am, acc, o);
        if ((threadIdx.x & 31) == __ffs(am) - 1 && acc != 0.0) atomicAdd(a.loss_out, acc);
    }
    adam_prim(a, i, gp, gq, gl, adam_scalars(a));
}

__global__ void k_step_inc(int32_t *step)
{
    *step += 1;
}

}  // namespace

cudaError_t launch_loss(const float *depth, const float *normal, const float *alpha,
                        const float *t_depth, const float *t_normal, int64_t n_pixels,
                        float lambda_n, float lambda_o, float o_eps, float rho_exp,
                        float *g_depth, float *g_normal, float *g_alpha, double *loss_out,
                        cudaStream_t st, const ViewDesc *views, int n_views,
                        const uint8_t *active, int normal_mode)
{
    if (n_pixels <= 0) return cudaSuccess;
    if (normal_mode != 0 && (normal_mode != 1 || !views || n_views < 1))
        return cudaErrorInvalidValue;
    int64_t blocks = (n_pixels + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    auto kern = normal_mode == 1 ? k_loss<1> : k_loss<0>;
    kern<<<static_cast<unsigned>(blocks), 256, 0, st>>>(depth, normal, alpha, t_depth, t_normal,
                                                        n_pixels, lambda_n, lambda_o, o_eps,
                                                        rho_exp, g_depth, g_normal, g_alpha,
                                                        loss_out,
                                                        views, n_views, active);
    return cudaGetLastError();
}

cudaError_t launch_adam(const AdamArgs &a, const float4 *g_pl, const float4 *g_q,
                        const float2 *g_ls, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    k_adam<<<static_cast<unsigned>((a.n + 255) / 256), 256, 0, st>>>(a, g_pl, g_q, g_ls);
    return cudaGetLastError();
}

cudaError_t launch_adam_fused(const AdamArgs &a, const float4 *wgrad, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    k_adam_fused<<<static_cast<unsigned>((a.n + 255) / 256), 256, 0, st>>>(a, wgrad);
    return cudaGetLastError();
}

cudaError_t launch_step_inc(int32_t *step, cudaStream_t st)
{
    k_step_inc<<<1, 1, 0, st>>>(step);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------------
// back-projection of a rendered range image (Sec. 3.3)
// ---------------------------------------------------------------------------------------------
namespace {

// one packed pixel per thread: its view (a scan of the per-view pixel offsets), its ray at the
// pixel centre, the range D / O where O >= o_min, and the point in the world frame
// R^c_w^T (p - t^c_w); NaN where invalid
__global__ void k_backproject(const ViewDesc *__restrict__ views, int n_views, int64_t n_pixels,
                              const float *__restrict__ depth, const float *__restrict__ alpha,
                              float o_min, float *__restrict__ points)
{
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n_pixels) return;
    int v = 0;
    while (v + 1 < n_views && views[v + 1].pixel_offset <= k) ++v;
    const ViewDesc &vd = views[v];
    const int64_t local = k - vd.pixel_offset;
    const int r = static_cast<int>(local / vd.cols), c = static_cast<int>(local % vd.cols);
    const float O = alpha[k];
    float px = __int_as_float(0x7FC00000), py = px, pz = px;
    if (O >= o_min) {
        const float d = depth[k] / O;
        const float g = 3.14159265358979f - vd.dgamma * (static_cast<float>(c) + 0.5f);
        const float th = vd.rows > 1 ? vd.elev_max - vd.dtheta * static_cast<float>(r)
                                     : vd.elev_max;
        float sg, cg, st, ct;
        sincosf(g, &sg, &cg);
        sincosf(th, &st, &ct);
        const float sx = d * ct * cg - vd.t_hi[0], sy = d * ct * sg - vd.t_hi[1],
                    sz = d * st - vd.t_hi[2];
        const float *R = vd.R_hi;
        px = R[0] * sx + R[3] * sy + R[6] * sz;
        py = R[1] * sx + R[4] * sy + R[7] * sz;
        pz = R[2] * sx + R[5] * sy + R[8] * sz;
    }
    points[k] = px;
    points[n_pixels + k] = py;
    points[2 * n_pixels + k] = pz;
}

}  // namespace

cudaError_t launch_backproject(const ViewDesc *views, int n_views, int64_t n_pixels,
                               const float *depth, const float *alpha, float o_min, float *points,
                               cudaStream_t st)
{
    if (n_pixels <= 0) return cudaSuccess;
    k_backproject<<<static_cast<unsigned>((n_pixels + 255) / 256), 256, 0, st>>>(
        views, n_views, n_pixels, depth, alpha, o_min, points);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------------------
// keyframe sampling (Sec. 3.3)
// ---------------------------------------------------------------------------------------------
namespace {

__global__ void k_sample_views(int n_views, int draws, const uint32_t *__restrict__ thr,
                               uint32_t seed_lo, uint32_t seed_hi, uint32_t *__restrict__ step,
                               uint8_t *__restrict__ active)
{
    const int lane = threadIdx.x;
    const uint32_t s = *step;
    for (int v = lane; v < n_views; v += 32) active[v] = 0;
    __syncwarp();
    for (int j = lane; j < draws; j += 32) {
        const uint32_t x = philox4x32_10(make_uint4(static_cast<uint32_t>(j), s, 0u, 0u),
                                         make_uint2(seed_lo, seed_hi)).x;
        int age = 0;
        for (int a = 0; a + 1 < n_views; ++a) age += x >= thr[a] ? 1 : 0;
        active[n_views - 1 - age] = 1;
    }
    __syncwarp();
    if (lane == 0) *step = s + 1u;
}

}  // namespace

cudaError_t launch_sample_views(int n_views, int draws, const uint32_t *thr, uint32_t seed_lo,
                                uint32_t seed_hi, uint32_t *step, uint8_t *active,
                                cudaStream_t st)
{
    k_sample_views<<<1, 32, 0, st>>>(n_views, draws, thr, seed_lo, seed_hi, step, active);
    return cudaGetLastError();
}

}  // namespace splat
