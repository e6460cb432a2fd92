// Photometric registration residual (Sec. 3.3.3, Eq. L_photo) and its Gauss-Newton normal
// equations in the pose, reduced over one view's pixels.
//
// Pixel u of the rendered view with O(u) >= o_min: d = D / O, p = d v(u), p' = T p with T the
// render -> query transform (binary32 3 x 4 on the device, so a Gauss-Newton loop can update it
// without the host); u' = phi(p') (continuous column and row of the same sensor model); the
// query range image is sampled bilinearly at u' (columns wrap; the four pixels must exist and be
// valid); r = |p'| - Dq(u').  With the right perturbation T exp(xi^), xi = (rho, omega),
// dr/dxi = [a, p x a] where a = R^T dr/dp'.  Huber IRLS weight w = min(1, delta / |r|).
// Each thread accumulates w J J^T (upper triangle), w J r, the Huber cost and the count over its
// pixels in binary32; warps reduce by shuffles, blocks in binary64 into the 29 outputs.
// HBM-bound: 8 bytes of the render per pixel and the query image's gathers (L2-resident).

#include "splat_internal.cuh"

namespace splat {
namespace {

constexpr int kPhotoThreads = 256;
constexpr int kPhotoOut = 29;   // 21 H (upper, row-major), 6 g, cost, count

__global__ void __launch_bounds__(kPhotoThreads) k_photometric(
    const ViewDesc vd, const float *__restrict__ depth, const float *__restrict__ alpha,
    const float *__restrict__ qdepth, const float *__restrict__ T, float o_min, float delta,
    double *__restrict__ out, float *__restrict__ per_pixel)
{
    __shared__ float s_part[kPhotoThreads / 32][kPhotoOut];
    float acc[kPhotoOut];
#pragma unroll
    for (int k = 0; k < kPhotoOut; ++k) acc[k] = 0.0f;
    float R[9], t[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R[3 * k] = __ldg(T + 4 * k);
        R[3 * k + 1] = __ldg(T + 4 * k + 1);
        R[3 * k + 2] = __ldg(T + 4 * k + 2);
        t[k] = __ldg(T + 4 * k + 3);
    }
    const int64_t P = static_cast<int64_t>(vd.rows) * vd.cols;
    const float dth = vd.rows > 1 ? vd.dtheta : vd.dgamma;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * kPhotoThreads + threadIdx.x; i < P;
         i += static_cast<int64_t>(gridDim.x) * kPhotoThreads) {
        float res = 0.0f, w = 0.0f, J[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        const float O = alpha[i];
        bool used = false;
        if (O >= o_min) {
            const int r = static_cast<int>(i / vd.cols), c = static_cast<int>(i % vd.cols);
            const float d = depth[i] / O;
            const float3 v = pixel_ray(vd, r, c);
            const float px = d * v.x, py = d * v.y, pz = d * v.z;
            const float x = R[0] * px + R[1] * py + R[2] * pz + t[0];
            const float y = R[3] * px + R[4] * py + R[5] * pz + t[1];
            const float z = R[6] * px + R[7] * py + R[8] * pz + t[2];
            const float rxy2 = x * x + y * y;
            if (rxy2 > 0.0f) {
                const float rxy = sqrtf(rxy2), rho2 = rxy2 + z * z, rho = sqrtf(rho2);
                const float cp = (3.14159265358979f - atan2f(y, x)) / vd.dgamma - 0.5f;
                const float rp = vd.rows > 1 ? (vd.elev_max - atan2f(z, rxy)) / dth : 0.0f;
                const float rf = floorf(rp), cf = floorf(cp);
                const int r0 = static_cast<int>(rf);
                if (rf >= 0.0f && r0 + 1 < vd.rows) {
                    int ca = static_cast<int>(cf) % vd.cols;
                    if (ca < 0) ca += vd.cols;
                    const int cb = ca + 1 == vd.cols ? 0 : ca + 1;
                    const float *row0 = qdepth + static_cast<int64_t>(r0) * vd.cols;
                    const float *row1 = row0 + vd.cols;
                    const float q00 = row0[ca], q01 = row0[cb], q10 = row1[ca], q11 = row1[cb];
                    if (q00 > 0.0f && q01 > 0.0f && q10 > 0.0f && q11 > 0.0f) {
                        const float fr = rp - rf, fc = cp - cf;
                        const float top = (1.0f - fc) * q00 + fc * q01;
                        const float bot = (1.0f - fc) * q10 + fc * q11;
                        const float sample = (1.0f - fr) * top + fr * bot;
                        const float dS_dc = (1.0f - fr) * (q01 - q00) + fr * (q11 - q10);
                        const float dS_dr = (1.0f - fc) * (q10 - q00) + fc * (q11 - q01);
                        // d c'/d p' = (y, -x, 0) / (dgamma rxy^2);
                        // d r'/d p' = -(-z x / (rxy rho^2), -z y / (rxy rho^2), rxy / rho^2) / dth
                        const float kc = dS_dc / (vd.dgamma * rxy2);
                        const float kr = dS_dr / (dth * rho2);
                        const float zr = z / rxy;
                        const float gx = x / rho - (kc * y + kr * zr * x);
                        const float gy = y / rho - (-kc * x + kr * zr * y);
                        const float gz = z / rho - (-kr * rxy);
                        // a = R^T g; J = [a, p x a]
                        const float ax = R[0] * gx + R[3] * gy + R[6] * gz;
                        const float ay = R[1] * gx + R[4] * gy + R[7] * gz;
                        const float az = R[2] * gx + R[5] * gy + R[8] * gz;
                        J[0] = ax;
                        J[1] = ay;
                        J[2] = az;
                        J[3] = py * az - pz * ay;
                        J[4] = pz * ax - px * az;
                        J[5] = px * ay - py * ax;
                        res = rho - sample;
                        const float ares = fabsf(res);
                        w = ares <= delta ? 1.0f : delta / ares;
                        acc[27] += ares <= delta ? 0.5f * res * res : delta * (ares - 0.5f * delta);
                        acc[28] += 1.0f;
                        used = true;
                    }
                }
            }
        }
        if (used) {
            int k = 0;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const float wa = w * J[a];
#pragma unroll
                for (int b = a; b < 6; ++b) acc[k++] += wa * J[b];
                acc[21 + a] += wa * res;
            }
        }
        if (per_pixel) {
            per_pixel[i] = res;
            per_pixel[P + i] = w;
#pragma unroll
            for (int a = 0; a < 6; ++a) per_pixel[(2 + a) * P + i] = J[a];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kPhotoOut; ++k) {
        float x = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        if (lane == 0) s_part[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kPhotoOut) {
        double s = 0.0;
        for (int w8 = 0; w8 < kPhotoThreads / 32; ++w8) s += static_cast<double>(s_part[w8][threadIdx.x]);
        if (s != 0.0) atomicAdd(out + threadIdx.x, s);
    }
}

}  // namespace

cudaError_t launch_photometric(const ViewDesc &vd, const float *depth, const float *alpha,
                               const float *qdepth, const float *T, float o_min, float delta,
                               double *out, float *per_pixel, int sms, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * kPhotoOut, st);
    if (e != cudaSuccess) return e;
    const int64_t P = static_cast<int64_t>(vd.rows) * vd.cols;
    if (P <= 0) return cudaSuccess;
    int64_t blocks = (P + kPhotoThreads - 1) / kPhotoThreads;
    const int64_t cap = static_cast<int64_t>(sms > 0 ? sms : 152) * 4;
    if (blocks > cap) blocks = cap;
    k_photometric<<<static_cast<unsigned>(blocks), kPhotoThreads, 0, st>>>(
        vd, depth, alpha, qdepth, T, o_min, delta, out, per_pixel);
    return cudaGetLastError();
}

}  // namespace splat
