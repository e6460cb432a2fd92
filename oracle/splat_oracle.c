/*
 * FP64 CPU oracle for the spherical 2D-Gaussian rasterizer of Splat-LOAM
 * (arXiv 2503.17491).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: it is used by the tests, by the smoke check and by the CPU
 * baseline leg of the benchmark.  It shares no code, header or table with the
 * CUDA library; both are written from the paper.
 *
 * What is here, and which passage each part follows:
 *
 *  1. or_pose_inverse      T^c_w from the sensor->world pose (Sec. 3.2.2:
 *                          T^k_w describes the world in the sensor frame).
 *  2. Binning contract     (Sec. 3.2.1 tiles + range sort, Sec. 3.2.3 bounding
 *                          box).  The per-primitive decisions that pick an
 *                          integer -- the f32 sort key kappa, the sign that
 *                          turns a normal towards the sensor and the tile
 *                          rectangle -- are taken in IEEE binary32 with a fixed
 *                          sequence of correctly rounded operations, so that a
 *                          CPU and a GPU that follow the sequence reach the same
 *                          bits.  Transcendentals in that sequence are written
 *                          out from their series (atan2 from the arctangent
 *                          Taylor series after a tan(pi/8) reduction, exp from
 *                          a Cody-Waite ln2 split and the exponential series),
 *                          so no libm result enters a decision.  This file must
 *                          be compiled with -ffp-contract=off.
 *  3. or_bin / or_tile_ranges   the per-tile lists sorted by (tile, kappa, id).
 *  4. or_render            FP64 forward: for every pixel ray, every primitive
 *                          (brute) or every primitive binned to its tile (culled),
 *                          in (kappa, id) order: ray/splat intersection by two
 *                          planes (Sec. 3.2.2, Eq. planes_to_splat; Supp. D.1),
 *                          Gaussian density, range, front-to-back alpha
 *                          blending (Eqs. ab_depth, ab_normal, ab_opacity).
 *  5. or_render_backward   FP64 analytic gradient (Supp. D.2), with the dL/dO
 *                          channel added and the chain rule through the
 *                          quaternion, log-scale and opacity logit.
 *  6. or_loss, or_adam     L_d + lambda_n L_n (+ lambda_o L_o) over valid
 *                          pixels (Eqs. loss_range, loss_normal, loss_opacity)
 *                          and a plain Adam step.
 *
 * Readings where the paper is silent (the image grid, cutoffs, normal frame and
 * sign, parametrisation) are listed with the tests that pin them; in short:
 *   column c has azimuth  pi - 2 pi (c + 1/2) / W,
 *   row r has elevation   elev_max - r (elev_max - elev_min) / (H - 1) (elev_max for H = 1),
 *   alpha = min(o G, alpha_max), skipped below alpha_min, stop before a primitive
 *   that would bring T below t_min, 3-sigma box test max|s_hat| <= sigma_cut,
 *   hits behind the sensor skipped, D/N/O not normalised, normals in the sensor
 *   frame flipped towards the sensor, q = (w,x,y,z) normalised, s = exp(log s),
 *   o = sigmoid(logit).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int or_version(void) { return 9; }

/* ------------------------------------------------------------------------- */
/* 1. pose                                                                   */
/* ------------------------------------------------------------------------- */

/* T_ws: row-major 4x4 sensor->world.  R_cw = R_ws^T, t_cw = -R_ws^T t_ws,
 * each t_cw entry summed in the order ((a + b) + c). */
void or_pose_inverse(const double *T_ws, double *R_cw, double *t_cw)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R_cw[3 * i + j] = T_ws[4 * j + i];
    for (int i = 0; i < 3; ++i) {
        double a = T_ws[4 * 0 + i] * T_ws[3];
        double b = T_ws[4 * 1 + i] * T_ws[7];
        double c = T_ws[4 * 2 + i] * T_ws[11];
        t_cw[i] = -((a + b) + c);
    }
}

/* ------------------------------------------------------------------------- */
/* 2. FP32 binning contract                                                  */
/* ------------------------------------------------------------------------- */

#define C_PI      3.14159274f   /* binary32 nearest pi   */
#define C_HALF_PI 1.57079637f   /* binary32 nearest pi/2 */
#define C_TWO_PI  6.28318548f   /* binary32 nearest 2 pi */
#define C_QPI     0.785398163f  /* binary32 nearest pi/4 */
#define C_TAN_PI8 0.414213562f  /* tan(pi/8) */

/* atan2 for the contract: reduce to t = min/max in [0,1]; for t > tan(pi/8)
 * use atan t = pi/4 + atan((t-1)/(t+1)); the reduced |z| <= tan(pi/8) goes
 * through the arctangent series z - z^3/3 + ... + z^17/17 (next term < 3e-9). */
float or_contract_atan2f(float y, float x)
{
    float ax = fabsf(x), ay = fabsf(y);
    float mx = ax > ay ? ax : ay;
    float mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float t = mn / mx;
    float z, base;
    if (t > C_TAN_PI8) { z = (t - 1.0f) / (t + 1.0f); base = C_QPI; }
    else { z = t; base = 0.0f; }
    float z2 = z * z;
    float p = 0.0588235294f;               /*  1/17 */
    p = fmaf(p, z2, -0.0666666667f);       /* -1/15 */
    p = fmaf(p, z2, 0.0769230769f);        /*  1/13 */
    p = fmaf(p, z2, -0.0909090909f);       /* -1/11 */
    p = fmaf(p, z2, 0.111111111f);         /*  1/9  */
    p = fmaf(p, z2, -0.142857143f);        /* -1/7  */
    p = fmaf(p, z2, 0.2f);                 /*  1/5  */
    p = fmaf(p, z2, -0.333333333f);        /* -1/3  */
    p = fmaf(p, z2, 1.0f);
    float a = fmaf(z, p, base);
    if (ay > ax) a = C_HALF_PI - a;
    if (x < 0.0f) a = C_PI - a;
    if (y < 0.0f) a = -a;
    return a;
}

/* exp for the contract: x = k ln2 + r with ln2 split as 2839/4096 (exact
 * times any |k| < 4096) plus the binary32 remainder; e^r from the exponential
 * series through r^7/7! (|r| <= 0.35, truncation < 6e-9); times 2^k built
 * from the exponent field. */
float or_contract_expf(float x)
{
    if (x > 80.0f) x = 80.0f;
    if (x < -80.0f) x = -80.0f;
    float k = rintf(x * 1.44269504f);
    float r = (x - k * 0.693115234375f) - k * 3.19461849e-05f;
    float p = 1.98412698e-04f;             /* 1/5040 */
    p = fmaf(p, r, 1.38888889e-03f);       /* 1/720  */
    p = fmaf(p, r, 8.33333333e-03f);       /* 1/120  */
    p = fmaf(p, r, 4.16666667e-02f);       /* 1/24   */
    p = fmaf(p, r, 0.166666667f);          /* 1/6    */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int ki = (int)k;
    union { uint32_t u; float f; } two_k;
    two_k.u = (uint32_t)(ki + 127) << 23;
    return p * two_k.f;
}

typedef struct { float x, y, z; } f3;

static f3 f3_rot(const float *R, f3 v) /* R row-major 3x3, ((a+b)+c) */
{
    f3 o;
    o.x = (R[0] * v.x + R[1] * v.y) + R[2] * v.z;
    o.y = (R[3] * v.x + R[4] * v.y) + R[5] * v.z;
    o.z = (R[6] * v.x + R[7] * v.y) + R[8] * v.z;
    return o;
}

/* Contract steps C1-C3: activation and sensor-frame vectors in binary32.
 * Returns 0 for a non-finite input or a zero quaternion. */
static int contract_vectors(const float *pl, const float *q, const float *ls,
                            const float *Rf, const float *tf,
                            f3 *ba, f3 *bb, f3 *bc, f3 *nr)
{
    for (int k = 0; k < 4; ++k)
        if (!isfinite(pl[k]) || !isfinite(q[k])) return 0;
    if (!isfinite(ls[0]) || !isfinite(ls[1])) return 0;
    float w = q[0], x = q[1], y = q[2], z = q[3];
    float qq = ((w * w + x * x) + y * y) + z * z;
    if (!(qq > 0.0f) || !isfinite(qq)) return 0;
    float r = sqrtf(qq);
    w = w / r; x = x / r; y = y / r; z = z / r;
    f3 ta = { 1.0f - 2.0f * (y * y + z * z), 2.0f * (x * y + w * z), 2.0f * (x * z - w * y) };
    f3 tb = { 2.0f * (x * y - w * z), 1.0f - 2.0f * (x * x + z * z), 2.0f * (y * z + w * x) };
    f3 tn = { 2.0f * (x * z + w * y), 2.0f * (y * z - w * x), 1.0f - 2.0f * (x * x + y * y) };
    float sa = or_contract_expf(ls[0]);
    float sb = or_contract_expf(ls[1]);
    f3 ra = f3_rot(Rf, ta), rb = f3_rot(Rf, tb), mu = { pl[0], pl[1], pl[2] };
    f3 rm = f3_rot(Rf, mu);
    ba->x = sa * ra.x; ba->y = sa * ra.y; ba->z = sa * ra.z;
    bb->x = sb * rb.x; bb->y = sb * rb.y; bb->z = sb * rb.z;
    bc->x = rm.x + tf[0]; bc->y = rm.y + tf[1]; bc->z = rm.z + tf[2];
    *nr = f3_rot(Rf, tn);
    return 1;
}

/* ln for the contract, x >= 1: x = 2^e m with m folded into [1/sqrt2, sqrt2), then
 * ln m = 2 atanh z, z = (m - 1)/(m + 1), |z| <= 0.172, from the series 2(z + z^3/3 + ... + z^9/9)
 * (next term < 3e-10). */
float or_contract_logf(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    int e = (int)((u >> 23) & 0xFF) - 127;
    uint32_t mu = (u & 0x7FFFFFu) | 0x3F800000u;
    float m;
    memcpy(&m, &mu, 4);
    if (m > 1.41421354f) { m = m * 0.5f; e = e + 1; }
    float z = (m - 1.0f) / (m + 1.0f);
    float z2 = z * z;
    float p = 0.111111111f;          /* 1/9 */
    p = fmaf(p, z2, 0.142857143f);   /* 1/7 */
    p = fmaf(p, z2, 0.2f);           /* 1/5 */
    p = fmaf(p, z2, 0.333333333f);   /* 1/3 */
    p = fmaf(p, z2, 1.0f);
    return fmaf((float)e, 0.693147182f, 2.0f * z * p);
}

/* Contract step C4: conservative spherical bounding box of the splat-space region where the
 * primitive can contribute: the 3-sigma box |s|_inf <= sigma (Sec. 3.2.3) intersected with the
 * disk where o G(s) >= alpha_min, i.e. |s| <= r_o = sqrt(2 ln(o / alpha_min)) (the alpha_min
 * cutoff of the blending), bounded by the polygon |s|_inf <= a = min(sigma, r_o) and
 * |s_a| + |s_b| <= sqrt2 r_o (an octagon when it cuts the square's corners), with a 0.1 % + 0.002
 * margin on r_o.  The polygon is mapped to the sensor frame, P = b_c + s_a b_a + s_b b_b.
 * Supp. B relaxes the tight quartic box to the projected vertices, which misses the elevation
 * bulge of an edge: here every edge's interior elevation extremum is added, and the poles and
 * the sensor-inside case are handled.
 * Azimuth: if the xy-projection of the polygon contains the z axis (with a small tolerance)
 * every column is covered; otherwise the azimuths span less than pi and their extremes are at the
 * vertices, measured relative to the centre direction so that the +-pi seam needs no case.
 * Elevation: extremes over the boundary (vertices, plus the one interior extremum an edge can
 * have, where d/dlambda of z/|xy| vanishes on P + lambda (Q - P)), widened to +-pi/2 when the
 * z axis pierces the polygon above or below the sensor.
 * Out: pixel rows [r0, r1], cyclic pixel columns [c0, c0 + nc) mod W, tile rows [tr0, tr1],
 * cyclic tile columns [tc0, tc0 + ntc) mod TC.  Returns the number of tiles (0 when no pixel ray
 * can reach the region). */
/* Radius of the contributing region in splat units: o G(s) >= alpha_min holds for
 * |s| <= sqrt(2 ln(o / alpha_min)), widened by 0.1 % + 0.002 to cover the binary32 rounding of
 * alpha on the GPU; 0 when o < 0.999 alpha_min (nothing can contribute), and o below alpha_min
 * by less than that is taken at alpha_min (radius 0.002). */
float or_contract_reach_radius(float o, float alpha_min)
{
    float x = o / alpha_min;
    if (x < 0.999f) return 0.0f;
    if (x < 1.0f) x = 1.0f;
    return sqrtf(2.0f * or_contract_logf(x)) * 1.001f + 0.002f;
}

/* keep the higher and the lower of the points seen so far, by elevation atan2(z, r), r >= 0:
 * z r' > z' r says that (z, r) lies above (z', r'); the first of equal points stays */
static void elev_candidate(float z, float r, float *zh, float *rh, float *zl, float *rl, int *have)
{
    if (!*have) {
        *zh = z; *rh = r; *zl = z; *rl = r; *have = 1;
        return;
    }
    if (z * *rh > *zh * r) { *zh = z; *rh = r; }
    if (z * *rl < *zl * r) { *zl = z; *rl = r; }
}

static int contract_bbox(f3 ba, f3 bb, f3 bc, float o, float alpha_min, float sigma, int H,
                         int W, float emin, float emax, int th, int tw, int32_t *pix,
                         int32_t *til)
{
    const float eps = 0.01f; /* pixel-unit margin */
    float ro = or_contract_reach_radius(o, alpha_min);
    if (ro == 0.0f) return 0;
    float a = ro < sigma ? ro : sigma;
    float k = (1.41421356f * ro) / a;   /* diamond |u| + |v| <= k in units of a */
    f3 A = { a * ba.x, a * ba.y, a * ba.z };
    f3 B = { a * bb.x, a * bb.y, a * bb.z };
    f3 C = bc;
    /* the octagon (|u|, |v| <= 1, |u| + |v| <= k in units of a); when the diamond misses the
     * square's corners (k >= 2) the cut c = 1 repeats each corner, and the repeated vertices
     * give zero-length edges that add nothing */
    const int nv = 8;
    float c = k < 2.0f ? k - 1.0f : 1.0f;
    float uv[16] = { 1.0f, -c, 1.0f, c, c, 1.0f, -c, 1.0f,
                     -1.0f, c, -1.0f, -c, -c, -1.0f, c, -1.0f };
    f3 P[8];
    for (int i = 0; i < nv; ++i) {
        float u = uv[2 * i], v = uv[2 * i + 1];
        P[i].x = (C.x + u * A.x) + v * B.x;
        P[i].y = (C.y + u * A.y) + v * B.y;
        P[i].z = (C.z + u * A.z) + v * B.z;
    }

    /* does the z axis cross the xy-shadow of the polygon?  c + u A + v B = 0 with |u|, |v| <= 1
     * and |u| + |v| <= k */
    float det = A.x * B.y - A.y * B.x;
    float ca = C.x * B.y - C.y * B.x;
    float cb = A.x * C.y - A.y * C.x;
    float la = fabsf(A.x) + fabsf(A.y), lb = fabsf(B.x) + fabsf(B.y);
    float lc = fabsf(C.x) + fabsf(C.y);
    float tol = 1e-5f * ((la + lb) * ((lc + la) + lb));
    float ad = fabsf(det);
    int inside = (fabsf(ca) <= ad + tol) && (fabsf(cb) <= ad + tol) &&
                 (fabsf(ca) + fabsf(cb) <= k * ad + 2.0f * tol);
    int pole_n = 0, pole_s = 0;
    if (inside) {
        if (ad > tol) {
            float u = -ca / det, v = -cb / det;
            float zh = (C.z + u * A.z) + v * B.z;
            float tz = 1e-5f * ((fabsf(C.z) + fabsf(A.z)) + fabsf(B.z));
            pole_n = zh > -tz;
            pole_s = zh < tz;
        } else {
            pole_n = pole_s = 1;
        }
    }

    /* elevation: the highest and the lowest of the vertices and of the edges' interior extrema,
     * ordered by z / |xy| without a division (z_i r_j against z_j r_i); one arctangent each */
    float zh = 0.0f, rh = 0.0f, zl = 0.0f, rl = 0.0f;
    int have = 0;
    for (int i = 0; i < nv; ++i) {
        f3 p = P[i], q = P[(i + 1) % nv];
        float rxy = sqrtf(p.x * p.x + p.y * p.y);
        elev_candidate(p.z, rxy, &zh, &rh, &zl, &rl, &have);
        f3 d = { q.x - p.x, q.y - p.y, q.z - p.z };
        float pd = p.x * d.x + p.y * d.y;
        float pp = p.x * p.x + p.y * p.y;
        float dd = d.x * d.x + d.y * d.y;
        float num = p.z * pd - d.z * pp;
        float den = d.z * pd - p.z * dd;
        if (den != 0.0f) {
            float lam = num / den;
            if (lam > 0.0f && lam < 1.0f) {
                f3 X = { p.x + lam * d.x, p.y + lam * d.y, p.z + lam * d.z };
                elev_candidate(X.z, sqrtf(X.x * X.x + X.y * X.y), &zh, &rh, &zl, &rl, &have);
            }
        }
    }
    float th_hi = or_contract_atan2f(zh, rh), th_lo = or_contract_atan2f(zl, rl);
    if (pole_n) th_hi = C_HALF_PI;
    if (pole_s) th_lo = -C_HALF_PI;

    float kr = (float)(H - 1) / (emax - emin);
    float vhi = (emax - th_hi) * kr - eps;
    float vlo = (emax - th_lo) * kr + eps;
    int r0 = (int)ceilf(vhi), r1 = (int)floorf(vlo);
    if (r0 < 0) r0 = 0;
    if (r1 > H - 1) r1 = H - 1;
    if (r0 > r1) return 0;

    int c0, nc;
    if (inside) {
        c0 = 0; nc = W;
    } else {
        /* the polygon's xy-shadow misses the origin, so it spans less than pi in azimuth: the
         * extreme vertices follow from the signs of cross products, one arctangent each,
         * relative to the centre direction */
        float gc = or_contract_atan2f(C.y, C.x);
        float xmin = P[0].x, ymin = P[0].y, xmax = P[0].x, ymax = P[0].y;
        for (int i = 1; i < nv; ++i) {
            if (xmax * P[i].y - ymax * P[i].x > 0.0f) { xmax = P[i].x; ymax = P[i].y; }
            if (xmin * P[i].y - ymin * P[i].x < 0.0f) { xmin = P[i].x; ymin = P[i].y; }
        }
        float dmax = or_contract_atan2f(C.x * ymax - C.y * xmax, C.x * xmax + C.y * ymax);
        float dmin = or_contract_atan2f(C.x * ymin - C.y * xmin, C.x * xmin + C.y * ymin);
        float glo = gc + dmin, ghi = gc + dmax;
        float kc = (float)W / C_TWO_PI;
        float uf = ((C_PI - ghi) * kc - 0.5f) - eps;
        float ul = ((C_PI - glo) * kc - 0.5f) + eps;
        int cf = (int)ceilf(uf), cl = (int)floorf(ul);
        if (cf > cl) return 0;
        nc = cl - cf + 1;
        if (nc >= W) { c0 = 0; nc = W; }
        else c0 = ((cf % W) + W) % W;
    }

    int TC = (W + tw - 1) / tw;
    int tr0 = r0 / th, tr1 = r1 / th;
    int tc0, ntc;
    if (nc == W) { tc0 = 0; ntc = TC; }
    else {
        int cl2 = c0 + nc - 1;
        tc0 = c0 / tw;
        int tc1 = cl2 < W ? cl2 / tw : TC + (cl2 - W) / tw;
        ntc = tc1 - tc0 + 1;
        if (ntc >= TC) { tc0 = 0; ntc = TC; }
    }
    pix[0] = r0; pix[1] = r1; pix[2] = c0; pix[3] = nc;
    til[0] = tr0; til[1] = tr1; til[2] = tc0; til[3] = ntc;
    return (tr1 - tr0 + 1) * ntc;
}

/* The binary32 contract for n primitives in one view (o = 1/(1 + exp(-logit)) in the
 * contract's arithmetic feeds the contributing region of the bounding box).
 * kappa: f32 centre range |b_c| (the range the per-tile lists are sorted by,
 * Sec. 3.2.1); flip: -1 when the sensor-frame normal R_cw t_n points away from
 * the sensor ((n . b_c) > 0) and flip_normals is set, else +1; pix_rect, tile_rect,
 * count as in contract_bbox.  valid[i] = 0 marks a non-finite input or a zero
 * quaternion (count 0). */
void or_project_contract(int64_t n, const float *pos_logit, const float *quat,
                         const float *log_scale, const double *T_ws,
                         int rows, int cols, float elev_min, float elev_max,
                         int tile_h, int tile_w, float sigma_cut, float alpha_min,
                         int flip_normals, float *kappa, int8_t *flip, int32_t *pix_rect,
                         int32_t *tile_rect, int32_t *count, uint8_t *valid)
{
    double Rd[9], td[3];
    or_pose_inverse(T_ws, Rd, td);
    float Rf[9], tf[3];
    for (int k = 0; k < 9; ++k) Rf[k] = (float)Rd[k];
    for (int k = 0; k < 3; ++k) tf[k] = (float)td[k];
    for (int64_t i = 0; i < n; ++i) {
        f3 ba, bb, bc, nr;
        int ok = contract_vectors(pos_logit + 4 * i, quat + 4 * i, log_scale + 2 * i,
                                  Rf, tf, &ba, &bb, &bc, &nr);
        valid[i] = (uint8_t)ok;
        for (int k = 0; k < 4; ++k) { pix_rect[4 * i + k] = 0; tile_rect[4 * i + k] = 0; }
        if (!ok) { kappa[i] = 0.0f; flip[i] = 1; count[i] = 0; continue; }
        float dot = (nr.x * bc.x + nr.y * bc.y) + nr.z * bc.z;
        flip[i] = (flip_normals && dot > 0.0f) ? (int8_t)-1 : (int8_t)1;
        kappa[i] = sqrtf((bc.x * bc.x + bc.y * bc.y) + bc.z * bc.z);
        float oc = 1.0f / (1.0f + or_contract_expf(-pos_logit[4 * i + 3]));
        count[i] = contract_bbox(ba, bb, bc, oc, alpha_min, sigma_cut, rows, cols, elev_min,
                                 elev_max, tile_h, tile_w, pix_rect + 4 * i, tile_rect + 4 * i);
    }
}

/* ------------------------------------------------------------------------- */
/* 3. per-tile lists                                                         */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t key; uint32_t id; } or_pair;

static int pair_cmp(const void *a, const void *b)
{
    const or_pair *x = (const or_pair *)a, *y = (const or_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Every (tile, primitive) pair of one view as key = (tile_offset + tile) << 32
 * | bits(kappa), value = primitive id, sorted by (key, id).  Tiles are numbered
 * row-major, tile = tile_row * TC + tile_col.  Returns the number of pairs, or
 * -1 if it exceeds cap (nothing written past cap). */
int64_t or_bin(int64_t n, const float *kappa, const int32_t *tile_rect,
               const int32_t *count, int rows, int cols, int tile_h, int tile_w,
               int64_t tile_offset, uint64_t *keys_out, uint32_t *ids_out, int64_t cap)
{
    (void)rows; (void)tile_h;
    int TC = (cols + tile_w - 1) / tile_w;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) m += count[i];
    if (m > cap) return -1;
    or_pair *buf = (or_pair *)malloc(sizeof(or_pair) * (size_t)(m > 0 ? m : 1));
    int64_t j = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (count[i] == 0) continue;
        const int32_t *t = tile_rect + 4 * i;
        for (int tr = t[0]; tr <= t[1]; ++tr)
            for (int k = 0; k < t[3]; ++k) {
                int tc = (t[2] + k) % TC;
                uint64_t tile = (uint64_t)(tile_offset + (int64_t)tr * TC + tc);
                buf[j].key = (tile << 32) | f32_bits(kappa[i]);
                buf[j].id = (uint32_t)i;
                ++j;
            }
    }
    qsort(buf, (size_t)m, sizeof(or_pair), pair_cmp);
    for (int64_t k = 0; k < m; ++k) { keys_out[k] = buf[k].key; ids_out[k] = buf[k].id; }
    free(buf);
    return m;
}

/* [start, end) of every tile t in [tile_offset, tile_offset + n_tiles) in a
 * sorted key list; empty tiles get start = end = 0. */
void or_tile_ranges(int64_t m, const uint64_t *keys, int64_t tile_offset,
                    int64_t n_tiles, int64_t *start, int64_t *end)
{
    for (int64_t t = 0; t < n_tiles; ++t) { start[t] = 0; end[t] = 0; }
    for (int64_t k = 0; k < m; ++k) {
        int64_t t = (int64_t)(keys[k] >> 32) - tile_offset;
        if (t < 0 || t >= n_tiles) continue;
        if (k == 0 || (keys[k - 1] >> 32) != (keys[k] >> 32)) start[t] = k;
        if (k == m - 1 || (keys[k + 1] >> 32) != (keys[k] >> 32)) end[t] = k + 1;
    }
}

/* Composite order for brute mode: indices of all primitives sorted by
 * (kappa, id) -- the range sort of Sec. 3.2.1 applied to one list. */
void or_sort_order(int64_t n, const float *kappa, int32_t *order)
{
    or_pair *buf = (or_pair *)malloc(sizeof(or_pair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { buf[i].key = f32_bits(kappa[i]); buf[i].id = (uint32_t)i; }
    qsort(buf, (size_t)n, sizeof(or_pair), pair_cmp);
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)buf[i].id;
    free(buf);
}

/* ------------------------------------------------------------------------- */
/* 4. FP64 render                                                            */
/* ------------------------------------------------------------------------- */

typedef struct {
    double ba[3], bb[3], bc[3], n[3];   /* sensor frame (Supp. D: T = T^c_w H) */
    double o, s[2], q[4], qlen, R[9];   /* q normalised; R row-major, columns t_a, t_b, t_n */
    double Rcw[9];
    int flip;
} or_prim;

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* R(q) for unit q = (w, x, y, z); row-major. */
static void quat_to_R(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Per primitive: o, mu, R = (t_a, t_b, t_n), S; then T^c_w H -> b_a, b_b, b_c
 * (Sec. 3.2 Eq. world_T_splat, Supp. D) and n = flip * R_cw t_n. */
static void prep_prims(int64_t n, const double *pos, const double *logit, const double *quat,
                       const double *log_scale, const int8_t *flip, const double *T_ws,
                       or_prim *P)
{
    double Rcw[9], tcw[3];
    or_pose_inverse(T_ws, Rcw, tcw);
    for (int64_t i = 0; i < n; ++i) {
        or_prim *p = &P[i];
        const double *q = quat + 4 * i;
        double ql = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        p->qlen = ql;
        for (int k = 0; k < 4; ++k) p->q[k] = ql > 0 ? q[k] / ql : (k == 0);
        quat_to_R(p->q, p->R);
        p->s[0] = exp(log_scale[2 * i]);
        p->s[1] = exp(log_scale[2 * i + 1]);
        p->o = 1.0 / (1.0 + exp(-logit[i]));
        p->flip = flip ? flip[i] : 1;
        memcpy(p->Rcw, Rcw, sizeof Rcw);
        double ta[3] = { p->R[0], p->R[3], p->R[6] };
        double tb[3] = { p->R[1], p->R[4], p->R[7] };
        double tn[3] = { p->R[2], p->R[5], p->R[8] };
        const double *mu = pos + 3 * i;
        for (int r = 0; r < 3; ++r) {
            const double *row = Rcw + 3 * r;
            p->ba[r] = p->s[0] * dot3(row, ta);
            p->bb[r] = p->s[1] * dot3(row, tb);
            p->bc[r] = dot3(row, mu) + tcw[r];
            p->n[r] = p->flip * dot3(row, tn);
        }
    }
}

typedef struct {
    double alpha_min, alpha_max, t_min, sigma;
    double band_box, band_alpha, band_t, band_front, band_clamp;
} or_cfg;

typedef struct {
    int32_t k;                /* primitive index */
    double alpha, G, T;       /* T = A_k, transmittance before k */
    int clamped;
    double s[2], p[3], ha[3], hb[3], nu[3], d;
} or_contrib;

/* Pixel ray of (r, c) and its two planes (Sec. 3.2.2):
 * h_x = v x u_z / |v x u_z|, h_y = h_x x v. */
static void pixel_ray(int r, int c, int H, int W, double emin, double emax,
                      double *v, double *hx, double *hy)
{
    double g = OR_PI - 2.0 * OR_PI * (c + 0.5) / W;
    double th = H > 1 ? emax - r * (emax - emin) / (H - 1) : emax;
    v[0] = cos(th) * cos(g); v[1] = cos(th) * sin(g); v[2] = sin(th);
    double uz[3] = { 0, 0, 1 }, t[3];
    cross3(v, uz, t);
    double l = sqrt(dot3(t, t));
    hx[0] = t[0] / l; hx[1] = t[1] / l; hx[2] = t[2] / l;
    cross3(hx, v, hy);
}

static int near_thr(double q, double thr, double band) { return fabs(q - thr) <= band; }

/* Front-to-back composite of one pixel over the primitive indices list[0..len)
 * (already in range order).  Fills D, N, O, T; records contributors if out
 * != NULL; sets band bits for decisions that lie near a threshold:
 * 1 box edge, 2 alpha_min, 4 stop on t_min, 8 behind/in-front sign,
 * 16 alpha_max clamp. */
static int composite_pixel(const or_prim *P, const int32_t *list, int64_t len,
                           const double *v, const double *hx, const double *hy,
                           const or_cfg *cf, double *D, double *N, double *O, double *Tout,
                           uint8_t *band, or_contrib **out, int64_t *out_cap)
{
    double T = 1.0, d_acc = 0, n_acc[3] = { 0, 0, 0 }, o_acc = 0;
    int ncontrib = 0;
    uint8_t bf = 0;
    for (int64_t j = 0; j < len; ++j) {
        const or_prim *p = &P[list[j]];
        /* planes into splat space: h_a = T^T h_x, h_b = T^T h_y */
        double ha[3] = { dot3(hx, p->ba), dot3(hx, p->bb), dot3(hx, p->bc) };
        double hb[3] = { dot3(hy, p->ba), dot3(hy, p->bb), dot3(hy, p->bc) };
        double ph[3];
        cross3(ha, hb, ph);
        if (ph[2] == 0.0) continue;
        double s[2] = { ph[0] / ph[2], ph[1] / ph[2] };
        double smax = fmax(fabs(s[0]), fabs(s[1]));
        if (near_thr(smax, cf->sigma, cf->band_box * cf->sigma)) bf |= 1;
        if (smax > cf->sigma) continue;
        double nu[3];
        for (int k = 0; k < 3; ++k) nu[k] = s[0] * p->ba[k] + s[1] * p->bb[k] + p->bc[k];
        double d = sqrt(dot3(nu, nu));
        double nv = dot3(nu, v);
        if (fabs(nv) <= cf->band_front * d) bf |= 8;
        if (nv <= 0.0) continue;
        double G = exp(-0.5 * (s[0] * s[0] + s[1] * s[1]));
        double a_raw = p->o * G;
        int clamped = a_raw > cf->alpha_max;
        if (near_thr(a_raw, cf->alpha_max, cf->band_clamp)) bf |= 16;
        double a = clamped ? cf->alpha_max : a_raw;
        if (near_thr(a, cf->alpha_min, cf->band_alpha)) bf |= 2;
        if (a < cf->alpha_min) continue;
        double tt = T * (1.0 - a);
        if (near_thr(tt, cf->t_min, cf->band_t * cf->t_min)) bf |= 4;
        if (tt < cf->t_min) break;
        double w = a * T;
        if (out) {
            if (ncontrib >= *out_cap) {
                *out_cap = *out_cap * 2 + 64;
                *out = (or_contrib *)realloc(*out, sizeof(or_contrib) * (size_t)*out_cap);
            }
            or_contrib *c = &(*out)[ncontrib];
            c->k = list[j]; c->alpha = a; c->G = G; c->T = T; c->clamped = clamped;
            c->s[0] = s[0]; c->s[1] = s[1];
            memcpy(c->p, ph, sizeof ph); memcpy(c->ha, ha, sizeof ha); memcpy(c->hb, hb, sizeof hb);
            memcpy(c->nu, nu, sizeof nu); c->d = d;
        }
        d_acc += w * d;
        for (int k = 0; k < 3; ++k) n_acc[k] += w * p->n[k];
        o_acc += w;
        T = tt;
        ++ncontrib;
    }
    *D = d_acc; N[0] = n_acc[0]; N[1] = n_acc[1]; N[2] = n_acc[2]; *O = o_acc; *Tout = T;
    if (band) *band = bf;
    return ncontrib;
}

static void set_cfg(or_cfg *c, const double *cfg, const double *band)
{
    c->alpha_min = cfg[0]; c->alpha_max = cfg[1]; c->t_min = cfg[2]; c->sigma = cfg[3];
    c->band_box = band ? band[0] : 0; c->band_alpha = band ? band[1] : 0;
    c->band_t = band ? band[2] : 0; c->band_front = band ? band[3] : 0;
    c->band_clamp = band ? band[4] : 0;
}

/* Which list a pixel composites: brute mode (tile_start == NULL) uses the
 * given order of all primitives; culled mode uses its tile's sorted list. */
static void pixel_list(int r, int c, int W, int tile_h, int tile_w,
                       const int32_t *order, int64_t n_order,
                       const int64_t *tile_start, const int64_t *tile_end,
                       const int32_t *tile_ids, const int32_t **list, int64_t *len)
{
    if (!tile_start) { *list = order; *len = n_order; return; }
    int TC = (W + tile_w - 1) / tile_w;
    int64_t t = (int64_t)(r / tile_h) * TC + c / tile_w;
    *list = tile_ids + tile_start[t];
    *len = tile_end[t] - tile_start[t];
}

/* FP64 forward render of one view.
 * cfg = {alpha_min, alpha_max, t_min, sigma_cut}; band = 5 band widths (see
 * composite_pixel) or NULL.  Outputs are H*W (N planar 3*H*W). */
void or_render(int64_t n, const double *pos, const double *logit, const double *quat,
               const double *log_scale, const int8_t *flip,
               const int32_t *order, int64_t n_order,
               const int64_t *tile_start, const int64_t *tile_end, const int32_t *tile_ids,
               const double *T_ws, int rows, int cols, double elev_min, double elev_max,
               int tile_h, int tile_w, const double *cfg, const double *band,
               const int32_t *pixels, int64_t n_pixels,
               double *D, double *N, double *O, double *T_final, int32_t *n_contrib,
               uint8_t *band_flags, int n_threads)
{
    or_prim *P = (or_prim *)malloc(sizeof(or_prim) * (size_t)(n > 0 ? n : 1));
    prep_prims(n, pos, logit, quat, log_scale, flip, T_ws, P);
    or_cfg cf;
    set_cfg(&cf, cfg, band);
    int64_t npx = pixels ? n_pixels : (int64_t)rows * cols;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t px = 0; px < npx; ++px) {
        int r = pixels ? pixels[2 * px] : (int)(px / cols);
        int c = pixels ? pixels[2 * px + 1] : (int)(px % cols);
        double v[3], hx[3], hy[3];
        pixel_ray(r, c, rows, cols, elev_min, elev_max, v, hx, hy);
        const int32_t *list; int64_t len;
        pixel_list(r, c, cols, tile_h, tile_w, order, n_order, tile_start, tile_end,
                   tile_ids, &list, &len);
        double Np[3];
        n_contrib[px] = composite_pixel(P, list, len, v, hx, hy, &cf, &D[px], Np, &O[px],
                                        &T_final[px], band_flags ? &band_flags[px] : NULL,
                                        NULL, NULL);
        N[px] = Np[0]; N[npx + px] = Np[1]; N[2 * npx + px] = Np[2];
    }
    free(P);
}

/* Every (pixel, primitive) pair whose ray reaches the primitive, tested one
 * by one with no compositing: p_z != 0, max|s_hat| <= sigma_cut, hit in
 * front, alpha >= alpha_min.  Writes up to cap pairs (pixel index r*W + c,
 * primitive) and returns the total number found. */
int64_t or_reach_pairs(int64_t n, const double *pos, const double *logit, const double *quat,
                       const double *log_scale, const double *T_ws, int rows, int cols,
                       double elev_min, double elev_max, const double *cfg,
                       int64_t *pix_out, int32_t *prim_out, int64_t cap)
{
    or_prim *P = (or_prim *)malloc(sizeof(or_prim) * (size_t)(n > 0 ? n : 1));
    prep_prims(n, pos, logit, quat, log_scale, NULL, T_ws, P);
    or_cfg cf;
    set_cfg(&cf, cfg, NULL);
    int64_t found = 0;
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) {
            double v[3], hx[3], hy[3];
            pixel_ray(r, c, rows, cols, elev_min, elev_max, v, hx, hy);
            for (int64_t i = 0; i < n; ++i) {
                const or_prim *p = &P[i];
                double ha[3] = { dot3(hx, p->ba), dot3(hx, p->bb), dot3(hx, p->bc) };
                double hb[3] = { dot3(hy, p->ba), dot3(hy, p->bb), dot3(hy, p->bc) };
                double ph[3];
                cross3(ha, hb, ph);
                if (ph[2] == 0.0) continue;
                double s0 = ph[0] / ph[2], s1 = ph[1] / ph[2];
                if (fmax(fabs(s0), fabs(s1)) > cf.sigma) continue;
                double nu[3];
                for (int k = 0; k < 3; ++k) nu[k] = s0 * p->ba[k] + s1 * p->bb[k] + p->bc[k];
                if (dot3(nu, v) <= 0.0) continue;
                double a = fmin(p->o * exp(-0.5 * (s0 * s0 + s1 * s1)), cf.alpha_max);
                if (a < cf.alpha_min) continue;
                if (found < cap) { pix_out[found] = (int64_t)r * cols + c; prim_out[found] = (int32_t)i; }
                ++found;
            }
        }
    free(P);
    return found;
}

/* ------------------------------------------------------------------------- */
/* 5. FP64 analytic backward (Supp. D.2)                                     */
/* ------------------------------------------------------------------------- */

/* dR/dq for unit q: contract G (row-major 3x3, dL/dR) with the derivative of
 * each entry of R(q) with respect to w, x, y, z. */
static void dR_dq(const double *q, const double *G, double *gq)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    /* rows: d/dw, d/dx, d/dy, d/dz of R (row-major) */
    double dw[9] = { 0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0 };
    double dx[9] = { 0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x };
    double dy[9] = { -4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y };
    double dz[9] = { -4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0 };
    gq[0] = gq[1] = gq[2] = gq[3] = 0;
    for (int k = 0; k < 9; ++k) {
        gq[0] += G[k] * dw[k]; gq[1] += G[k] * dx[k];
        gq[2] += G[k] * dy[k]; gq[3] += G[k] * dz[k];
    }
}

/* Gradient of L = sum_px gD D + gN . N + gO O with respect to the FP64
 * parameters.  Outputs: g_pos 3n, g_logit n, g_quat 4n, g_log_scale 2n and the
 * sensor-frame intermediates g_b 9n (b_a, b_b, b_c), g_n 3n, g_o n. */
void or_render_backward(int64_t n, const double *pos, const double *logit, const double *quat,
                        const double *log_scale, const int8_t *flip,
                        const int32_t *order, int64_t n_order,
                        const int64_t *tile_start, const int64_t *tile_end, const int32_t *tile_ids,
                        const double *T_ws, int rows, int cols, double elev_min, double elev_max,
                        int tile_h, int tile_w, const double *cfg,
                        const int32_t *pixels, int64_t n_pixels,
                        const double *gD, const double *gN, const double *gO,
                        double *g_pos, double *g_logit, double *g_quat, double *g_log_scale,
                        double *g_b, double *g_n, double *g_o, int n_threads)
{
    or_prim *P = (or_prim *)malloc(sizeof(or_prim) * (size_t)(n > 0 ? n : 1));
    prep_prims(n, pos, logit, quat, log_scale, flip, T_ws, P);
    or_cfg cf;
    set_cfg(&cf, cfg, NULL);
    int64_t npx = pixels ? n_pixels : (int64_t)rows * cols;
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    /* per-thread accumulators of 13 values per primitive: g_ba, g_bb, g_bc, g_n, g_o */
    double *acc = (double *)calloc((size_t)nt * (size_t)(n > 0 ? n : 1) * 13, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *A = acc + (size_t)tid * (size_t)n * 13;
        or_contrib *buf = NULL;
        int64_t cap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t px = 0; px < npx; ++px) {
            {
                int r = pixels ? pixels[2 * px] : (int)(px / cols);
                int c = pixels ? pixels[2 * px + 1] : (int)(px % cols);
                double v[3], hx[3], hy[3];
                pixel_ray(r, c, rows, cols, elev_min, elev_max, v, hx, hy);
                const int32_t *list; int64_t len;
                pixel_list(r, c, cols, tile_h, tile_w, order, n_order, tile_start, tile_end,
                           tile_ids, &list, &len);
                double Dp, Np[3], Op, Tp;
                int m = composite_pixel(P, list, len, v, hx, hy, &cf, &Dp, Np, &Op, &Tp, NULL,
                                        &buf, &cap);
                double gd = gD[px], gn[3] = { gN[px], gN[npx + px], gN[2 * npx + px] }, go = gO[px];
                /* B_{.,k} = sum_{i>k} x_i alpha_i A_i, accumulated back to front */
                double Bd = 0, Bn[3] = { 0, 0, 0 }, Bo = 0;
                for (int j = m - 1; j >= 0; --j) {
                    const or_contrib *ck = &buf[j];
                    const or_prim *p = &P[ck->k];
                    double a = ck->alpha, Ak = ck->T, om = 1.0 - a;
                    double dD = ck->d * Ak - Bd / om;
                    double dO = Ak - Bo / om;
                    double gA = gd * dD + go * dO;
                    for (int k = 0; k < 3; ++k) gA += gn[k] * (p->n[k] * Ak - Bn[k] / om);
                    double w = a * Ak;
                    Bd += ck->d * w; Bo += w;
                    for (int k = 0; k < 3; ++k) Bn[k] += p->n[k] * w;
                    double gdk = gd * w;            /* dL/dd_k */
                    double *Ak13 = A + (size_t)ck->k * 13;
                    for (int k = 0; k < 3; ++k) Ak13[9 + k] += gn[k] * w;  /* dL/dn_k */
                    double gAe = ck->clamped ? 0.0 : gA;
                    Ak13[12] += gAe * ck->G;                               /* dL/do */
                    /* dL/ds_hat: density term and range term */
                    double gs[2];
                    for (int k = 0; k < 2; ++k) {
                        const double *bk = k == 0 ? p->ba : p->bb;
                        gs[k] = -gAe * a * ck->s[k] + gdk * dot3(ck->nu, bk) / ck->d;
                    }
                    /* dL/dp_hat, s_hat = (p_x/p_z, p_y/p_z) */
                    double pz = ck->p[2];
                    double gp[3] = { gs[0] / pz, gs[1] / pz,
                                     -(ck->p[0] * gs[0] + ck->p[1] * gs[1]) / (pz * pz) };
                    /* rho_a = g_p x h_a = dL/dh_b ; rho_b = g_p x h_b = -dL/dh_a */
                    double ra[3], rb[3];
                    cross3(gp, ck->ha, ra);
                    cross3(gp, ck->hb, rb);
                    for (int k = 0; k < 3; ++k) {
                        double nd = ck->nu[k] / ck->d;
                        Ak13[0 + k] += -rb[0] * hx[k] + ra[0] * hy[k] + gdk * ck->s[0] * nd;
                        Ak13[3 + k] += -rb[1] * hx[k] + ra[1] * hy[k] + gdk * ck->s[1] * nd;
                        Ak13[6 + k] += -rb[2] * hx[k] + ra[2] * hy[k] + gdk * nd;
                    }
                }
            }
        }
        free(buf);
    }
    /* reduce threads, then chain to the parameters */
    for (int64_t i = 0; i < n; ++i) {
        double s13[13] = { 0 };
        for (int t = 0; t < nt; ++t)
            for (int k = 0; k < 13; ++k) s13[k] += acc[((size_t)t * (size_t)n + (size_t)i) * 13 + k];
        const or_prim *p = &P[i];
        for (int k = 0; k < 9; ++k) g_b[9 * i + k] = s13[k];
        for (int k = 0; k < 3; ++k) g_n[3 * i + k] = s13[9 + k];
        g_o[i] = s13[12];
        const double *Rcw = p->Rcw;
        double gta[3], gtb[3], gtn[3], gmu[3];
        for (int j = 0; j < 3; ++j) {   /* R_cw^T g */
            gmu[j] = Rcw[j] * s13[6] + Rcw[3 + j] * s13[7] + Rcw[6 + j] * s13[8];
            gta[j] = p->s[0] * (Rcw[j] * s13[0] + Rcw[3 + j] * s13[1] + Rcw[6 + j] * s13[2]);
            gtb[j] = p->s[1] * (Rcw[j] * s13[3] + Rcw[3 + j] * s13[4] + Rcw[6 + j] * s13[5]);
            gtn[j] = p->flip * (Rcw[j] * s13[9] + Rcw[3 + j] * s13[10] + Rcw[6 + j] * s13[11]);
        }
        for (int k = 0; k < 3; ++k) g_pos[3 * i + k] = gmu[k];
        /* dL/ds_a = g_ba . (R_cw t_a) = g_ba . b_a / s_a ; d/dlog s = s d/ds */
        g_log_scale[2 * i] = dot3(s13 + 0, p->ba);
        g_log_scale[2 * i + 1] = dot3(s13 + 3, p->bb);
        g_logit[i] = s13[12] * p->o * (1.0 - p->o);
        double G[9];
        for (int r = 0; r < 3; ++r) { G[3 * r + 0] = gta[r]; G[3 * r + 1] = gtb[r]; G[3 * r + 2] = gtn[r]; }
        double gqn[4];
        dR_dq(p->q, G, gqn);
        double qg = 0;
        for (int k = 0; k < 4; ++k) qg += p->q[k] * gqn[k];
        for (int k = 0; k < 4; ++k)
            g_quat[4 * i + k] = p->qlen > 0 ? (gqn[k] - p->q[k] * qg) / p->qlen : 0.0;
    }
    free(acc);
    free(P);
}

/* Gradient with respect to the sensor pose, from the per-primitive sensor-frame gradients of
 * or_render_backward.  The world-to-sensor transform enters only through b_a = s_a R t_a,
 * b_b = s_b R t_b, b_c = R mu + t and n = +-R t_n (Supp. D.1; the tracking step of Sec. 3.3
 * optimises this pose).  Perturbing it on the left, T^c_w <- exp(xi^) T^c_w with
 * xi = (rho, omega) in the sensor frame, moves every point as b_c + omega x b_c + rho and every
 * direction as b + omega x b, so
 *   dL/drho = sum_i g_bc,i,
 *   dL/domega = sum_i (b_c,i x g_bc,i + b_a,i x g_ba,i + b_b,i x g_bb,i + n_i x g_n,i).
 * g_b is n x 9 (g_ba, g_bb, g_bc), g_n is n x 3; out = (dL/drho, dL/domega). */
void or_pose_gradient(int64_t n, const double *pos, const double *logit, const double *quat,
                      const double *log_scale, const int8_t *flip, const double *T_ws,
                      const double *g_b, const double *g_n, double *out)
{
    or_prim *P = (or_prim *)malloc(sizeof(or_prim) * (size_t)(n > 0 ? n : 1));
    prep_prims(n, pos, logit, quat, log_scale, flip, T_ws, P);
    for (int k = 0; k < 6; ++k) out[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const or_prim *p = &P[i];
        const double *ga = g_b + 9 * i, *gb = g_b + 9 * i + 3, *gc = g_b + 9 * i + 6;
        const double *gn = g_n + 3 * i;
        double c1[3], c2[3], c3[3], c4[3];
        cross3(p->bc, gc, c1);
        cross3(p->ba, ga, c2);
        cross3(p->bb, gb, c3);
        cross3(p->n, gn, c4);
        for (int k = 0; k < 3; ++k) {
            out[k] += gc[k];
            out[3 + k] += c1[k] + c2[k] + c3[k] + c4[k];
        }
    }
    free(P);
}

/* ------------------------------------------------------------------------- */
/* 6. loss and Adam                                                          */
/* ------------------------------------------------------------------------- */

/* L = sum_{valid} |D - Dt| + lambda_n (1 - N . Nt) + lambda_o (-log max(O, o_eps))
 * over pixels with Dt > 0 (the valid mask M_v), with its per-pixel gradients
 * (sign(0) = 0; d/dO is -lambda_o / O where O > o_eps, else 0). */
double or_loss(int64_t npx, const double *D, const double *N, const double *O,
               const double *Dt, const double *Nt, double lambda_n, double lambda_o,
               double o_eps, double rho_exp, double *gD, double *gN, double *gO)
{
    double L = 0;
    for (int64_t i = 0; i < npx; ++i) {
        gD[i] = 0; gO[i] = 0;
        for (int k = 0; k < 3; ++k) gN[k * npx + i] = 0;
        if (!(Dt[i] > 0)) continue;
        /* rho_d of Eq. loss_range, a weight that depends on the measured range: Dt^rho_exp */
        double rho = rho_exp == 0.0 ? 1.0 : pow(Dt[i], rho_exp);
        double e = D[i] - Dt[i];
        L += rho * fabs(e);
        gD[i] = rho * (e > 0 ? 1.0 : (e < 0 ? -1.0 : 0.0));
        double dn = 0;
        for (int k = 0; k < 3; ++k) dn += N[k * npx + i] * Nt[k * npx + i];
        L += lambda_n * (1.0 - dn);
        for (int k = 0; k < 3; ++k) gN[k * npx + i] = -lambda_n * Nt[k * npx + i];
        if (lambda_o != 0) {
            double o = O[i] > o_eps ? O[i] : o_eps;
            L += lambda_o * (-log(o));
            gO[i] = O[i] > o_eps ? -lambda_o / O[i] : 0.0;
        }
    }
    return L;
}

/* Adam (bias-corrected), step = 1 for the first update. */
void or_adam(int64_t n, double *p, const double *g, double *m, double *v,
             double lr, double b1, double b2, double eps, int step)
{
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1 - b1) * g[i];
        v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
