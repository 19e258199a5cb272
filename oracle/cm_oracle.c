/*
 * cm_oracle.c -- plain, slow CPU oracle for the contrast-maximisation (CM)
 * loss and its gradient, written from the paper (arXiv 2412.06359,
 * "On-Device Self-Supervised Learning of Low-Latency Monocular Depth from
 * Only Events").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline / reference legs of bench.py load this library.  The product (the
 * CUDA library under paper_2412_06359_gb300/) never calls it, and the two share
 * no code, header or table.
 *
 * What it computes, step by step, in the order of the paper:
 *   S1  flow from inverse depth and 6-DoF ego-motion (Sec. 3.2, Eq. 2, taken
 *       in its instantaneous form: the rigid motion field with intrinsics)
 *   S2  every event pushed bin by bin to the bin edges, re-sampling the flow
 *       bilinearly at its current position (Sec. 3.1 iterative warp, Sec. 3.3)
 *   S3  an event that leaves the image at any computed point is masked out of
 *       every image of warped events (Sec. 3.1 regularisation, Fig. 2)
 *   S4  bilinear splat into polarity-split IWEs of counts and timestamp sums
 *       (Sec. 3.1, kernel kappa of Eq. 1)
 *   S5  per reference time: the squared average-timestamp images summed over
 *       pixels and both polarities, scaled by the number of non-empty pixels,
 *       averaged over the references (Eq. 1 and the text after it)
 *   S6  the exact derivative of S2-S5 with respect to the flow (Sec. 3.3,
 *       backward pass), on the branch selected by the floor / mask / support
 *       decisions, with the right-derivative at integer coordinates
 *   S7  the chain from the flow gradient to inverse depth and ego-motion
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes of the repository):
 *   - average timestamp of event k at reference tau_r: 1 - |tau_r - tau_k|,
 *     with time normalised to the window, tau = (t - t0) / (t1 - t0)
 *   - T_p(x) = S_p(x) / (C_p(x) + eps); loss at reference r:
 *       L_r = sum_x (T_+(x)^2 + T_-(x)^2) / (N_nz(r) + eps),
 *     N_nz(r) = number of pixels with a splat contribution of either polarity;
 *       L = (1/R) sum_r L_r
 *   - bin of an event: b = min(floor(tau * B), B - 1); bin edges tau_j = j / B;
 *     references: the window end only (R = 1) or all B + 1 edges (R = B + 1)
 *   - pixel centres at integers, image interval closed: 0 <= x <= W-1
 *   - flow sampled with clamped corner indices (the clamped corner always has
 *     weight zero inside the closed image)
 *   - positions: either FP64 throughout (pos_f32 = 0; the plain definition) or
 *     in FP32 with the fixed sequence of correctly rounded operations of the
 *     GPU kernels (pos_f32 = 1).  The floor of a position decides the cell, the
 *     support and the mask, and the eps-regularised ratio makes the loss and
 *     its gradient sensitive to sub-ULP position changes, so parity against an
 *     FP32 kernel takes those decisions in FP32 (the kernel's precision).  All
 *     other arithmetic is FP64 in both modes.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math; the
 * FP32 position path relies on IEEE single precision with no contraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_REF_END 0      /* one reference time, at the window end */
#define ORC_REF_ALL 1      /* all bin edges j = 0..B */
#define ORC_MAX_BINS 64

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------- */
/* S1: flow from inverse depth and ego-motion (Sec. 3.2, Eq. 2)               */
/* ------------------------------------------------------------------------- */

/*
 * Rigid motion field of a static scene seen by a camera moving with linear
 * velocity v and angular velocity w (camera frame, x right, y down, z forward):
 * for normalised coordinates xn = (u - cx)/fx, yn = (v - cy)/fy and inverse
 * depth rho,
 *   d(xn)/dt = rho (-vx + xn vz) + xn yn wx - (1 + xn^2) wy + yn wz
 *   d(yn)/dt = rho (-vy + yn vz) + (1 + yn^2) wx - xn yn wy - xn wz
 * and the flow over a window of length dt in pixels is
 *   flow = dt * (fx d(xn)/dt, fy d(yn)/dt).
 * This is the first-order (dt -> 0) form of Eq. 2, x' ~ K P D(x) K^-1 x.
 * ego = (vx, vy, vz, wx, wy, wz).  Layout: rho[H][W], flow[H][W][2].
 */
void orc_flow_from_depth(int32_t W, int32_t H, double fx, double fy, double cx, double cy,
                         const double* rho, const double* ego, double dt, double* flow)
{
    const double vx = ego[0], vy = ego[1], vz = ego[2];
    const double wx = ego[3], wy = ego[4], wz = ego[5];
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const double xn = ((double)u - cx) / fx;
            const double yn = ((double)v - cy) / fy;
            const double r = rho[(int64_t)v * W + u];
            const double xdot = r * (-vx + xn * vz) + xn * yn * wx - (1.0 + xn * xn) * wy + yn * wz;
            const double ydot = r * (-vy + yn * vz) + (1.0 + yn * yn) * wx - xn * yn * wy - xn * wz;
            flow[2 * ((int64_t)v * W + u) + 0] = dt * fx * xdot;
            flow[2 * ((int64_t)v * W + u) + 1] = dt * fy * ydot;
        }
    }
}

/*
 * The same motion field in FP32, with the operation sequence that decides the
 * positions of the FP32 trajectory (pos_f32 = 1).  Every operation is one
 * correctly rounded IEEE single operation; fmaf is the fused multiply-add.
 *   ifx = 1/fx, ify = 1/fy, sx = dt*fx, sy = dt*fy
 *   xn = (u - cx) * ifx,  yn = (v - cy) * ify,  xy = xn * yn
 *   xd = rho * fma(xn, vz, -vx);  xd = fma(xy, wx, xd);
 *   xd = fma(-fma(xn, xn, 1), wy, xd);  xd = fma(yn, wz, xd)
 *   yd = rho * fma(yn, vz, -vy);  yd = fma(fma(yn, yn, 1), wx, yd);
 *   yd = fma(-xy, wy, yd);  yd = fma(-xn, wz, yd)
 *   flow = (sx * xd, sy * yd)
 */
void orc_flow_from_depth_f32(int32_t W, int32_t H, float fx, float fy, float cx, float cy,
                             const float* rho, const float* ego, float dt, float* flow)
{
    const float vx = ego[0], vy = ego[1], vz = ego[2];
    const float wx = ego[3], wy = ego[4], wz = ego[5];
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    const float sx = dt * fx, sy = dt * fy;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const float xn = ((float)u - cx) * ifx;
            const float yn = ((float)v - cy) * ify;
            const float r = rho[(int64_t)v * W + u];
            const float xy = xn * yn;
            float xd = r * fmaf(xn, vz, -vx);
            xd = fmaf(xy, wx, xd);
            xd = fmaf(-fmaf(xn, xn, 1.0f), wy, xd);
            xd = fmaf(yn, wz, xd);
            float yd = r * fmaf(yn, vz, -vy);
            yd = fmaf(fmaf(yn, yn, 1.0f), wx, yd);
            yd = fmaf(-xy, wy, yd);
            yd = fmaf(-xn, wz, yd);
            flow[2 * ((int64_t)v * W + u) + 0] = sx * xd;
            flow[2 * ((int64_t)v * W + u) + 1] = sy * yd;
        }
    }
}

/*
 * S7: chain rule from dL/dflow to dL/d(rho) and dL/d(ego) through the motion
 * field above (FP64).  dego is overwritten with the sum over all pixels.
 */
void orc_depth_ego_grad(int32_t W, int32_t H, double fx, double fy, double cx, double cy,
                        const double* rho, const double* ego, double dt, const double* dflow,
                        double* drho, double* dego)
{
    const double vx = ego[0], vy = ego[1], vz = ego[2];
    double g[6] = {0, 0, 0, 0, 0, 0};
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t i = (int64_t)v * W + u;
            const double xn = ((double)u - cx) / fx;
            const double yn = ((double)v - cy) / fy;
            const double r = rho[i];
            /* G = dL/d(xdot, ydot) */
            const double Gx = dt * fx * dflow[2 * i + 0];
            const double Gy = dt * fy * dflow[2 * i + 1];
            if (drho) drho[i] = Gx * (-vx + xn * vz) + Gy * (-vy + yn * vz);
            g[0] += -r * Gx;
            g[1] += -r * Gy;
            g[2] += r * (xn * Gx + yn * Gy);
            g[3] += xn * yn * Gx + (1.0 + yn * yn) * Gy;
            g[4] += -(1.0 + xn * xn) * Gx - xn * yn * Gy;
            g[5] += yn * Gx - xn * Gy;
        }
    }
    for (int i = 0; i < 6; ++i) dego[i] = g[i];
}

/*
 * Eq. 2 literally: x' ~ K [R | t] D(x) K^-1 x, with the camera displaced by
 * (v dt, w dt) over the window, i.e. points map as X' = R X + t with
 * R = Rodrigues(-w dt) and t = -v dt, and depth D = 1 / rho.  Returns the
 * pixel displacement x' - x.  Used to pin the motion field of S1 (the two
 * agree to first order in dt) and as the discrete-flow variant.
 */
static void rodrigues(const double k[3], double Rm[3][3])
{
    const double th = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    double a, b;
    if (th < 1e-12) { a = 1.0; b = 0.5; }
    else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
    const double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
    double K2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[i][j] = 0;
            for (int l = 0; l < 3; ++l) K2[i][j] += K[i][l] * K[l][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rm[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + b * K2[i][j];
}

void orc_flow_eq2(int32_t W, int32_t H, double fx, double fy, double cx, double cy,
                  const double* rho, const double* ego, double dt, double* flow)
{
    const double k[3] = {-ego[3] * dt, -ego[4] * dt, -ego[5] * dt};
    const double t[3] = {-ego[0] * dt, -ego[1] * dt, -ego[2] * dt};
    double Rm[3][3];
    rodrigues(k, Rm);
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t i = (int64_t)v * W + u;
            const double Z = 1.0 / rho[i];
            const double X[3] = {Z * ((double)u - cx) / fx, Z * ((double)v - cy) / fy, Z};
            double Xp[3];
            for (int a = 0; a < 3; ++a) Xp[a] = Rm[a][0] * X[0] + Rm[a][1] * X[1] + Rm[a][2] * X[2] + t[a];
            flow[2 * i + 0] = fx * Xp[0] / Xp[2] + cx - (double)u;
            flow[2 * i + 1] = fy * Xp[1] / Xp[2] + cy - (double)v;
        }
    }
}

/*
 * Eq. 2 with one pose per bin (the discrete-flow variant): bin i of nb moves
 * the camera with velocity v_i and angular velocity w_i (ego[6i .. 6i+5]) for
 * dt_bin seconds, and its flow is `scale` times the pixel displacement of
 * orc_flow_eq2 (scale = nb expresses it in px per window when the nb bins
 * split the window evenly, the unit of the iterative warp).  FP64, the plain
 * definition.  flow is [nb][H][W][2].
 */
void orc_flow_eq2_bins(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho,
                       const double* ego, int32_t nb, double dt_bin, double scale, double* flow)
{
    const int64_t HW = (int64_t)W * H;
    for (int32_t i = 0; i < nb; ++i) {
        double* f = flow + 2 * HW * i;
        orc_flow_eq2(W, H, fx, fy, cx, cy, rho, ego + 6 * i, dt_bin, f);
        for (int64_t q = 0; q < 2 * HW; ++q) f[q] *= scale;
    }
}

/*
 * The same in FP32 with the operation sequence of the GPU kernels, which
 * decides the positions of the FP32 trajectory when these flows drive it
 * (every operation one correctly rounded IEEE single operation, fmaf fused):
 *   per bin:  k = -(w * dt), t = -(v * dt) (componentwise);
 *             kxx = kx*kx, kyy = ky*ky, kzz = kz*kz, kxy = kx*ky, kxz = kx*kz, kyz = ky*kz
 *             s = (kxx + kyy) + kzz
 *             a = sin(th)/th and b = (1 - cos th)/th^2 as their Taylor series in s
 *                 (terms up to s^9, Horner from the highest term: c = fma(c, s, c_n))
 *             R00 = fma(b, -(kyy + kzz), 1)   R01 = fma(b, kxy, -(a*kz))   R02 = fma(b, kxz, a*ky)
 *             R10 = fma(b, kxy, a*kz)         R11 = fma(b, -(kxx + kzz), 1) R12 = fma(b, kyz, -(a*kx))
 *             R20 = fma(b, kxz, -(a*ky))      R21 = fma(b, kyz, a*kx)      R22 = fma(b, -(kxx + kyy), 1)
 *             Ad_i = b * -(...) (the diagonal of R - I, the same sums as R_ii)
 *   per pixel: xn = (u - cx) * (1/fx), yn = (v - cy) * (1/fy), Z = 1/rho,
 *             the displacement d of disp_f32 below; flow = (scale * d.x, scale * d.y)
 * The displacement is fx (P0/P2 - xn), the same quantity as fx P0/P2 + cx - u.
 */
static const double ORC_SIN_SERIES[10] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0,
                                          -1.0 / 39916800.0, 1.0 / 6227020800.0, -1.0 / 1307674368000.0,
                                          1.0 / 355687428096000.0, -1.0 / 121645100408832000.0};
static const double ORC_COS_SERIES[10] = {1.0 / 2.0, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0,
                                          -1.0 / 479001600.0, 1.0 / 87178291200.0, -1.0 / 20922789888000.0,
                                          1.0 / 6402373705728000.0, -1.0 / 2432902008176640000.0};

static void rot_f32(const float* e, float dt, float Rm[9], float tv[3], float Ad[3])
{
    const float kx = -(e[3] * dt), ky = -(e[4] * dt), kz = -(e[5] * dt);
    tv[0] = -(e[0] * dt);
    tv[1] = -(e[1] * dt);
    tv[2] = -(e[2] * dt);
    const float kxx = kx * kx, kyy = ky * ky, kzz = kz * kz;
    const float kxy = kx * ky, kxz = kx * kz, kyz = ky * kz;
    const float s = (kxx + kyy) + kzz;
    float a = (float)ORC_SIN_SERIES[9], b = (float)ORC_COS_SERIES[9];
    for (int n = 8; n >= 0; --n) {
        a = fmaf(a, s, (float)ORC_SIN_SERIES[n]);
        b = fmaf(b, s, (float)ORC_COS_SERIES[n]);
    }
    Ad[0] = b * -(kyy + kzz);
    Ad[1] = b * -(kxx + kzz);
    Ad[2] = b * -(kxx + kyy);
    Rm[0] = fmaf(b, -(kyy + kzz), 1.0f);
    Rm[1] = fmaf(b, kxy, -(a * kz));
    Rm[2] = fmaf(b, kxz, a * ky);
    Rm[3] = fmaf(b, kxy, a * kz);
    Rm[4] = fmaf(b, -(kxx + kzz), 1.0f);
    Rm[5] = fmaf(b, kyz, -(a * kx));
    Rm[6] = fmaf(b, kxz, -(a * ky));
    Rm[7] = fmaf(b, kyz, a * kx);
    Rm[8] = fmaf(b, -(kxx + kyy), 1.0f);
}

/* The displacement of pixel (u, v) in FP32 (the sequence of the kernels):
 * with m = (xn, yn, 1) and A = R - I (its diagonal built directly),
 *   c_0j = fma(-xn, A_2j, A_0j), c_1j = fma(-yn, A_2j, A_1j)      (j = 0, 1, 2)
 *   s0 = fma(c_00, xn, fma(c_01, yn, c_02)),  s1 = fma(c_10, xn, fma(c_11, yn, c_12))
 *   e0 = fma(Z, s0, fma(-xn, t2, t0)),        e1 = fma(Z, s1, fma(-yn, t2, t1))
 *   P2 = fma(Z, fma(R20, xn, fma(R21, yn, R22)), t2),  iz = 1 / P2
 *   d = (fx * (e0 * iz), fy * (e1 * iz))
 * e0 = P0 - xn P2 taken in this form is exactly 0 for a camera at rest and
 * never cancels two large terms. */
static void disp_f32(const float Rm[9], const float tv[3], const float Ad[3], float xn, float yn, float Z, float fx,
                     float fy, float* dx, float* dy, float* P2out)
{
    const float A00 = Ad[0], A11 = Ad[1], A22 = Ad[2];
    const float c00 = fmaf(-xn, Rm[6], A00), c01 = fmaf(-xn, Rm[7], Rm[1]), c02 = fmaf(-xn, A22, Rm[2]);
    const float c10 = fmaf(-yn, Rm[6], Rm[3]), c11 = fmaf(-yn, Rm[7], A11), c12 = fmaf(-yn, A22, Rm[5]);
    const float s0 = fmaf(c00, xn, fmaf(c01, yn, c02));
    const float s1 = fmaf(c10, xn, fmaf(c11, yn, c12));
    const float e0 = fmaf(Z, s0, fmaf(-xn, tv[2], tv[0]));
    const float e1 = fmaf(Z, s1, fmaf(-yn, tv[2], tv[1]));
    const float P2 = fmaf(Z, fmaf(Rm[6], xn, fmaf(Rm[7], yn, Rm[8])), tv[2]);
    const float iz = 1.0f / P2;
    *dx = fx * (e0 * iz);
    *dy = fy * (e1 * iz);
    *P2out = P2;
}

void orc_flow_eq2_bins_f32(int32_t W, int32_t H, float fx, float fy, float cx, float cy, const float* rho,
                           const float* ego, int32_t nb, float dt_bin, float scale, float* flow)
{
    const int64_t HW = (int64_t)W * H;
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    for (int32_t i = 0; i < nb; ++i) {
        float Rm[9], tv[3], Ad[3];
        rot_f32(ego + 6 * i, dt_bin, Rm, tv, Ad);
        for (int32_t v = 0; v < H; ++v) {
            for (int32_t u = 0; u < W; ++u) {
                const int64_t q = (int64_t)v * W + u;
                const float xn = ((float)u - cx) * ifx;
                const float yn = ((float)v - cy) * ify;
                const float Z = 1.0f / rho[q];
                float dx, dy, P2;
                disp_f32(Rm, tv, Ad, xn, yn, Z, fx, fy, &dx, &dy, &P2);
                flow[2 * (HW * i + q) + 0] = scale * dx;
                flow[2 * (HW * i + q) + 1] = scale * dy;
            }
        }
    }
}

/*
 * Derivative of the Rodrigues rotation R(k) = I + a K + b K^2, K = [k]x,
 * a = sin(th)/th, b = (1 - cos th)/th^2, th = |k|, with respect to k_c:
 *   dR/dk_c = a E_c + b (E_c K + K E_c) + (a'/th K + b'/th K^2) k_c,
 * E_c = [e_c]x, a' = da/dth, b' = db/dth (derived from the formula by the
 * product and chain rules).  Near th = 0 the ratios a'/th -> -1/3 and
 * b'/th -> -1/12 are taken from their series.
 */
static void rodrigues_grad(const double k[3], double dR[3][3][3])
{
    const double th2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double th = sqrt(th2);
    double a, b, ap, bp; /* ap = a'/th, bp = b'/th */
    if (th < 1e-4) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
        ap = -1.0 / 3.0 + th2 / 30.0;
        bp = -1.0 / 12.0 + th2 / 180.0;
    } else {
        const double sn = sin(th), cs = cos(th);
        a = sn / th;
        b = (1.0 - cs) / th2;
        ap = (th * cs - sn) / (th2 * th);
        bp = (th * sn - 2.0 * (1.0 - cs)) / (th2 * th2);
    }
    const double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
    double K2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            K2[i][j] = 0;
            for (int l = 0; l < 3; ++l) K2[i][j] += K[i][l] * K[l][j];
        }
    for (int c = 0; c < 3; ++c) {
        double E[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        /* [e_c]x */
        if (c == 0) { E[1][2] = -1; E[2][1] = 1; }
        if (c == 1) { E[0][2] = 1; E[2][0] = -1; }
        if (c == 2) { E[0][1] = -1; E[1][0] = 1; }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double EK = 0, KE = 0;
                for (int l = 0; l < 3; ++l) {
                    EK += E[i][l] * K[l][j];
                    KE += K[i][l] * E[l][j];
                }
                dR[c][i][j] = a * E[i][j] + b * (EK + KE) + (ap * K[i][j] + bp * K2[i][j]) * k[c];
            }
    }
}

/*
 * Adjoint of orc_flow_eq2_bins: given dL/dflow [nb][H][W][2], dL/d(rho) [H][W]
 * (summed over the bins) and dL/d(ego) [nb][6], FP64, by the chain rule
 * through the projection, the rigid transform and Rodrigues' formula:
 *   with P = R X + t, X = (xn, yn, 1)/rho and G = scale * dL/dflow,
 *   dL/dP = (G_x fx / P2, G_y fy / P2, -(G_x fx P0 + G_y fy P1) / P2^2)
 *   dL/dt = sum dL/dP, dL/dR = sum dL/dP X^T, dL/dX = R^T dL/dP,
 *   dL/drho = -(dL/dX . (xn, yn, 1)) / rho^2,
 *   dL/dv = -dt dL/dt, dL/dw_c = -dt sum_ab dL/dR_ab dR_ab/dk_c (k = -w dt).
 */
void orc_flow_eq2_grad(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho,
                       const double* ego, int32_t nb, double dt_bin, double scale, const double* dflow,
                       double* drho, double* dego)
{
    const int64_t HW = (int64_t)W * H;
    for (int64_t q = 0; q < HW; ++q) drho[q] = 0.0;
    for (int32_t i = 0; i < nb; ++i) {
        const double* e = ego + 6 * i;
        const double k[3] = {-e[3] * dt_bin, -e[4] * dt_bin, -e[5] * dt_bin};
        const double t[3] = {-e[0] * dt_bin, -e[1] * dt_bin, -e[2] * dt_bin};
        double Rm[3][3];
        rodrigues(k, Rm);
        double gt[3] = {0, 0, 0}, M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int32_t v = 0; v < H; ++v) {
            for (int32_t u = 0; u < W; ++u) {
                const int64_t q = (int64_t)v * W + u;
                const double xn = ((double)u - cx) / fx, yn = ((double)v - cy) / fy;
                const double Z = 1.0 / rho[q];
                const double X[3] = {Z * xn, Z * yn, Z};
                double P[3];
                for (int r = 0; r < 3; ++r) P[r] = Rm[r][0] * X[0] + Rm[r][1] * X[1] + Rm[r][2] * X[2] + t[r];
                const double Gx = scale * dflow[2 * (HW * i + q) + 0], Gy = scale * dflow[2 * (HW * i + q) + 1];
                const double dP[3] = {Gx * fx / P[2], Gy * fy / P[2],
                                      -(Gx * fx * P[0] + Gy * fy * P[1]) / (P[2] * P[2])};
                for (int r = 0; r < 3; ++r) {
                    gt[r] += dP[r];
                    for (int c = 0; c < 3; ++c) M[r][c] += dP[r] * X[c];
                }
                double dX[3];
                for (int c = 0; c < 3; ++c) dX[c] = Rm[0][c] * dP[0] + Rm[1][c] * dP[1] + Rm[2][c] * dP[2];
                const double dZ = dX[0] * xn + dX[1] * yn + dX[2];
                drho[q] += -Z * Z * dZ;
            }
        }
        double dR[3][3][3];
        rodrigues_grad(k, dR);
        for (int c = 0; c < 3; ++c) {
            double dk = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int s2 = 0; s2 < 3; ++s2) dk += M[r][s2] * dR[c][r][s2];
            dego[6 * i + c] = -dt_bin * gt[c];
            dego[6 * i + 3 + c] = -dt_bin * dk;
        }
    }
}

/*
 * Geometry-consistency loss (Sec. 3.2, Eq. 3), read as in the consistency loss
 * the paper cites: every pixel x of view 0 with depth D0 = 1/rho0 is moved by
 * the camera motion between the two views (the rigid transform of Eq. 2:
 * P = R X + t, R = Rodrigues(-w dt), t = -v dt); its forward-projected depth
 * is a = P2, its projection x' lands in view 1, where the interpolated depth b
 * is the bilinear sample of D1 = 1/rho1 at x' (corner indices clamped).  Valid
 * pixels V: P2 > 0 and x' inside the closed image box.
 *   L_geo = (1 / |V|) sum_{x in V} |a - b| / (a + b)
 * The projection decides integers (valid or not, the sample's cell, the sign
 * of a - b), so the decisions are taken in the kernels' FP32 sequence
 * (orc_geo_proj_f32) and the loss in FP64 on those decisions; the gradient is
 * that of the branch the decisions select (sign 0 when a = b in FP32).
 */
/* The decisions in FP32: the projection, the valid flag, and the sign of
 * a - b (the branch of |a - b|), with
 *   ax = x' - floor(x'), bx = 1 - ax (likewise y), w00 = bx*by, w10 = ax*by,
 *   w01 = bx*ay, w11 = ax*ay, D_c = 1/rho1_c,
 *   b = fma(w11, D11, fma(w01, D01, fma(w10, D10, w00*D00))),  a = P2. */
void orc_geo_proj_f32(int32_t W, int32_t H, float fx, float fy, float cx, float cy, const float* rho0,
                      const float* rho1, const float* ego, float dt, float* proj, uint8_t* ok, int8_t* sgn)
{
    float Rm[9], tv[3], Ad[3];
    rot_f32(ego, dt, Rm, tv, Ad);
    const float ifx = 1.0f / fx, ify = 1.0f / fy;
    const float W1 = (float)(W - 1), H1 = (float)(H - 1);
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t q = (int64_t)v * W + u;
            const float xn = ((float)u - cx) * ifx;
            const float yn = ((float)v - cy) * ify;
            const float Z = 1.0f / rho0[q];
            float dx, dy, P2;
            disp_f32(Rm, tv, Ad, xn, yn, Z, fx, fy, &dx, &dy, &P2);
            const float xp = (float)u + dx;
            const float yp = (float)v + dy;
            proj[2 * q] = xp;
            proj[2 * q + 1] = yp;
            ok[q] = P2 > 0.0f && xp >= 0.0f && xp <= W1 && yp >= 0.0f && yp <= H1;
            sgn[q] = 0;
            if (!ok[q]) continue;
            const float fx0 = floorf(xp), fy0 = floorf(yp);
            const int ix = (int)fx0, iy = (int)fy0;
            const int ix1 = ix + 1 < W ? ix + 1 : W - 1, iy1 = iy + 1 < H ? iy + 1 : H - 1;
            const float ax = xp - fx0, ay = yp - fy0, bx = 1.0f - ax, by = 1.0f - ay;
            const float w00 = bx * by, w10 = ax * by, w01 = bx * ay, w11 = ax * ay;
            const float D00 = 1.0f / rho1[(int64_t)iy * W + ix], D10 = 1.0f / rho1[(int64_t)iy * W + ix1];
            const float D01 = 1.0f / rho1[(int64_t)iy1 * W + ix], D11 = 1.0f / rho1[(int64_t)iy1 * W + ix1];
            const float b = fmaf(w11, D11, fmaf(w01, D01, fmaf(w10, D10, w00 * D00)));
            sgn[q] = P2 > b ? 1 : (P2 < b ? -1 : 0);
        }
    }
}

double orc_geo(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho0,
               const double* rho1, const double* ego, double dt, const float* proj, const uint8_t* ok,
               const int8_t* sgn, double dloss, int64_t* count, double* drho0, double* drho1, double* dego)
{
    const int64_t HW = (int64_t)W * H;
    const double k[3] = {-ego[3] * dt, -ego[4] * dt, -ego[5] * dt};
    const double t[3] = {-ego[0] * dt, -ego[1] * dt, -ego[2] * dt};
    double Rm[3][3];
    rodrigues(k, Rm);
    int64_t nv = 0;
    for (int64_t q = 0; q < HW; ++q) nv += ok[q] != 0;
    *count = nv;
    if (drho0)
        for (int64_t q = 0; q < HW; ++q) drho0[q] = drho1[q] = 0.0;
    double gt[3] = {0, 0, 0}, M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double sum = 0.0;
    const double g = nv > 0 ? dloss / (double)nv : 0.0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t q = (int64_t)v * W + u;
            if (!ok[q]) continue;
            const double xn = ((double)u - cx) / fx, yn = ((double)v - cy) / fy;
            const double Z = 1.0 / rho0[q];
            const double X[3] = {Z * xn, Z * yn, Z};
            double P[3];
            for (int r = 0; r < 3; ++r) P[r] = Rm[r][0] * X[0] + Rm[r][1] * X[1] + Rm[r][2] * X[2] + t[r];
            const double xp = fx * P[0] / P[2] + cx, yp = fy * P[1] / P[2] + cy;
            /* the decided cell; the weights from the FP64 position */
            const int ix = (int)floorf(proj[2 * q]), iy = (int)floorf(proj[2 * q + 1]);
            const int ix1 = ix + 1 < W ? ix + 1 : W - 1, iy1 = iy + 1 < H ? iy + 1 : H - 1;
            const double ax = xp - ix, ay = yp - iy;
            const int64_t c00 = (int64_t)iy * W + ix, c10 = (int64_t)iy * W + ix1;
            const int64_t c01 = (int64_t)iy1 * W + ix, c11 = (int64_t)iy1 * W + ix1;
            const double D00 = 1.0 / rho1[c00], D10 = 1.0 / rho1[c10], D01 = 1.0 / rho1[c01], D11 = 1.0 / rho1[c11];
            const double w00 = (1 - ax) * (1 - ay), w10 = ax * (1 - ay), w01 = (1 - ax) * ay, w11 = ax * ay;
            const double a = P[2];
            const double b = w00 * D00 + w10 * D10 + w01 * D01 + w11 * D11;
            const double sg = (double)sgn[q]; /* the branch of |a - b| decided in FP32 */
            sum += (sg != 0.0 ? sg * (a - b) : fabs(a - b)) / (a + b);
            if (!drho0) continue;
            const double dfa = g * sg * 2.0 * b / ((a + b) * (a + b));
            const double dfb = -g * sg * 2.0 * a / ((a + b) * (a + b));
            const double dbx = (1 - ay) * (D10 - D00) + ay * (D11 - D01);
            const double dby = (1 - ax) * (D01 - D00) + ax * (D11 - D10);
            /* x' = fx P0/P2 + cx, y' = fy P1/P2 + cy */
            const double dP[3] = {dfb * dbx * fx / P[2], dfb * dby * fy / P[2],
                                  dfa - dfb * (dbx * fx * P[0] + dby * fy * P[1]) / (P[2] * P[2])};
            for (int r = 0; r < 3; ++r) {
                gt[r] += dP[r];
                for (int c = 0; c < 3; ++c) M[r][c] += dP[r] * X[c];
            }
            double dX[3];
            for (int c = 0; c < 3; ++c) dX[c] = Rm[0][c] * dP[0] + Rm[1][c] * dP[1] + Rm[2][c] * dP[2];
            drho0[q] += -Z * Z * (dX[0] * xn + dX[1] * yn + dX[2]);
            /* b = sum_c w_c / rho1_c */
            drho1[c00] -= dfb * w00 * D00 * D00;
            drho1[c10] -= dfb * w10 * D10 * D10;
            drho1[c01] -= dfb * w01 * D01 * D01;
            drho1[c11] -= dfb * w11 * D11 * D11;
        }
    }
    if (drho0) {
        double dR[3][3][3];
        rodrigues_grad(k, dR);
        for (int c = 0; c < 3; ++c) {
            double dk = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int s2 = 0; s2 < 3; ++s2) dk += M[r][s2] * dR[c][r][s2];
            dego[c] = -dt * gt[c];
            dego[3 + c] = -dt * dk;
        }
    }
    return nv > 0 ? sum / (double)nv : 0.0;
}

/*
 * The network's input frame (Sec. 4.1, supp. Table 4: a (2, H, W) input): the
 * events of a window accumulated per pixel and polarity, channel 0 positive,
 * channel 1 negative; events outside the sensor are skipped.  frame is
 * [2][H][W], overwritten.
 */
void orc_event_frame(int32_t W, int32_t H, int64_t n, const int16_t* x, const int16_t* y, const int8_t* p,
                     double* frame)
{
    const int64_t HW = (int64_t)W * H;
    for (int64_t q = 0; q < 2 * HW; ++q) frame[q] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        if (x[k] < 0 || x[k] >= W || y[k] < 0 || y[k] >= H) continue;
        frame[(p[k] > 0 ? 0 : HW) + (int64_t)y[k] * W + x[k]] += 1.0;
    }
}

/* ------------------------------------------------------------------------- */
/* S2-S6: warp, mask, splat, loss, gradient                                  */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t W, H;            /* sensor size */
    int32_t nbins;           /* B >= 1 */
    int32_t ref_mode;        /* ORC_REF_END or ORC_REF_ALL */
    int32_t n_flow_bins;     /* 1 (one field for every bin) or B (one per bin) */
    int32_t pos_f32;         /* 1: positions in FP32 (kernel precision); 0: FP64 */
    int32_t branch_mode;     /* 0: decide; 1: decide and record; 2: replay record */
    int32_t pad_;
    int64_t n;               /* number of events */
    const int16_t* x;        /* [n] pixel column */
    const int16_t* y;        /* [n] pixel row */
    const float* t;          /* [n] timestamp */
    const int8_t* p;         /* [n] polarity, > 0 positive, else negative */
    double t0, t1;           /* window (FP32 values carried exactly) */
    double eps;              /* regulariser of both ratios */
    double dloss;            /* upstream gradient dOut/dL for the backward */
    const double* flow;      /* [nfb][H][W][2], FP64 values */
    const float* flow32;     /* [nfb][H][W][2], FP32 flow for pos_f32 = 1 */
    /* branch record, [n] and [n][B+1]: used when branch_mode != 0 */
    int32_t* br_cell;        /* [n][B+1][2] floor of each computed position */
    uint8_t* br_supp;        /* [n][B+1] bit c: corner c carries a nonzero weight */
    uint8_t* br_valid;       /* [n] */
    int32_t* br_bin;         /* [n] */
    /* outputs; NULL = not wanted */
    double* loss;            /* [1] */
    double* loss_r;          /* [R] */
    int64_t* nnz_r;          /* [R] */
    double* iwe;             /* [R][H][W][4] = (C+, S+, C-, S-) */
    double* dflow;           /* [nfb][H][W][2] */
    uint8_t* valid;          /* [n] */
    double* pos;             /* [n][B+1][2] trajectory (computed edges; others NaN) */
} orc_cm_args;

/* corner order c = 0..3: (ix, iy), (ix+1, iy), (ix, iy+1), (ix+1, iy+1) */

typedef struct {
    int B, R, jlo, jhi;      /* computed edges jlo..jhi */
    int ref_edge[ORC_MAX_BINS + 1];
    double tau_edge[ORC_MAX_BINS + 1];
} orc_setup;

static const double* field64(const orc_cm_args* a, int j)
{
    return a->flow + (a->n_flow_bins == 1 ? 0 : (int64_t)j * a->W * a->H * 2);
}

static const float* field32(const orc_cm_args* a, int j)
{
    return a->flow32 + (a->n_flow_bins == 1 ? 0 : (int64_t)j * a->W * a->H * 2);
}

/* bilinear sample of one field at (px, py) in cell (ix, iy), FP64; also the
 * 2x2 Jacobian d(u)/d(px, py) and the four weights with their (clamped)
 * pixel indices */
static void sample64(const double* U, int W, int H, double px, double py, int ix, int iy,
                     double u[2], double J[2][2], double w[4], int64_t idx[4])
{
    const double ax = px - (double)ix, ay = py - (double)iy;
    const double bx = 1.0 - ax, by = 1.0 - ay;
    const int ix1 = ix + 1 < W ? ix + 1 : W - 1;
    const int iy1 = iy + 1 < H ? iy + 1 : H - 1;
    idx[0] = (int64_t)iy * W + ix;
    idx[1] = (int64_t)iy * W + ix1;
    idx[2] = (int64_t)iy1 * W + ix;
    idx[3] = (int64_t)iy1 * W + ix1;
    w[0] = bx * by;
    w[1] = ax * by;
    w[2] = bx * ay;
    w[3] = ax * ay;
    for (int d = 0; d < 2; ++d) {
        const double u00 = U[2 * idx[0] + d], u10 = U[2 * idx[1] + d];
        const double u01 = U[2 * idx[2] + d], u11 = U[2 * idx[3] + d];
        u[d] = w[0] * u00 + w[1] * u10 + w[2] * u01 + w[3] * u11;
        J[d][0] = by * (u10 - u00) + ay * (u11 - u01);
        J[d][1] = bx * (u01 - u00) + ax * (u11 - u10);
    }
}

/* FP32 bilinear sample with the fixed operation order of the kernels:
 *   ax = px - floor(px), bx = 1 - ax (same in y)
 *   w00 = bx*by, w10 = ax*by, w01 = bx*ay, w11 = ax*ay
 *   u = w00*u00;  u = fma(w10, u10, u);  u = fma(w01, u01, u);  u = fma(w11, u11, u) */
static void sample32(const float* U, int W, int H, float px, float py, float u[2])
{
    const float fx0 = floorf(px), fy0 = floorf(py);
    const float ax = px - fx0, ay = py - fy0;
    const float bx = 1.0f - ax, by = 1.0f - ay;
    const float w00 = bx * by, w10 = ax * by, w01 = bx * ay, w11 = ax * ay;
    const int ix = (int)fx0, iy = (int)fy0;
    const int ix1 = ix + 1 < W ? ix + 1 : W - 1;
    const int iy1 = iy + 1 < H ? iy + 1 : H - 1;
    const float* p00 = U + 2 * ((int64_t)iy * W + ix);
    const float* p10 = U + 2 * ((int64_t)iy * W + ix1);
    const float* p01 = U + 2 * ((int64_t)iy1 * W + ix);
    const float* p11 = U + 2 * ((int64_t)iy1 * W + ix1);
    for (int d = 0; d < 2; ++d) {
        float s = w00 * p00[d];
        s = fmaf(w10, p10[d], s);
        s = fmaf(w01, p01[d], s);
        s = fmaf(w11, p11[d], s);
        u[d] = s;
    }
}

static int inside64(double px, double py, int W, int H)
{
    return px >= 0.0 && px <= (double)(W - 1) && py >= 0.0 && py <= (double)(H - 1);
}

static int inside32(float px, float py, int W, int H)
{
    return px >= 0.0f && px <= (float)(W - 1) && py >= 0.0f && py <= (float)(H - 1);
}

/* support bits of the four corners at position (px, py) in cell (ix, iy): a
 * corner is in the support when it lies in the image and its bilinear weight
 * is nonzero (the fractional part of the position in that direction is not 0) */
static uint8_t support_bits(double px, double py, int ix, int iy, int W, int H)
{
    const int nzx = px != (double)ix, nzy = py != (double)iy;
    const int in1 = ix + 1 <= W - 1, in2 = iy + 1 <= H - 1;
    uint8_t s = 1;
    if (nzx && in1) s |= 2;
    if (nzy && in2) s |= 4;
    if (nzx && nzy && in1 && in2) s |= 8;
    return s;
}

/* Bin index of normalised time tau: b = min(floor(tau * B), B - 1), clamped
 * below at 0.  In the FP32 mode tau = (t - t0) / (t1 - t0) and tau * B are
 * single-precision operations, as in the kernels. */
static int bin_of(const orc_cm_args* a, int B, int64_t k, double* tau64, float* tau32)
{
    const double tau = ((double)a->t[k] - a->t0) / (a->t1 - a->t0);
    const float t0f = (float)a->t0, t1f = (float)a->t1;
    const float tf = (a->t[k] - t0f) / (t1f - t0f);
    *tau64 = tau;
    *tau32 = tf;
    double q = a->pos_f32 ? (double)floorf(tf * (float)B) : floor(tau * (double)B);
    int b = (int)(q < 0 ? 0 : q);
    if (b > B - 1) b = B - 1;
    return b;
}

/*
 * S2 + S3 for one event: the trajectory at the computed edges jlo..jhi, the
 * cell of each point, the support bits and the validity (every computed point
 * inside the image).  Forward (Sec. 3.1, iterative warp):
 *   x_{b+1} = x_k + (tau_{b+1} - tau_k) u_b(x_k),  x_{j+1} = x_j + (1/B) u_j(x_j)
 * backward:
 *   x_b = x_k - (tau_k - tau_b) u_b(x_k),          x_{j-1} = x_j - (1/B) u_{j-1}(x_j)
 * where u_j(x) is the bilinear sample of the flow of bin j at x.
 * Returns 1 when the event is valid.  pos, cell, supp are indexed by edge j.
 */
static int trajectory(const orc_cm_args* a, const orc_setup* s, int64_t k, int* bin_out,
                      double* tau_out, double pos[][2], int cell[][2], uint8_t supp[])
{
    const int W = a->W, H = a->H, B = s->B;
    const int xk = a->x[k], yk = a->y[k];
    double tau;
    float tau32;
    int b = bin_of(a, B, k, &tau, &tau32);
    *tau_out = tau;
    if (a->branch_mode == 2) b = a->br_bin[k];
    *bin_out = b;
    if (xk < 0 || xk > W - 1 || yk < 0 || yk > H - 1) return 0;
    const int replay = a->branch_mode == 2;
    int ok = 1;
    if (a->pos_f32 && !replay) {
        /* FP32 trajectory with the kernels' operation order:
         *   tau_j = j / B, h = 1 / B (single-precision divisions)
         *   forward:  x = fma(tau_{b+1} - tau, u_b(x_k), x_k), then x = fma(h, u_j(x), x)
         *   backward: x = fma(-(tau - tau_b), u_b(x_k), x_k), then x = fma(-h, u_{j-1}(x), x) */
        const float Bf = (float)B, h = 1.0f / Bf;
        float p32[ORC_MAX_BINS + 1][2];
        float u0[2];
        sample32(field32(a, b), W, H, (float)xk, (float)yk, u0);
        if (s->jhi > b) {
            const float dt = (float)(b + 1) / Bf - tau32;
            p32[b + 1][0] = fmaf(dt, u0[0], (float)xk);
            p32[b + 1][1] = fmaf(dt, u0[1], (float)yk);
            for (int j = b + 1; j < s->jhi; ++j) {
                if (!inside32(p32[j][0], p32[j][1], W, H)) { ok = 0; break; }
                float u[2];
                sample32(field32(a, j), W, H, p32[j][0], p32[j][1], u);
                p32[j + 1][0] = fmaf(h, u[0], p32[j][0]);
                p32[j + 1][1] = fmaf(h, u[1], p32[j][1]);
            }
            if (ok && !inside32(p32[s->jhi][0], p32[s->jhi][1], W, H)) ok = 0;
        }
        if (ok && s->jlo <= b) {
            const float dt = tau32 - (float)b / Bf;
            p32[b][0] = fmaf(-dt, u0[0], (float)xk);
            p32[b][1] = fmaf(-dt, u0[1], (float)yk);
            for (int j = b; j > s->jlo; --j) {
                if (!inside32(p32[j][0], p32[j][1], W, H)) { ok = 0; break; }
                float u[2];
                sample32(field32(a, j - 1), W, H, p32[j][0], p32[j][1], u);
                p32[j - 1][0] = fmaf(-h, u[0], p32[j][0]);
                p32[j - 1][1] = fmaf(-h, u[1], p32[j][1]);
            }
            if (ok && !inside32(p32[s->jlo][0], p32[s->jlo][1], W, H)) ok = 0;
        }
        if (!ok) return 0;
        for (int j = s->jlo; j <= s->jhi; ++j) {
            pos[j][0] = (double)p32[j][0];
            pos[j][1] = (double)p32[j][1];
            cell[j][0] = (int)floor(pos[j][0]);
            cell[j][1] = (int)floor(pos[j][1]);
            supp[j] = support_bits(pos[j][0], pos[j][1], cell[j][0], cell[j][1], W, H);
        }
        return 1;
    }

    /* FP64 trajectory (the plain definition), or a replay of a recorded branch:
     * cells, support and validity taken from the record, positions in FP64 */
    const double h = 1.0 / (double)B;
    if (replay && !a->br_valid[k]) return 0;
    const int64_t rb = k * (int64_t)(B + 1);
    double u0[2], J[2][2], w[4];
    int64_t idx[4];
    sample64(field64(a, b), W, H, (double)xk, (double)yk, xk, yk, u0, J, w, idx);
#define ORC_SET_CELL(j)                                                                         \
    do {                                                                                        \
        if (replay) {                                                                           \
            cell[j][0] = a->br_cell[2 * (rb + (j)) + 0];                                        \
            cell[j][1] = a->br_cell[2 * (rb + (j)) + 1];                                        \
            supp[j] = a->br_supp[rb + (j)];                                                     \
        } else {                                                                                \
            if (!inside64(pos[j][0], pos[j][1], W, H)) return 0;                                \
            cell[j][0] = (int)floor(pos[j][0]);                                                 \
            cell[j][1] = (int)floor(pos[j][1]);                                                 \
            supp[j] = support_bits(pos[j][0], pos[j][1], cell[j][0], cell[j][1], W, H);         \
        }                                                                                       \
    } while (0)
    if (s->jhi > b) {
        const double dt = s->tau_edge[b + 1] - tau;
        pos[b + 1][0] = (double)xk + dt * u0[0];
        pos[b + 1][1] = (double)yk + dt * u0[1];
        ORC_SET_CELL(b + 1);
        for (int j = b + 1; j < s->jhi; ++j) {
            double u[2];
            sample64(field64(a, j), W, H, pos[j][0], pos[j][1], cell[j][0], cell[j][1], u, J, w, idx);
            pos[j + 1][0] = pos[j][0] + h * u[0];
            pos[j + 1][1] = pos[j][1] + h * u[1];
            ORC_SET_CELL(j + 1);
        }
    }
    if (s->jlo <= b) {
        const double dt = tau - s->tau_edge[b];
        pos[b][0] = (double)xk - dt * u0[0];
        pos[b][1] = (double)yk - dt * u0[1];
        ORC_SET_CELL(b);
        for (int j = b; j > s->jlo; --j) {
            double u[2];
            sample64(field64(a, j - 1), W, H, pos[j][0], pos[j][1], cell[j][0], cell[j][1], u, J, w, idx);
            pos[j - 1][0] = pos[j][0] - h * u[0];
            pos[j - 1][1] = pos[j][1] - h * u[1];
            ORC_SET_CELL(j - 1);
        }
    }
#undef ORC_SET_CELL
    return 1;
}

static int setup(const orc_cm_args* a, orc_setup* s)
{
    if (a->W < 2 || a->H < 2 || a->nbins < 1 || a->nbins > ORC_MAX_BINS) return ORC_EINVAL;
    if (!(a->t1 > a->t0) || a->n < 0 || !(a->eps > 0)) return ORC_EINVAL;
    if (a->n_flow_bins != 1 && a->n_flow_bins != a->nbins) return ORC_EINVAL;
    if (a->ref_mode != ORC_REF_END && a->ref_mode != ORC_REF_ALL) return ORC_EINVAL;
    if (a->pos_f32 && !a->flow32) return ORC_EINVAL;
    if (a->branch_mode == 2 && (a->pos_f32 || !a->br_cell || !a->br_supp || !a->br_valid || !a->br_bin))
        return ORC_EINVAL;
    if (a->branch_mode == 1 && (!a->br_cell || !a->br_supp || !a->br_valid || !a->br_bin)) return ORC_EINVAL;
    const int B = a->nbins;
    s->B = B;
    for (int j = 0; j <= B; ++j) s->tau_edge[j] = (double)j / (double)B;
    if (a->ref_mode == ORC_REF_END) {
        s->R = 1;
        s->ref_edge[0] = B;
        s->jlo = -1; /* set per event: the forward chain only */
        s->jhi = B;
    } else {
        s->R = B + 1;
        for (int r = 0; r <= B; ++r) s->ref_edge[r] = r;
        s->jlo = 0;
        s->jhi = B;
    }
    return ORC_OK;
}

/* computed edges of event k: with one reference at the window end only the
 * forward chain b+1..B is pushed; with all edges both chains, 0..B */
static void event_range(const orc_cm_args* a, const orc_setup* s0, int64_t k, orc_setup* s)
{
    *s = *s0;
    if (a->ref_mode == ORC_REF_END) {
        double t64;
        float t32;
        const int b = a->branch_mode == 2 ? a->br_bin[k] : bin_of(a, s0->B, k, &t64, &t32);
        s->jlo = b + 1;
    }
}

int orc_cm(orc_cm_args* a)
{
    orc_setup s0;
    int st = setup(a, &s0);
    if (st) return st;
    const int W = a->W, H = a->H, B = s0.B, R = s0.R;
    const int64_t HW = (int64_t)W * H;

    double* iwe = (double*)calloc((size_t)(R * HW * 4), sizeof(double));
    uint8_t* hit = (uint8_t*)calloc((size_t)(R * HW), 1);
    if (!iwe || !hit) { free(iwe); free(hit); return ORC_ENOMEM; }

    double pos[ORC_MAX_BINS + 1][2];
    int cell[ORC_MAX_BINS + 1][2];
    uint8_t supp[ORC_MAX_BINS + 1];

    /* ---- forward: S2 trajectory, S3 mask, S4 splat ---- */
    for (int64_t k = 0; k < a->n; ++k) {
        orc_setup s;
        int b;
        double tau;
        event_range(a, &s0, k, &s);
        const int ok = trajectory(a, &s, k, &b, &tau, pos, cell, supp);
        if (a->valid) a->valid[k] = (uint8_t)ok;
        if (a->branch_mode == 1) {
            a->br_valid[k] = (uint8_t)ok;
            a->br_bin[k] = b;
            for (int j = 0; j <= B; ++j) {
                const int64_t q = k * (int64_t)(B + 1) + j;
                const int have = ok && j >= s.jlo && j <= s.jhi;
                a->br_cell[2 * q + 0] = have ? cell[j][0] : 0;
                a->br_cell[2 * q + 1] = have ? cell[j][1] : 0;
                a->br_supp[q] = have ? supp[j] : 0;
            }
        }
        if (a->pos) {
            for (int j = 0; j <= B; ++j) {
                const int have = ok && j >= s.jlo && j <= s.jhi;
                a->pos[2 * (k * (B + 1) + j) + 0] = have ? pos[j][0] : NAN;
                a->pos[2 * (k * (B + 1) + j) + 1] = have ? pos[j][1] : NAN;
            }
        }
        if (!ok) continue;
        const int pol = a->p[k] > 0 ? 0 : 1;
        for (int r = 0; r < R; ++r) {
            const int j = s.ref_edge[r];
            const double tbar = 1.0 - fabs(s.tau_edge[j] - tau);
            const int ix = cell[j][0], iy = cell[j][1];
            const double ax = pos[j][0] - ix, ay = pos[j][1] - iy;
            const double wc[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};
            const int dx[4] = {0, 1, 0, 1}, dy[4] = {0, 0, 1, 1};
            for (int c = 0; c < 4; ++c) {
                if (!(supp[j] >> c & 1)) continue;
                const int64_t pix = (int64_t)(iy + dy[c]) * W + (ix + dx[c]);
                double* q = iwe + 4 * (r * HW + pix) + 2 * pol;
                q[0] += wc[c];
                q[1] += wc[c] * tbar;
                hit[r * HW + pix] = 1;
            }
        }
    }

    /* ---- S5: loss (Eq. 1 with the scaling and masking regularisers) ---- */
    double L = 0.0;
    double* nnz = (double*)malloc(sizeof(double) * (size_t)R);
    if (!nnz) { free(iwe); free(hit); return ORC_ENOMEM; }
    for (int r = 0; r < R; ++r) {
        int64_t cnt = 0;
        double sum = 0.0;
        for (int64_t i = 0; i < HW; ++i) {
            const double* q = iwe + 4 * (r * HW + i);
            const double Tp = q[1] / (q[0] + a->eps);
            const double Tm = q[3] / (q[2] + a->eps);
            sum += Tp * Tp + Tm * Tm;
            cnt += hit[r * HW + i];
        }
        const double Lr = sum / ((double)cnt + a->eps);
        nnz[r] = (double)cnt;
        if (a->loss_r) a->loss_r[r] = Lr;
        if (a->nnz_r) a->nnz_r[r] = cnt;
        L += Lr;
    }
    L /= (double)R;
    if (a->loss) a->loss[0] = L;
    if (a->iwe) memcpy(a->iwe, iwe, sizeof(double) * (size_t)(R * HW * 4));

    /* ---- S6: exact gradient with respect to the flow (reverse mode) ----
     * dL/dS_p(x) = kappa 2T/(C+eps),  dL/dC_p(x) = -kappa 2T^2/(C+eps),
     * kappa = dloss / (R (N_nz + eps)).  For an event with average timestamp
     * tbar splatting weight w_c to pixel c, dL/dw_c = phi_c = kappa 2T(tbar - T)/(C+eps),
     * and the position adjoint at that reference is a = sum_c grad(w_c) phi_c over
     * the in-image corners (right-derivative at integer coordinates).  The
     * adjoint lambda is carried back along each chain of pushes:
     *   forward chain  x_{j+1} = x_j + h u_j(x_j):
     *     dL/du_j[c] += h w_c(x_j) lambda_{j+1};  lambda_j = a_j + (I + h J_j)^T lambda_{j+1}
     *   first push     x_{b+1} = x_k + d u_b(x_k):  dL/du_b[x_k] += d lambda_{b+1}
     *   backward chain x_{j-1} = x_j - h u_{j-1}(x_j):
     *     dL/du_{j-1}[c] -= h w_c(x_j) lambda_{j-1};  lambda_j = a_j + (I - h J_{j-1})^T lambda_{j-1}
     *   first push     x_b = x_k - d u_b(x_k):      dL/du_b[x_k] -= d lambda_b */
    if (a->dflow) {
        const int nfb = a->n_flow_bins;
        memset(a->dflow, 0, sizeof(double) * (size_t)(nfb * HW * 2));
        double aj[ORC_MAX_BINS + 1][2];
        int isref[ORC_MAX_BINS + 1];
        for (int64_t k = 0; k < a->n; ++k) {
            orc_setup s;
            int b;
            double tau;
            event_range(a, &s0, k, &s);
            if (!trajectory(a, &s, k, &b, &tau, pos, cell, supp)) continue;
            const int pol = a->p[k] > 0 ? 0 : 1;
            for (int j = 0; j <= B; ++j) { aj[j][0] = aj[j][1] = 0.0; isref[j] = 0; }
            for (int r = 0; r < R; ++r) {
                const int j = s.ref_edge[r];
                isref[j] = 1;
                const double tbar = 1.0 - fabs(s.tau_edge[j] - tau);
                const double kappa = a->dloss / ((double)R * (nnz[r] + a->eps));
                const int ix = cell[j][0], iy = cell[j][1];
                const double ax = pos[j][0] - ix, ay = pos[j][1] - iy;
                const int dx[4] = {0, 1, 0, 1}, dy[4] = {0, 0, 1, 1};
                /* d(w_c)/dx, d(w_c)/dy for c = 00, 10, 01, 11 */
                const double gwx[4] = {-(1 - ay), (1 - ay), -ay, ay};
                const double gwy[4] = {-(1 - ax), -ax, (1 - ax), ax};
                for (int c = 0; c < 4; ++c) {
                    const int cx = ix + dx[c], cy = iy + dy[c];
                    if (cx > W - 1 || cy > H - 1) continue;
                    const double* q = iwe + 4 * (r * HW + (int64_t)cy * W + cx) + 2 * pol;
                    const double C = q[0], S = q[1];
                    const double T = S / (C + a->eps);
                    const double phi = kappa * 2.0 * T * (tbar - T) / (C + a->eps);
                    aj[j][0] += gwx[c] * phi;
                    aj[j][1] += gwy[c] * phi;
                }
            }
            const double h = 1.0 / (double)B;
            const int xk = a->x[k], yk = a->y[k];
            double u[2], J[2][2], w[4];
            int64_t idx[4];
            /* forward chain */
            if (s.jhi > b) {
                double lam[2] = {0.0, 0.0};
                for (int j = s.jhi; j >= b + 1; --j) {
                    if (isref[j]) { lam[0] += aj[j][0]; lam[1] += aj[j][1]; }
                    if (j > b + 1) {
                        const int js = j - 1; /* push from edge js to js + 1 with field js */
                        double* G = a->dflow + (nfb == 1 ? 0 : (int64_t)js * HW * 2);
                        sample64(field64(a, js), W, H, pos[js][0], pos[js][1], cell[js][0], cell[js][1], u, J, w, idx);
                        for (int c = 0; c < 4; ++c) {
                            G[2 * idx[c] + 0] += h * w[c] * lam[0];
                            G[2 * idx[c] + 1] += h * w[c] * lam[1];
                        }
                        const double l0 = lam[0] + h * (J[0][0] * lam[0] + J[1][0] * lam[1]);
                        const double l1 = lam[1] + h * (J[0][1] * lam[0] + J[1][1] * lam[1]);
                        lam[0] = l0;
                        lam[1] = l1;
                    } else {
                        const double d = s.tau_edge[b + 1] - tau;
                        double* G = a->dflow + (nfb == 1 ? 0 : (int64_t)b * HW * 2);
                        const int64_t i0 = (int64_t)yk * W + xk;
                        G[2 * i0 + 0] += d * lam[0];
                        G[2 * i0 + 1] += d * lam[1];
                    }
                }
            }
            /* backward chain */
            if (s.jlo <= b) {
                double lam[2] = {0.0, 0.0};
                for (int j = s.jlo; j <= b; ++j) {
                    if (isref[j]) { lam[0] += aj[j][0]; lam[1] += aj[j][1]; }
                    if (j < b) {
                        const int js = j + 1; /* push from edge js to js - 1 with field js - 1 = j */
                        double* G = a->dflow + (nfb == 1 ? 0 : (int64_t)j * HW * 2);
                        sample64(field64(a, j), W, H, pos[js][0], pos[js][1], cell[js][0], cell[js][1], u, J, w, idx);
                        for (int c = 0; c < 4; ++c) {
                            G[2 * idx[c] + 0] -= h * w[c] * lam[0];
                            G[2 * idx[c] + 1] -= h * w[c] * lam[1];
                        }
                        const double l0 = lam[0] - h * (J[0][0] * lam[0] + J[1][0] * lam[1]);
                        const double l1 = lam[1] - h * (J[0][1] * lam[0] + J[1][1] * lam[1]);
                        lam[0] = l0;
                        lam[1] = l1;
                    } else {
                        const double d = tau - s.tau_edge[b];
                        double* G = a->dflow + (nfb == 1 ? 0 : (int64_t)b * HW * 2);
                        const int64_t i0 = (int64_t)yk * W + xk;
                        G[2 * i0 + 0] -= d * lam[0];
                        G[2 * i0 + 1] -= d * lam[1];
                    }
                }
            }
        }
    }
    free(nnz);
    free(iwe);
    free(hit);
    return ORC_OK;
}

int orc_abi_version(void) { return 1; }
