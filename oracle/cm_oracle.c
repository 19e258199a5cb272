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
 *   - every operation is FP64: positions, weights, sums, the loss and the
 *     gradient.  The oracle shares no arithmetic with the FP32 GPU path.
 *
 * Straddles (how an FP32 result is judged against this FP64 definition).  The
 * floor of a trajectory position decides the flow cell, the pixels a splat
 * touches and whether a corner carries weight (so which pixels are non-empty
 * and N_nz); the image border decides the mask; floor(tau B) decides the bin.
 * The loss jumps where such a decision changes (a pixel reached by a tiny
 * weight counts fully in N_nz and in the sum of T^2), and the gradient jumps
 * too (kinks of the bilinear weights).  orc_cm_bounds bounds, coordinate by
 * coordinate, how far an FP32 evaluation of the trajectory can be from the
 * FP64 one (a forward error bound from the magnitudes of the quantities
 * involved), flags every decision within that distance of its threshold, and
 * returns the interval of N_nz and of the loss over every outcome of the
 * flagged decisions.  An FP32 result passes when its N_nz lies in the interval
 * and its loss within the stated tolerance of it; gradients are compared on the
 * events no decision of which is flagged.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no fast-math).
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

/* ------------------------------------------------------------------------- */
/* Error bounds of an FP32 evaluation (used to flag straddles)               */
/* ------------------------------------------------------------------------- */

#define ORC_U 5.9604644775390625e-08 /* 2^-24: unit roundoff of IEEE single precision */

/*
 * Bound on |flow32 - flow| per pixel for the motion field of S1 evaluated in
 * FP32 (any evaluation order): each of the products and sums that make up
 * d(xn)/dt and d(yn)/dt is rounded once, and xn, yn carry the rounding of
 * (u - cx) / fx, so the error is at most c u M, where M is the sum of the
 * magnitudes of the terms, u = 2^-24 and c = 20 (the rounded operations on the
 * longest path, with a margin); the product with dt f adds 2u of the result.
 * eb[H][W] is the bound of the larger of the two components.
 */
void orc_flow_error_bound(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho,
                          const double* ego, double dt, double* eb)
{
    const double vx = fabs(ego[0]), vy = fabs(ego[1]), vz = fabs(ego[2]);
    const double wx = fabs(ego[3]), wy = fabs(ego[4]), wz = fabs(ego[5]);
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const double xn = fabs(((double)u - cx) / fx), yn = fabs(((double)v - cy) / fy);
            const double r = fabs(rho[(int64_t)v * W + u]);
            const double Mx = r * (vx + xn * vz) + xn * yn * wx + (1.0 + xn * xn) * wy + yn * wz;
            const double My = r * (vy + yn * vz) + (1.0 + yn * yn) * wx + xn * yn * wy + xn * wz;
            const double bx = 22.0 * ORC_U * dt * fx * Mx, by = 22.0 * ORC_U * dt * fy * My;
            eb[(int64_t)v * W + u] = bx > by ? bx : by;
        }
    }
}

/* |R - I| bounded entrywise by |a K| + |b K^2| (R = I + a K + b K^2 of
 * Rodrigues' formula; a ~ 1, b ~ 1/2) */
static void rot_abs(const double k[3], double Aabs[3][3])
{
    const double th = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    double a, b;
    if (th < 1e-12) { a = 1.0; b = 0.5; }
    else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
    const double K[3][3] = {{0, -k[2], k[1]}, {k[2], 0, -k[0]}, {-k[1], k[0], 0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double K2 = 0;
            for (int l = 0; l < 3; ++l) K2 += K[i][l] * K[l][j];
            Aabs[i][j] = fabs(a * K[i][j]) + fabs(b * K2);
        }
}

/*
 * Bound on the FP32 error of the Eq. 2 displacement of one pixel,
 * d = f (P0/P2 - xn) (and likewise y), for an evaluation in the form
 * P0/P2 - xn = (Z s0 + t0 - xn t2) / P2, s0 = ((R - I) m)_0 - xn ((R - I) m)_2,
 * m = (xn, yn, 1), that never subtracts two large terms: the numerator and P2
 * are sums of terms of magnitudes Me and Mp2, each rounded a bounded number of
 * times (c u M with c = 16, covering also the rounding of xn, yn, Z = 1/rho and
 * of the rotation's entries), and the quotient adds the error of P2 and two
 * roundings.  e0, e1: the exact numerators; P2: the exact depth.
 */
static void eq2_bound(const double Aabs[3][3], const double t[3], double xn, double yn, double Z, double P2,
                      double e0, double e1, double fx, double fy, double* ebx, double* eby, double* ebp2)
{
    const double m[3] = {fabs(xn), fabs(yn), 1.0};
    double Am[3];
    for (int i = 0; i < 3; ++i) Am[i] = Aabs[i][0] * m[0] + Aabs[i][1] * m[1] + Aabs[i][2] * m[2];
    const double Za = fabs(Z);
    const double Me0 = Za * (Am[0] + m[0] * Am[2]) + fabs(t[0]) + m[0] * fabs(t[2]);
    const double Me1 = Za * (Am[1] + m[1] * Am[2]) + fabs(t[1]) + m[1] * fabs(t[2]);
    const double Mp2 = Za * (1.0 + Am[2]) + fabs(t[2]);
    const double c = 16.0 * ORC_U;
    const double eP2 = c * Mp2, aP2 = fabs(P2);
    *ebx = fx * (c * Me0 / aP2 + fabs(e0) * eP2 / (aP2 * aP2) + 3.0 * ORC_U * fabs(e0) / aP2);
    *eby = fy * (c * Me1 / aP2 + fabs(e1) * eP2 / (aP2 * aP2) + 3.0 * ORC_U * fabs(e1) / aP2);
    *ebp2 = eP2;
}

/*
 * Bound on |flow32 - flow| per bin and pixel for orc_flow_eq2_bins evaluated
 * in FP32 (eq2_bound; the product with `scale` adds 2u of the result).
 * eb[nb][H][W]: the larger of the two components.
 */
void orc_flow_eq2_error_bound(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho,
                              const double* ego, int32_t nb, double dt_bin, double scale, double* eb)
{
    const int64_t HW = (int64_t)W * H;
    for (int32_t i = 0; i < nb; ++i) {
        const double* e = ego + 6 * i;
        const double k[3] = {-e[3] * dt_bin, -e[4] * dt_bin, -e[5] * dt_bin};
        const double t[3] = {-e[0] * dt_bin, -e[1] * dt_bin, -e[2] * dt_bin};
        double Rm[3][3], Aabs[3][3];
        rodrigues(k, Rm);
        rot_abs(k, Aabs);
        for (int32_t v = 0; v < H; ++v) {
            for (int32_t u = 0; u < W; ++u) {
                const int64_t q = (int64_t)v * W + u;
                const double xn = ((double)u - cx) / fx, yn = ((double)v - cy) / fy;
                const double Z = 1.0 / rho[q];
                double P[3];
                for (int a = 0; a < 3; ++a) P[a] = Z * (Rm[a][0] * xn + Rm[a][1] * yn + Rm[a][2]) + t[a];
                const double e0 = P[0] - xn * P[2], e1 = P[1] - yn * P[2];
                double bx, by, bp;
                eq2_bound(Aabs, t, xn, yn, Z, P[2], e0, e1, fx, fy, &bx, &by, &bp);
                bx = fabs(scale) * bx + 2.0 * ORC_U * fabs(scale * fx * e0 / P[2]);
                by = fabs(scale) * by + 2.0 * ORC_U * fabs(scale * fy * e1 / P[2]);
                eb[HW * i + q] = bx > by ? bx : by;
            }
        }
    }
}

/*
 * Geometry-consistency loss (Sec. 3.2, Eq. 3), read as in the consistency loss
 * the paper cites: every pixel x of view 0 with depth D0 = 1/rho0 is moved by
 * the camera motion between the two views (the rigid transform of Eq. 2:
 * P = R X + t, R = Rodrigues(-w dt), t = -v dt); its forward-projected depth
 * is a = P2, its projection x' = (fx P0/P2 + cx, fy P1/P2 + cy) lands in view
 * 1, where the interpolated depth b is the bilinear sample of D1 = 1/rho1 at
 * x' (corner indices clamped).  Valid pixels V: P2 > 0 and x' inside the
 * closed image box.
 *   L_geo = (1 / |V|) sum_{x in V} |a - b| / (a + b)
 * FP64 throughout.  The gradient is that of the branch the decisions select
 * (valid set, sample cell, sign of a - b; sign 0 where a = b).
 * dec: NULL, or per pixel the decisions (cell [HW][2], valid [HW], sign [HW])
 * to record (mode 1) or to replay with FP64 positions (mode 2, frozen-branch
 * differences).
 */
typedef struct {
    int32_t mode;   /* 0: decide; 1: decide and record; 2: replay */
    int32_t pad_;
    int32_t* cell;  /* [HW][2] */
    uint8_t* ok;    /* [HW] */
    int8_t* sgn;    /* [HW] */
} orc_geo_dec;

/* the projection of pixel (u, v) of view 0: x', y', the depth a = P2, and the
 * quantities the error bound needs */
typedef struct {
    double xn, yn, Z, X[3], P[3], xp, yp;
} geo_proj;

static void geo_project(double Rm[3][3], const double t[3], double fx, double fy, double cx, double cy, int u, int v,
                        double rho0, geo_proj* g)
{
    g->xn = ((double)u - cx) / fx;
    g->yn = ((double)v - cy) / fy;
    g->Z = 1.0 / rho0;
    g->X[0] = g->Z * g->xn;
    g->X[1] = g->Z * g->yn;
    g->X[2] = g->Z;
    for (int r = 0; r < 3; ++r) g->P[r] = Rm[r][0] * g->X[0] + Rm[r][1] * g->X[1] + Rm[r][2] * g->X[2] + t[r];
    /* x' = fx P0/P2 + cx written as the pixel plus its displacement
     * fx (P0 - xn P2) / P2 (the same value; exactly the pixel at rest) */
    g->xp = (double)u + fx * (g->P[0] - g->xn * g->P[2]) / g->P[2];
    g->yp = (double)v + fy * (g->P[1] - g->yn * g->P[2]) / g->P[2];
}

static int geo_inside(double xp, double yp, int W, int H)
{
    return xp >= 0.0 && xp <= (double)(W - 1) && yp >= 0.0 && yp <= (double)(H - 1);
}

/* b = bilinear sample of 1/rho1 at (xp, yp) in cell (ix, iy), its gradient
 * with respect to (xp, yp), the four weights and corner indices */
static double geo_sample(const double* rho1, int W, int H, double xp, double yp, int ix, int iy, double* dbx,
                         double* dby, double w[4], int64_t c[4], double D[4])
{
    const int ix1 = ix + 1 < W ? ix + 1 : W - 1, iy1 = iy + 1 < H ? iy + 1 : H - 1;
    const double ax = xp - ix, ay = yp - iy;
    c[0] = (int64_t)iy * W + ix;
    c[1] = (int64_t)iy * W + ix1;
    c[2] = (int64_t)iy1 * W + ix;
    c[3] = (int64_t)iy1 * W + ix1;
    for (int q = 0; q < 4; ++q) D[q] = 1.0 / rho1[c[q]];
    w[0] = (1 - ax) * (1 - ay);
    w[1] = ax * (1 - ay);
    w[2] = (1 - ax) * ay;
    w[3] = ax * ay;
    *dbx = (1 - ay) * (D[1] - D[0]) + ay * (D[3] - D[2]);
    *dby = (1 - ax) * (D[2] - D[0]) + ax * (D[3] - D[1]);
    return w[0] * D[0] + w[1] * D[1] + w[2] * D[2] + w[3] * D[3];
}

double orc_geo(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho0,
               const double* rho1, const double* ego, double dt, const orc_geo_dec* dec, double dloss,
               int64_t* count, double* drho0, double* drho1, double* dego)
{
    const int64_t HW = (int64_t)W * H;
    const double k[3] = {-ego[3] * dt, -ego[4] * dt, -ego[5] * dt};
    const double t[3] = {-ego[0] * dt, -ego[1] * dt, -ego[2] * dt};
    const int mode = dec ? dec->mode : 0;
    double Rm[3][3];
    rodrigues(k, Rm);
    /* the decisions of every pixel */
    uint8_t* ok = (uint8_t*)malloc((size_t)HW);
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)HW);
    int8_t* sgn = (int8_t*)malloc((size_t)HW);
    if (!ok || !cell || !sgn) { free(ok); free(cell); free(sgn); return NAN; }
    int64_t nv = 0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t q = (int64_t)v * W + u;
            if (mode == 2) {
                ok[q] = dec->ok[q];
                cell[2 * q] = dec->cell[2 * q];
                cell[2 * q + 1] = dec->cell[2 * q + 1];
                sgn[q] = dec->sgn[q];
            } else {
                geo_proj g;
                geo_project(Rm, t, fx, fy, cx, cy, u, v, rho0[q], &g);
                ok[q] = g.P[2] > 0.0 && geo_inside(g.xp, g.yp, W, H);
                cell[2 * q] = ok[q] ? (int32_t)floor(g.xp) : 0;
                cell[2 * q + 1] = ok[q] ? (int32_t)floor(g.yp) : 0;
                sgn[q] = 0;
                if (ok[q]) {
                    double dbx, dby, w[4], D[4];
                    int64_t c[4];
                    const double b = geo_sample(rho1, W, H, g.xp, g.yp, cell[2 * q], cell[2 * q + 1], &dbx, &dby, w,
                                                c, D);
                    sgn[q] = g.P[2] > b ? 1 : (g.P[2] < b ? -1 : 0);
                }
                if (mode == 1) {
                    dec->ok[q] = ok[q];
                    dec->cell[2 * q] = cell[2 * q];
                    dec->cell[2 * q + 1] = cell[2 * q + 1];
                    dec->sgn[q] = sgn[q];
                }
            }
            nv += ok[q] != 0;
        }
    }
    *count = nv;
    if (drho0)
        for (int64_t q = 0; q < HW; ++q) drho0[q] = drho1[q] = 0.0;
    double gt[3] = {0, 0, 0}, M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double sum = 0.0;
    const double gs = nv > 0 ? dloss / (double)nv : 0.0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t q = (int64_t)v * W + u;
            if (!ok[q]) continue;
            geo_proj g;
            geo_project(Rm, t, fx, fy, cx, cy, u, v, rho0[q], &g);
            double dbx, dby, w[4], D[4];
            int64_t c[4];
            const double a = g.P[2];
            const double b = geo_sample(rho1, W, H, g.xp, g.yp, cell[2 * q], cell[2 * q + 1], &dbx, &dby, w, c, D);
            /* |a - b| on the recorded branch when replaying, else its value */
            const double sg = (double)sgn[q];
            sum += (mode == 2 ? sg * (a - b) : fabs(a - b)) / (a + b);
            if (!drho0) continue;
            const double dfa = gs * sg * 2.0 * b / ((a + b) * (a + b));
            const double dfb = -gs * sg * 2.0 * a / ((a + b) * (a + b));
            /* x' = fx P0/P2 + cx, y' = fy P1/P2 + cy */
            const double P2 = g.P[2];
            const double dP[3] = {dfb * dbx * fx / P2, dfb * dby * fy / P2,
                                  dfa - dfb * (dbx * fx * g.P[0] + dby * fy * g.P[1]) / (P2 * P2)};
            for (int r = 0; r < 3; ++r) {
                gt[r] += dP[r];
                for (int cc = 0; cc < 3; ++cc) M[r][cc] += dP[r] * g.X[cc];
            }
            double dX[3];
            for (int cc = 0; cc < 3; ++cc) dX[cc] = Rm[0][cc] * dP[0] + Rm[1][cc] * dP[1] + Rm[2][cc] * dP[2];
            drho0[q] += -g.Z * g.Z * (dX[0] * g.xn + dX[1] * g.yn + dX[2]);
            /* b = sum_c w_c / rho1_c */
            for (int cc = 0; cc < 4; ++cc) drho1[c[cc]] -= dfb * w[cc] * D[cc] * D[cc];
        }
    }
    if (drho0) {
        double dR[3][3][3];
        rodrigues_grad(k, dR);
        for (int cc = 0; cc < 3; ++cc) {
            double dk = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int s2 = 0; s2 < 3; ++s2) dk += M[r][s2] * dR[cc][r][s2];
            dego[cc] = -dt * gt[cc];
            dego[3 + cc] = -dt * dk;
        }
    }
    free(ok);
    free(cell);
    free(sgn);
    return nv > 0 ? sum / (double)nv : 0.0;
}

/*
 * Straddles of the geometry-consistency loss for an FP32 evaluation that keeps
 * the projection as the pixel plus the FP32 displacement (eq2_bound): per
 * pixel, with margins safety x the error bound of x', y', a and b,
 *   bit 0: x' or y' within its margin of an integer (the sample cell; a kink
 *          of the gradient, the loss is continuous there),
 *   bit 1: x' or y' within its margin of the border, or P2 within its margin
 *          of 0 (the valid set: the loss jumps),
 *   bit 2: |a - b| within the margin of a - b (the branch of |a - b|: a kink).
 * count_lo/hi: the valid count over every outcome of the bit-1 decisions;
 * loss_lo/hi: the loss over those outcomes (a pixel's term |a-b|/(a+b) lies in
 * [0, 1] for positive depths).  Returns the number of flagged pixels.
 */
int64_t orc_geo_bounds(int32_t W, int32_t H, double fx, double fy, double cx, double cy, const double* rho0,
                       const double* rho1, const double* ego, double dt, double safety, uint8_t* flags,
                       int64_t* count_lo, int64_t* count_hi, double* loss_lo, double* loss_hi)
{
    const double k[3] = {-ego[3] * dt, -ego[4] * dt, -ego[5] * dt};
    const double t[3] = {-ego[0] * dt, -ego[1] * dt, -ego[2] * dt};
    double Rm[3][3], Aabs[3][3];
    rodrigues(k, Rm);
    rot_abs(k, Aabs);
    int64_t nsure = 0, nmaybe = 0, nflag = 0;
    double ssure = 0.0;
    for (int32_t v = 0; v < H; ++v) {
        for (int32_t u = 0; u < W; ++u) {
            const int64_t q = (int64_t)v * W + u;
            geo_proj g;
            geo_project(Rm, t, fx, fy, cx, cy, u, v, rho0[q], &g);
            const double e0 = g.P[0] - g.xn * g.P[2], e1 = g.P[1] - g.yn * g.P[2];
            double ebx, eby, ebp;
            eq2_bound(Aabs, t, g.xn, g.yn, g.Z, g.P[2], e0, e1, fx, fy, &ebx, &eby, &ebp);
            /* the displacement is added to the integer pixel: no further rounding of x'
             * (an exact displacement, error bound 0, decides exactly: margin 0) */
            const double mx = ebx > 0.0 ? safety * (ebx + ORC_U) : 0.0;
            const double my = eby > 0.0 ? safety * (eby + ORC_U) : 0.0, mp = safety * ebp;
            uint8_t f = 0;
            const double W1 = (double)(W - 1), H1 = (double)(H - 1);
            if (fabs(g.P[2]) <= mp || (mx > 0.0 && (fabs(g.xp) <= mx || fabs(g.xp - W1) <= mx)) ||
                (my > 0.0 && (fabs(g.yp) <= my || fabs(g.yp - H1) <= my)))
                f |= 2;
            const int valid = g.P[2] > 0.0 && geo_inside(g.xp, g.yp, W, H);
            if (valid) {
                if ((mx > 0.0 && fabs(g.xp - floor(g.xp + 0.5)) <= mx) ||
                    (my > 0.0 && fabs(g.yp - floor(g.yp + 0.5)) <= my))
                    f |= 1;
                double dbx, dby, w[4], D[4];
                int64_t c[4];
                const double b = geo_sample(rho1, W, H, g.xp, g.yp, (int)floor(g.xp), (int)floor(g.yp), &dbx, &dby,
                                            w, c, D);
                /* b: weights from x' (its error times the slope) and 1/rho1 (two roundings each) */
                const double Dmax = fmax(fmax(fabs(D[0]), fabs(D[1])), fmax(fabs(D[2]), fabs(D[3])));
                const double eb = fabs(dbx) * (ebx + ORC_U) + fabs(dby) * (eby + ORC_U) + 8.0 * ORC_U * Dmax;
                if (fabs(g.P[2] - b) <= safety * (ebp + eb)) f |= 4;
                if (f & 2) nmaybe += 1;
                else {
                    nsure += 1;
                    ssure += fabs(g.P[2] - b) / (g.P[2] + b);
                }
            } else if (f & 2) {
                nmaybe += 1;
            }
            if (flags) flags[q] = f;
            nflag += f != 0;
        }
    }
    *count_lo = nsure;
    *count_hi = nsure + nmaybe;
    *loss_lo = nsure + nmaybe > 0 ? ssure / (double)(nsure + nmaybe) : 0.0;
    *loss_hi = nsure > 0 ? (ssure + (double)nmaybe) / (double)nsure : (nmaybe > 0 ? 1.0 : 0.0);
    return nflag;
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
    int32_t branch_mode;     /* 0: decide; 1: decide and record; 2: replay record */
    int64_t n;               /* number of events */
    const int16_t* x;        /* [n] pixel column */
    const int16_t* y;        /* [n] pixel row */
    const float* t;          /* [n] timestamp */
    const int8_t* p;         /* [n] polarity, > 0 positive, else negative */
    double t0, t1;           /* window (FP32 values carried exactly) */
    double eps;              /* regulariser of both ratios */
    double dloss;            /* upstream gradient dOut/dL for the backward */
    const double* flow;      /* [nfb][H][W][2], FP64 values */
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

static int inside64(double px, double py, int W, int H)
{
    return px >= 0.0 && px <= (double)(W - 1) && py >= 0.0 && py <= (double)(H - 1);
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

/* Bin index of normalised time tau = (t - t0) / (t1 - t0):
 * b = min(floor(tau * B), B - 1), clamped below at 0. */
static int bin_of(const orc_cm_args* a, int B, int64_t k, double* tau64)
{
    const double tau = ((double)a->t[k] - a->t0) / (a->t1 - a->t0);
    *tau64 = tau;
    const double q = floor(tau * (double)B);
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
    int b = bin_of(a, B, k, &tau);
    *tau_out = tau;
    if (a->branch_mode == 2) b = a->br_bin[k];
    *bin_out = b;
    if (xk < 0 || xk > W - 1 || yk < 0 || yk > H - 1) return 0;
    const int replay = a->branch_mode == 2;

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
    if (a->branch_mode == 2 && (!a->br_cell || !a->br_supp || !a->br_valid || !a->br_bin))
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
        const int b = a->branch_mode == 2 ? a->br_bin[k] : bin_of(a, s0->B, k, &t64);
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

/* ------------------------------------------------------------------------- */
/* Straddles of an FP32 evaluation: flags and the interval of the loss       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double safety;          /* margin of a decision = safety x (error bound + u); 0 error -> 0 margin */
    int32_t pad_;
    int32_t pad2_;
    const double* eflow;    /* [nfb][H][W] bound on |flow32 - flow| per pixel, or NULL: the flow values
                             * are FP32 numbers given to both evaluations exactly */
    /* outputs; NULL = not wanted */
    uint8_t* flags;         /* [n]: bit 0 a point within its margin of an integer coordinate (cell and
                             * support decisions), bit 1 within its margin of the image border (the mask),
                             * bit 2 tau B within its margin of an interior bin edge (the bin) */
    double* err;            /* [n][B+1][2] error bound of each computed point (NaN elsewhere) */
    double* loss_lo;        /* [1] */
    double* loss_hi;        /* [1] */
    double* loss_r_lo;      /* [R] */
    double* loss_r_hi;      /* [R] */
    int64_t* nnz_lo;        /* [R] */
    int64_t* nnz_hi;        /* [R] */
    int64_t counts[4];      /* events with bit 0, bit 1, bit 2, any bit */
} orc_bounds;

/* largest change of each flow component between neighbouring pixels along x
 * (L[d][0]) and along y (L[d][1]) over rows iy-1..iy+2 and columns ix-1..ix+2
 * (clamped): a Lipschitz constant of the bilinear interpolant within one pixel
 * of cell (ix, iy) */
static void lipschitz(const double* U, int W, int H, int ix, int iy, double L[2][2])
{
    L[0][0] = L[0][1] = L[1][0] = L[1][1] = 0.0;
    for (int yy = iy - 1; yy <= iy + 2; ++yy) {
        const int y0 = yy < 0 ? 0 : (yy > H - 1 ? H - 1 : yy);
        for (int xx = ix - 1; xx <= ix + 2; ++xx) {
            const int x0 = xx < 0 ? 0 : (xx > W - 1 ? W - 1 : xx);
            const int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
            const double* p = U + 2 * ((int64_t)y0 * W + x0);
            const double* px = U + 2 * ((int64_t)y0 * W + x1);
            const double* py = U + 2 * ((int64_t)y1 * W + x0);
            for (int d = 0; d < 2; ++d) {
                const double gx = fabs(px[d] - p[d]), gy = fabs(py[d] - p[d]);
                if (gx > L[d][0]) L[d][0] = gx;
                if (gy > L[d][1]) L[d][1] = gy;
            }
        }
    }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* flags of one point from its position and error bound; returns 0 when the
 * point lies outside the image beyond its margin (outside in any evaluation) */
static int point_flags(const double p[2], const double e[2], double safety, int W, int H, double m[2],
                       uint8_t* flag)
{
    const double ext[2] = {(double)(W - 1), (double)(H - 1)};
    for (int d = 0; d < 2; ++d) {
        m[d] = e[d] > 0.0 ? safety * (e[d] + ORC_U) : 0.0;
        if (p[d] < -m[d] || p[d] > ext[d] + m[d]) return 0;
        if (m[d] > 0.0) {
            if (fabs(p[d]) <= m[d] || fabs(p[d] - ext[d]) <= m[d]) *flag |= 2;
            if (fabs(p[d] - floor(p[d] + 0.5)) <= m[d]) *flag |= 1;
        }
    }
    return 1;
}

/*
 * The FP64 trajectory of event k with a bound on the error of an FP32
 * evaluation of every point, and the event's flags.  The bound assumes the
 * evaluation keeps each point as the event's pixel plus an FP32 offset (so a
 * rounding costs u times the offset, not u times the coordinate) and follows
 * each push x' = x + hs u(x):
 *   e' = e + |hs| (L e + 8 u max|u_c| + max eflow_c) + u |hs u| + u |x' - x_k|
 * (L: Lipschitz constants of the sampled field near x, u_c / eflow_c: the
 * corner values and their bounds); the first push of a chain adds the error
 * of tau and of tau_j to its time step.  A point outside the image by less
 * than its margin is carried on (the flow sampled at the nearest image point)
 * and makes the event's validity uncertain (flag bit 1).
 * Returns 0 for an event that is outside the image (or the sensor) in any
 * evaluation, 1 for a valid one, 2 for one whose validity is uncertain.
 */
static int traj_bound(const orc_cm_args* a, const orc_setup* s, const double* eflow, double safety, int64_t k,
                      int* bin_out, double* tau_out, double pos[][2], double err[][2], double mar[][2],
                      uint8_t* flag)
{
    const int W = a->W, H = a->H, B = s->B;
    const int64_t HW = (int64_t)W * H;
    const int xk = a->x[k], yk = a->y[k];
    double tau;
    const int b = bin_of(a, B, k, &tau);
    *tau_out = tau;
    *bin_out = b;
    *flag = 0;
    if (xk < 0 || xk > W - 1 || yk < 0 || yk > H - 1) return 0;
    const double etau = 4.0 * ORC_U * fabs(tau);
    {
        const double q = tau * (double)B, qr = floor(q + 0.5);
        const double mq = safety * ((double)B * etau + 2.0 * ORC_U * fabs(q));
        if (qr >= 1.0 && qr <= (double)(B - 1) && fabs(q - qr) <= mq && mq > 0.0) *flag |= 4;
    }
    const double h = 1.0 / (double)B;
    int status = 1;
    const double* U0 = field64(a, b);
    const double* E0 = eflow ? eflow + (a->n_flow_bins == 1 ? 0 : (int64_t)b * HW) : NULL;
    const int64_t i0 = (int64_t)yk * W + xk;
    const double u0[2] = {U0[2 * i0], U0[2 * i0 + 1]};
    const double e0 = E0 ? E0[i0] : 0.0;
    for (int dir = 0; dir < 2; ++dir) {
        /* dir 0: forward chain b+1 .. jhi; dir 1: backward chain b .. jlo */
        if (dir == 0 && !(s->jhi > b)) continue;
        if (dir == 1 && !(s->jlo <= b)) continue;
        const int jfirst = dir == 0 ? b + 1 : b;
        const double dt = dir == 0 ? s->tau_edge[b + 1] - tau : -(tau - s->tau_edge[b]);
        const double edt = etau + ORC_U * s->tau_edge[dir == 0 ? b + 1 : b] + ORC_U * fabs(dt);
        for (int d = 0; d < 2; ++d) {
            const double disp = dt * u0[d];
            pos[jfirst][d] = (double)(d == 0 ? xk : yk) + disp;
            err[jfirst][d] = (u0[d] != 0.0 || e0 > 0.0) ? fabs(u0[d]) * edt + fabs(dt) * e0 + ORC_U * fabs(disp)
                                                         : 0.0;
        }
        if (!point_flags(pos[jfirst], err[jfirst], safety, W, H, mar[jfirst], flag)) return 0;
        if (!inside64(pos[jfirst][0], pos[jfirst][1], W, H)) status = 2;
        const int jend = dir == 0 ? s->jhi : s->jlo;
        const int step = dir == 0 ? 1 : -1;
        const double hs = dir == 0 ? h : -h;
        for (int j = jfirst; j != jend; j += step) {
            const int field = dir == 0 ? j : j - 1;
            const int jn = j + step;
            /* sample at the point, moved into the image when it lies just outside */
            const double px = clampd(pos[j][0], 0.0, (double)(W - 1)), py = clampd(pos[j][1], 0.0, (double)(H - 1));
            const int ix = (int)floor(px), iy = (int)floor(py);
            double u[2], J[2][2], w[4];
            int64_t idx[4];
            const double* U = field64(a, field);
            sample64(U, W, H, px, py, ix, iy, u, J, w, idx);
            double L[2][2];
            lipschitz(U, W, H, ix, iy, L);
            double umax[2] = {0, 0}, emax = 0.0;
            const double* E = eflow ? eflow + (a->n_flow_bins == 1 ? 0 : (int64_t)field * HW) : NULL;
            for (int c = 0; c < 4; ++c) {
                for (int d = 0; d < 2; ++d)
                    if (fabs(U[2 * idx[c] + d]) > umax[d]) umax[d] = fabs(U[2 * idx[c] + d]);
                if (E && E[idx[c]] > emax) emax = E[idx[c]];
            }
            for (int d = 0; d < 2; ++d) {
                const double inc = hs * u[d];
                pos[jn][d] = pos[j][d] + inc;
                const double off = pos[jn][d] - (double)(d == 0 ? xk : yk);
                const int exact = err[j][0] == 0.0 && err[j][1] == 0.0 && emax == 0.0 && umax[d] == 0.0;
                err[jn][d] = exact ? err[j][d]
                                   : err[j][d] + fabs(hs) * (L[d][0] * err[j][0] + L[d][1] * err[j][1] +
                                                             8.0 * ORC_U * umax[d] + emax) +
                                         ORC_U * fabs(inc) + ORC_U * fabs(off);
            }
            if (!point_flags(pos[jn], err[jn], safety, W, H, mar[jn], flag)) return 0;
            if (!inside64(pos[jn][0], pos[jn][1], W, H)) status = 2;
        }
    }
    if (*flag & 2) status = 2;
    return status;
}

/* one maybe contribution: weight in [0, wmax] of average timestamp tbar to
 * polarity pol of pixel pix at reference r */
typedef struct {
    int64_t key;   /* (r * HW + pix) * 2 + pol */
    double wmax, tbar;
} orc_maybe;

static int cmp_maybe(const void* x, const void* y)
{
    const int64_t a = ((const orc_maybe*)x)->key, b = ((const orc_maybe*)y)->key;
    return a < b ? -1 : (a > b);
}

/* range of T = (S + sum w_i t_i) / (C + sum w_i + eps) over w_i in [0, wmax_i]:
 * a linear-fractional function of the w_i, extreme at a vertex of the box */
static void t_range(double C, double S, const orc_maybe* m, int k, double eps, double* lo, double* hi)
{
    if (k > 12) {
        double sw = 0, swt = 0;
        for (int i = 0; i < k; ++i) {
            sw += m[i].wmax;
            swt += m[i].wmax * m[i].tbar;
        }
        *lo = S / (C + sw + eps);
        *hi = (S + swt) / (C + eps);
        return;
    }
    double tl = INFINITY, th = -INFINITY;
    for (int v = 0; v < (1 << k); ++v) {
        double c = C, sm = S;
        for (int i = 0; i < k; ++i)
            if (v >> i & 1) {
                c += m[i].wmax;
                sm += m[i].wmax * m[i].tbar;
            }
        const double T = sm / (c + eps);
        if (T < tl) tl = T;
        if (T > th) th = T;
    }
    *lo = tl;
    *hi = th;
}

/*
 * Flags and the loss interval (see the header).  Per reference and pixel the
 * splat is split into sure contributions (both axis factors of the corner away
 * from a flagged decision, event surely valid) and maybe contributions (weight
 * anywhere in [0, its bound]): a corner whose factor is within the margin of 0
 * on the near side of an integer, the mirror corner on the far side (where an
 * FP32 floor on the other side of the integer would put the small weight), and
 * every corner of an event of uncertain validity.  N_nz(r) lies between the
 * pixels with a sure contribution and those plus the pixels with only maybe
 * ones; the sum of T^2 between the sums of each pixel's extremes; L_r and L
 * between the ratios of those bounds.
 */
int orc_cm_bounds(const orc_cm_args* a, orc_bounds* o)
{
    orc_setup s0;
    int st = setup(a, &s0);
    if (st) return st;
    if (a->branch_mode != 0 || !(o->safety >= 0)) return ORC_EINVAL;
    const int W = a->W, H = a->H, B = s0.B, R = s0.R;
    const int64_t HW = (int64_t)W * H;
    double* iwe = (double*)calloc((size_t)(R * HW * 4), sizeof(double));
    uint8_t* hit = (uint8_t*)calloc((size_t)(R * HW), 1);
    size_t mcap = 1024, mn = 0;
    orc_maybe* mb = (orc_maybe*)malloc(sizeof(orc_maybe) * mcap);
    if (!iwe || !hit || !mb) { free(iwe); free(hit); free(mb); return ORC_ENOMEM; }
    double pos[ORC_MAX_BINS + 1][2], err[ORC_MAX_BINS + 1][2], mar[ORC_MAX_BINS + 1][2];
    for (int q = 0; q < 4; ++q) o->counts[q] = 0;
    for (int64_t k = 0; k < a->n; ++k) {
        orc_setup s;
        int b;
        double tau;
        uint8_t flag = 0;
        event_range(a, &s0, k, &s);
        for (int j = 0; j <= B; ++j) err[j][0] = err[j][1] = NAN;
        const int status = traj_bound(a, &s, o->eflow, o->safety, k, &b, &tau, pos, err, mar, &flag);
        if (o->flags) o->flags[k] = flag;
        if (o->err)
            for (int j = 0; j <= B; ++j) {
                const int have = status && j >= s.jlo && j <= s.jhi;
                o->err[2 * (k * (B + 1) + j) + 0] = have ? err[j][0] : NAN;
                o->err[2 * (k * (B + 1) + j) + 1] = have ? err[j][1] : NAN;
            }
        for (int q = 0; q < 3; ++q) o->counts[q] += (flag >> q) & 1;
        o->counts[3] += flag != 0;
        if (!status) continue;
        const int pol = a->p[k] > 0 ? 0 : 1;
        for (int r = 0; r < R; ++r) {
            const int j = s.ref_edge[r];
            const double tbar = 1.0 - fabs(s.tau_edge[j] - tau);
            /* per axis: up to three columns / rows, each with a factor, a bound
             * on it and whether it is sure */
            int cix[2][3], ncand[2];
            double fac[2][3], fmax[2][3];
            int sure[2][3];
            for (int d = 0; d < 2; ++d) {
                const double x = pos[j][d], m = mar[j][d];
                const int x0 = (int)floor(x);
                const double f = x - x0;
                int n = 0;
                if (m > 0.0 && f <= m) {
                    cix[d][n] = x0; fac[d][n] = 1 - f; fmax[d][n] = 1 - f + m; sure[d][n++] = 1;
                    cix[d][n] = x0 + 1; fac[d][n] = f; fmax[d][n] = f + m; sure[d][n++] = 0;
                    cix[d][n] = x0 - 1; fac[d][n] = 0; fmax[d][n] = m - f; sure[d][n++] = 0;
                } else if (m > 0.0 && 1 - f <= m) {
                    cix[d][n] = x0 + 1; fac[d][n] = f; fmax[d][n] = f + m; sure[d][n++] = 1;
                    cix[d][n] = x0; fac[d][n] = 1 - f; fmax[d][n] = 1 - f + m; sure[d][n++] = 0;
                    cix[d][n] = x0 + 2; fac[d][n] = 0; fmax[d][n] = m - (1 - f); sure[d][n++] = 0;
                } else {
                    cix[d][n] = x0; fac[d][n] = 1 - f; fmax[d][n] = 1 - f + m; sure[d][n++] = 1;
                    cix[d][n] = x0 + 1; fac[d][n] = f; fmax[d][n] = f + m; sure[d][n++] = 1;
                }
                ncand[d] = n;
            }
            for (int cy = 0; cy < ncand[1]; ++cy) {
                for (int cx = 0; cx < ncand[0]; ++cx) {
                    const int X = cix[0][cx], Y = cix[1][cy];
                    if (X < 0 || X > W - 1 || Y < 0 || Y > H - 1) continue;
                    const int64_t pix = (int64_t)Y * W + X;
                    const int is_sure = status == 1 && sure[0][cx] && sure[1][cy];
                    if (is_sure) {
                        const double wgt = fac[0][cx] * fac[1][cy];
                        if (wgt <= 0.0) continue;
                        double* q = iwe + 4 * (r * HW + pix) + 2 * pol;
                        q[0] += wgt;
                        q[1] += wgt * tbar;
                        hit[r * HW + pix] = 1;
                    } else {
                        const double wmax = (sure[0][cx] && status == 1 ? fac[0][cx] : fmax[0][cx]) *
                                            (sure[1][cy] && status == 1 ? fac[1][cy] : fmax[1][cy]);
                        if (!(wmax > 0.0)) continue;
                        if (mn == mcap) {
                            mcap *= 2;
                            orc_maybe* nb = (orc_maybe*)realloc(mb, sizeof(orc_maybe) * mcap);
                            if (!nb) { free(iwe); free(hit); free(mb); return ORC_ENOMEM; }
                            mb = nb;
                        }
                        mb[mn].key = (r * HW + pix) * 2 + pol;
                        mb[mn].wmax = wmax;
                        mb[mn].tbar = tbar;
                        mn += 1;
                    }
                }
            }
        }
    }
    qsort(mb, mn, sizeof(orc_maybe), cmp_maybe);
    /* per reference: sums over the pixels without maybe contributions, then
     * the pixels with some */
    double Llo = 0.0, Lhi = 0.0;
    size_t mi = 0;
    for (int r = 0; r < R; ++r) {
        double slo = 0.0, shi = 0.0;
        int64_t nlo = 0, nmaybe = 0;
        for (int64_t i = 0; i < HW; ++i) {
            const double* q = iwe + 4 * (r * HW + i);
            const int64_t kp = (r * HW + i) * 2;
            double tlo[2], thi[2];
            int any_maybe = 0;
            for (int p = 0; p < 2; ++p) {
                size_t m0 = mi;
                while (mi < mn && mb[mi].key == kp + p) ++mi;
                const int km = (int)(mi - m0);
                any_maybe |= km > 0;
                if (km == 0) {
                    tlo[p] = thi[p] = q[2 * p + 1] / (q[2 * p] + a->eps);
                } else {
                    t_range(q[2 * p], q[2 * p + 1], mb + m0, km, a->eps, &tlo[p], &thi[p]);
                }
            }
            slo += tlo[0] * tlo[0] + tlo[1] * tlo[1];
            shi += thi[0] * thi[0] + thi[1] * thi[1];
            if (hit[r * HW + i]) nlo += 1;
            else if (any_maybe) nmaybe += 1;
        }
        const double lo = slo / ((double)(nlo + nmaybe) + a->eps);
        const double hi = shi / ((double)nlo + a->eps);
        if (o->loss_r_lo) o->loss_r_lo[r] = lo;
        if (o->loss_r_hi) o->loss_r_hi[r] = hi;
        if (o->nnz_lo) o->nnz_lo[r] = nlo;
        if (o->nnz_hi) o->nnz_hi[r] = nlo + nmaybe;
        Llo += lo;
        Lhi += hi;
    }
    if (o->loss_lo) o->loss_lo[0] = Llo / (double)R;
    if (o->loss_hi) o->loss_hi[0] = Lhi / (double)R;
    free(iwe);
    free(hit);
    free(mb);
    return ORC_OK;
}

int orc_abi_version(void) { return 2; }
