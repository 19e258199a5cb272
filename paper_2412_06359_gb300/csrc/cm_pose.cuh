// cm_pose.cuh -- the rigid motion of a camera between two views (Sec. 3.2,
// Eq. 2) as the kernels compute it: the rotation by Rodrigues' formula, the
// transform of a pixel's back-projected point, and the derivative of the
// rotation with respect to its exponential coordinates.  Shared by the
// discrete flow (cm_eq2.cu) and the geometry-consistency loss (cm_geo.cu).
//
// A camera moving with velocity v and angular velocity w for dt seconds maps
// the point X of a pixel (X = (xn, yn, 1) / rho) to P = R X + t with
// R = Rodrigues(k), k = -w dt, t = -v dt.
//
// FP32 arithmetic contract.  The projected positions decide integer outcomes
// downstream (cells, supports, the mask, valid pixels), so every operation is
// one explicit correctly rounded single-precision operation in a fixed order:
//   per bin:   kxx = kx*kx, kyy = ky*ky, kzz = kz*kz, kxy = kx*ky, kxz = kx*kz, kyz = ky*kz
//              s = (kxx + kyy) + kzz
//              a = sin(th)/th, b = (1 - cos th)/th^2 as Taylor series in s through s^9,
//                  Horner from the highest term: c = fma(c, s, c_n)
//              R00 = fma(b, -(kyy + kzz), 1)  R01 = fma(b, kxy, -(a*kz))  R02 = fma(b, kxz, a*ky)
//              R10 = fma(b, kxy, a*kz)        R11 = fma(b, -(kxx + kzz), 1) R12 = fma(b, kyz, -(a*kx))
//              R20 = fma(b, kxz, -(a*ky))     R21 = fma(b, kyz, a*kx)     R22 = fma(b, -(kxx + kyy), 1)
//              Ad_i = b * -(...), the diagonal of A = R - I (the same sums as R_ii)
//   per pixel: xn = (u - cx) * (1/fx), yn = (v - cy) * (1/fy), Z = 1/rho, m = (xn, yn, 1)
//              c_0j = fma(-xn, A_2j, A_0j), c_1j = fma(-yn, A_2j, A_1j)     (j = 0, 1, 2)
//              s0 = fma(c_00, xn, fma(c_01, yn, c_02)),  s1 = fma(c_10, xn, fma(c_11, yn, c_12))
//              e0 = fma(Z, s0, fma(-xn, t2, t0)),        e1 = fma(Z, s1, fma(-yn, t2, t1))
//              P2 = fma(Z, fma(R20, xn, fma(R21, yn, R22)), t2),  iz = 1/P2
//              displacement d = (fx * (e0 * iz), fy * (e1 * iz))
// e0 is P0 - xn P2 (P = R X + t, X = Z m), so d = fx (P0/P2 - xn), the
// displacement of the pixel, taken in a form that is exactly 0 for a camera
// at rest and never cancels two large terms.
// Every 1/x above is one correctly rounded reciprocal (__frcp_rn: the same
// value as the correctly rounded division 1/x, in fewer instructions).
#pragma once

#include <cmath>
#include <cstdint>

#include "cm_device.cuh"

namespace cmk {

// Taylor coefficients of sin(th)/th and (1 - cos th)/th^2 in s = th^2
__device__ constexpr float kSinSeries[10] = {
    (float)1.0, (float)(-1.0 / 6.0), (float)(1.0 / 120.0), (float)(-1.0 / 5040.0), (float)(1.0 / 362880.0),
    (float)(-1.0 / 39916800.0), (float)(1.0 / 6227020800.0), (float)(-1.0 / 1307674368000.0),
    (float)(1.0 / 355687428096000.0), (float)(-1.0 / 121645100408832000.0)};
__device__ constexpr float kCosSeries[10] = {
    (float)(1.0 / 2.0), (float)(-1.0 / 24.0), (float)(1.0 / 720.0), (float)(-1.0 / 40320.0),
    (float)(1.0 / 3628800.0), (float)(-1.0 / 479001600.0), (float)(1.0 / 87178291200.0),
    (float)(-1.0 / 20922789888000.0), (float)(1.0 / 6402373705728000.0), (float)(-1.0 / 2432902008176640000.0)};

struct Pose {
    float R[9];
    float t[3];
    float Ad[3];  // diagonal of R - I, computed directly (no cancellation against 1)
};

__device__ __forceinline__ Pose pose_of(const float* __restrict__ e, float dt)
{
    Pose p;
    const float kx = -__fmul_rn(__ldg(e + 3), dt), ky = -__fmul_rn(__ldg(e + 4), dt), kz = -__fmul_rn(__ldg(e + 5), dt);
    p.t[0] = -__fmul_rn(__ldg(e + 0), dt);
    p.t[1] = -__fmul_rn(__ldg(e + 1), dt);
    p.t[2] = -__fmul_rn(__ldg(e + 2), dt);
    const float kxx = __fmul_rn(kx, kx), kyy = __fmul_rn(ky, ky), kzz = __fmul_rn(kz, kz);
    const float kxy = __fmul_rn(kx, ky), kxz = __fmul_rn(kx, kz), kyz = __fmul_rn(ky, kz);
    const float s = __fadd_rn(__fadd_rn(kxx, kyy), kzz);
    float a = kSinSeries[9], b = kCosSeries[9];
#pragma unroll
    for (int n = 8; n >= 0; --n) {
        a = __fmaf_rn(a, s, kSinSeries[n]);
        b = __fmaf_rn(b, s, kCosSeries[n]);
    }
    p.Ad[0] = __fmul_rn(b, -__fadd_rn(kyy, kzz));
    p.Ad[1] = __fmul_rn(b, -__fadd_rn(kxx, kzz));
    p.Ad[2] = __fmul_rn(b, -__fadd_rn(kxx, kyy));
    p.R[0] = __fmaf_rn(b, -__fadd_rn(kyy, kzz), 1.0f);
    p.R[1] = __fmaf_rn(b, kxy, -__fmul_rn(a, kz));
    p.R[2] = __fmaf_rn(b, kxz, __fmul_rn(a, ky));
    p.R[3] = __fmaf_rn(b, kxy, __fmul_rn(a, kz));
    p.R[4] = __fmaf_rn(b, -__fadd_rn(kxx, kzz), 1.0f);
    p.R[5] = __fmaf_rn(b, kyz, -__fmul_rn(a, kx));
    p.R[6] = __fmaf_rn(b, kxz, -__fmul_rn(a, ky));
    p.R[7] = __fmaf_rn(b, kyz, __fmul_rn(a, kx));
    p.R[8] = __fmaf_rn(b, -__fadd_rn(kxx, kyy), 1.0f);
    return p;
}

// the camera-frame point of pixel (u, v) and its normalised coordinates
// Sums of c[0..11] over the 32 lanes of a warp by recursive halving (each lane
// passes on the half it does not keep: 6 + 3 exchanges, then three butterfly
// steps on 3 values; 18 shuffles instead of 60).  Afterwards c[0..2] of lane l
// hold the sums of elements 3 (l >> 3) .. 3 (l >> 3) + 2.
__device__ __forceinline__ void warp_sum12(float (&c)[12])
{
    const int l = threadIdx.x & 31;
    const bool h16 = (l & 16) != 0, h8 = (l & 8) != 0;
    float h[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float keep = h16 ? c[6 + j] : c[j], give = h16 ? c[j] : c[6 + j];
        h[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float keep = h8 ? h[3 + j] : h[j], give = h8 ? h[j] : h[3 + j];
        c[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
#pragma unroll
    for (int o = 4; o >= 1; o >>= 1)
#pragma unroll
        for (int j = 0; j < 3; ++j) c[j] += __shfl_xor_sync(0xffffffffu, c[j], o);
}

struct PixelPoint {
    float xn, yn, Z;
};

__device__ __forceinline__ PixelPoint pixel_point(int u, int v, float rho, float fx, float fy, float cx, float cy)
{
    PixelPoint q;
    q.xn = __fmul_rn(__fsub_rn((float)u, cx), __frcp_rn(fx));
    q.yn = __fmul_rn(__fsub_rn((float)v, cy), __frcp_rn(fy));
    q.Z = __frcp_rn(rho);  // correctly rounded 1/rho (the same value as the division)
    return q;
}

// the displacement of the pixel and the depth P2 of its moved point (the
// sequence of the contract above), from the thirteen entries of the pose it uses
__device__ __forceinline__ float2 displacement_of(float Ad0, float R1, float R2, float R3, float Ad1, float R5,
                                                  float R6, float R7, float Ad2, float R8, float t0, float t1,
                                                  float t2, const PixelPoint& q, float fx, float fy, float& P2)
{
    const float xn = q.xn, yn = q.yn;
    const float c00 = __fmaf_rn(-xn, R6, Ad0), c01 = __fmaf_rn(-xn, R7, R1);
    const float c02 = __fmaf_rn(-xn, Ad2, R2);
    const float c10 = __fmaf_rn(-yn, R6, R3), c11 = __fmaf_rn(-yn, R7, Ad1);
    const float c12 = __fmaf_rn(-yn, Ad2, R5);
    const float s0 = __fmaf_rn(c00, xn, __fmaf_rn(c01, yn, c02));
    const float s1 = __fmaf_rn(c10, xn, __fmaf_rn(c11, yn, c12));
    const float e0 = __fmaf_rn(q.Z, s0, __fmaf_rn(-xn, t2, t0));
    const float e1 = __fmaf_rn(q.Z, s1, __fmaf_rn(-yn, t2, t1));
    P2 = __fmaf_rn(q.Z, __fmaf_rn(R6, xn, __fmaf_rn(R7, yn, R8)), t2);
    const float iz = __frcp_rn(P2);  // correctly rounded 1/P2
    return make_float2(__fmul_rn(fx, __fmul_rn(e0, iz)), __fmul_rn(fy, __fmul_rn(e1, iz)));
}

__device__ __forceinline__ float2 displacement(const Pose& p, const PixelPoint& q, float fx, float fy, float& P2)
{
    return displacement_of(p.Ad[0], p.R[1], p.R[2], p.R[3], p.Ad[1], p.R[5], p.R[6], p.R[7], p.Ad[2], p.R[8], p.t[0],
                           p.t[1], p.t[2], q, fx, fy, P2);
}

// The entries of a pose the displacement uses, packed for three 16-byte and
// one 4-byte shared-memory loads: (Ad0, R01, R02, R10), (Ad1, R12, R20, R21),
// (Ad2, R22, t0, t1), t2.
struct PoseD {
    float4 a, b, c;
    float t2;
};

__device__ __forceinline__ PoseD pack_displacement(const Pose& p)
{
    return PoseD{make_float4(p.Ad[0], p.R[1], p.R[2], p.R[3]), make_float4(p.Ad[1], p.R[5], p.R[6], p.R[7]),
                 make_float4(p.Ad[2], p.R[8], p.t[0], p.t[1]), p.t[2]};
}

__device__ __forceinline__ float2 displacement(const PoseD& p, const PixelPoint& q, float fx, float fy, float& P2)
{
    return displacement_of(p.a.x, p.a.y, p.a.z, p.a.w, p.b.x, p.b.y, p.b.z, p.b.w, p.c.x, p.c.y, p.c.z, p.c.w, p.t2,
                           q, fx, fy, P2);
}

__device__ __forceinline__ void transform(const Pose& p, const PixelPoint& q, float X[3], float P[3])
{
    X[0] = __fmul_rn(q.Z, q.xn);
    X[1] = __fmul_rn(q.Z, q.yn);
    X[2] = q.Z;
#pragma unroll
    for (int r = 0; r < 3; ++r)
        P[r] = __fmaf_rn(p.R[3 * r + 2], X[2], __fmaf_rn(p.R[3 * r + 1], X[1], __fmaf_rn(p.R[3 * r], X[0], p.t[r])));
}

// Derivative of Rodrigues' formula R(k) = I + a K + b K^2 (K = [k]x,
// a = sin(th)/th, b = (1 - cos th)/th^2) with respect to k_c, in FP64:
//   dR/dk_c = a E_c + b (E_c K + K E_c) + (a'/th K + b'/th K^2) k_c,  E_c = [e_c]x,
// the ratios a'/th, b'/th from their series near th = 0.
__device__ inline void rodrigues_grad(const double k[3], double dR[3][9])
{
    const double th2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const double th = sqrt(th2);
    double a, b, ap, bp;
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
    const double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    for (int c = 0; c < 3; ++c) {
        double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (c == 0) {
            E[5] = -1;
            E[7] = 1;
        } else if (c == 1) {
            E[2] = 1;
            E[6] = -1;
        } else {
            E[1] = -1;
            E[3] = 1;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double EK = 0.0, KE = 0.0;
                for (int l = 0; l < 3; ++l) {
                    EK += E[3 * i + l] * K[3 * l + j];
                    KE += K[3 * i + l] * E[3 * l + j];
                }
                dR[c][3 * i + j] = a * E[3 * i + j] + b * (EK + KE) + (ap * K[3 * i + j] + bp * K2[3 * i + j]) * k[c];
            }
    }
}

// dL/d(v, w) of one pose from the sums dL/dt (s[0..2]) and dL/dR = sum dL/dP X^T
// (s[3..11], row-major), FP64: dL/dv = -dt dL/dt, dL/dw_c = -dt sum dL/dR_ab dR_ab/dk_c
__device__ inline void pose_grad(const double s[12], const float* e, float dtf, float* out6)
{
    const double dt = (double)dtf;
    const double k[3] = {-(double)e[3] * dt, -(double)e[4] * dt, -(double)e[5] * dt};
    double dR[3][9];
    rodrigues_grad(k, dR);
    for (int j = 0; j < 3; ++j) {
        double dk = 0.0;
        for (int m = 0; m < 9; ++m) dk += s[3 + m] * dR[j][m];
        out6[j] = (float)(-dt * s[j]);
        out6[3 + j] = (float)(-dt * dk);
    }
}

}  // namespace cmk
