// cm_kernels.cu -- the kernels of one window: flow from depth (S1), warp +
// splat (S2-S4), loss reduction (S5), adjoint (S6), depth / ego gradient (S7),
// and their host-side launchers.
#include "cm_device.cuh"
#include "cm_launch.h"

namespace cmk {

// ---------------------------------------------------------------------------
// S1: rigid motion field (Sec. 3.2, Eq. 2 in its instantaneous form), FP32
// with the operation order stated in cm_device.cuh's contract:
//   xn = (u - cx) * (1/fx),  yn = (v - cy) * (1/fy),  xy = xn*yn
//   xd = rho * fma(xn, vz, -vx); xd = fma(xy, wx, xd); xd = fma(-fma(xn, xn, 1), wy, xd); xd = fma(yn, wz, xd)
//   yd = rho * fma(yn, vz, -vy); yd = fma(fma(yn, yn, 1), wx, yd); yd = fma(-xy, wy, yd); yd = fma(-xn, wz, yd)
//   flow = ((dt*fx) * xd, (dt*fy) * yd)
__device__ __forceinline__ float2 motion_field(int u, int v, float rho, const float* __restrict__ ego, float fx,
                                               float fy, float cx, float cy, float dt)
{
    const float vx = __ldg(ego + 0), vy = __ldg(ego + 1), vz = __ldg(ego + 2);
    const float wx = __ldg(ego + 3), wy = __ldg(ego + 4), wz = __ldg(ego + 5);
    const float ifx = __fdiv_rn(1.0f, fx), ify = __fdiv_rn(1.0f, fy);
    const float sx = __fmul_rn(dt, fx), sy = __fmul_rn(dt, fy);
    const float xn = __fmul_rn(__fsub_rn((float)u, cx), ifx);
    const float yn = __fmul_rn(__fsub_rn((float)v, cy), ify);
    const float xy = __fmul_rn(xn, yn);
    float xd = __fmul_rn(rho, __fmaf_rn(xn, vz, -vx));
    xd = __fmaf_rn(xy, wx, xd);
    xd = __fmaf_rn(-__fmaf_rn(xn, xn, 1.0f), wy, xd);
    xd = __fmaf_rn(yn, wz, xd);
    float yd = __fmul_rn(rho, __fmaf_rn(yn, vz, -vy));
    yd = __fmaf_rn(__fmaf_rn(yn, yn, 1.0f), wx, yd);
    yd = __fmaf_rn(-xy, wy, yd);
    yd = __fmaf_rn(-xn, wz, yd);
    return make_float2(__fmul_rn(sx, xd), __fmul_rn(sy, yd));
}

__global__ void __launch_bounds__(256) k_flow(int W, int H, const float* __restrict__ rho,
                                              const float* __restrict__ ego, float fx, float fy, float cx, float cy,
                                              float dt, float2* __restrict__ flow)
{
    const size_t HW = (size_t)W * H;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / W), u = (int)(i - (size_t)v * W);
        flow[i] = motion_field(u, v, __ldg(rho + i), ego, fx, fy, cx, cy, dt);
    }
}

// ---------------------------------------------------------------------------
// S2-S4: one thread per event (grid-stride)
template <int MAXB>
__global__ void __launch_bounds__(kEventThreads) k_splat(Win d)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x)
        splat_event<MAXB>(d, k);
}

// S6: one thread per event (grid-stride)
template <int MAXB>
__global__ void __launch_bounds__(kEventThreads) k_adjoint(Win d)
{
    const float dl = __ldg(d.dloss);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x)
        adjoint_event<MAXB>(d, k, dl);
}

// ---------------------------------------------------------------------------
// S5: loss.  Pass 1 (grid = loss_tiles x R): per pixel T = S/(C+eps) for both
// polarities, sum of T^2 and the non-empty count per tile; the plane is
// rewritten in place as (A+, T+, A-, T-) with A = 2T/(C+eps), which is all the
// adjoint needs.  Pass 2 (one block): fixed-order reduction of the tiles.
__global__ void __launch_bounds__(256) k_loss_partial(Win d)
{
    const int r = blockIdx.y;
    const size_t HW = plane_size(d);
    float4* plane = d.iwe + (size_t)r * HW;
    const float eps = d.eps;
    float s = 0.0f;
    int cnt = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const float4 q = plane[i];
        const float cp = q.x + eps, cm = q.z + eps;
        const float tp = q.y / cp, tm = q.w / cm;
        s = fmaf(tp, tp, s);
        s = fmaf(tm, tm, s);
        cnt += (q.x > 0.0f || q.z > 0.0f) ? 1 : 0;
        plane[i] = make_float4(2.0f * tp / cp, tp, 2.0f * tm / cm, tm);
    }
    __shared__ float ss[8];
    __shared__ int sc[8];
    s = warp_sum(s);
    cnt = warp_sum(cnt);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ss[w] = s;
        sc[w] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.0f;
        int c = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            a += ss[i];
            c += sc[i];
        }
        d.loss_part[(size_t)r * d.loss_tiles + blockIdx.x] = make_float2(a, (float)c);
    }
}

__global__ void __launch_bounds__(1024) k_loss_final(Win d)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ double lr[64];
    for (int r = w; r < d.R; r += nw) {
        double s = 0.0, c = 0.0;
        for (int i = l; i < d.loss_tiles; i += 32) {
            const float2 q = d.loss_part[(size_t)r * d.loss_tiles + i];
            s += (double)q.x;
            c += (double)q.y;
        }
        s = warp_sum(s);
        c = warp_sum(c);
        if (l == 0) {
            const double L = s / (c + (double)d.eps);
            lr[r] = L;
            d.loss_r[r] = (float)L;
            d.nnz_r[r] = (int32_t)c;
            d.norm[r] = (float)(1.0 / ((double)d.R * (c + (double)d.eps)));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0;
        for (int r = 0; r < d.R; ++r) L += lr[r];
        d.loss[0] = (float)(L / d.R);
    }
}

// ---------------------------------------------------------------------------
// S7: dL/d(rho) per pixel and the six dL/d(ego) sums (fixed-order reduction)
__global__ void __launch_bounds__(256) k_depth_ego(Win d)
{
    const int W = d.W;
    const size_t HW = plane_size(d);
    const float vx = __ldg(d.ego + 0), vy = __ldg(d.ego + 1), vz = __ldg(d.ego + 2);
    const float ifx = 1.0f / d.fx, ify = 1.0f / d.fy;
    const float sx = d.dt * d.fx, sy = d.dt * d.fy;
    float g[6] = {0, 0, 0, 0, 0, 0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (size_t)gridDim.x * blockDim.x) {
        const int v = (int)(i / W), u = (int)(i - (size_t)v * W);
        const float xn = ((float)u - d.cx) * ifx, yn = ((float)v - d.cy) * ify;
        const float r = __ldg(d.rho + i);
        const float2 df = d.dflow[i];
        const float Gx = sx * df.x, Gy = sy * df.y;
        if (d.drho) d.drho[i] = Gx * (xn * vz - vx) + Gy * (yn * vz - vy);
        g[0] -= r * Gx;
        g[1] -= r * Gy;
        g[2] += r * (xn * Gx + yn * Gy);
        g[3] += xn * yn * Gx + (1.0f + yn * yn) * Gy;
        g[4] -= (1.0f + xn * xn) * Gx + xn * yn * Gy;
        g[5] += yn * Gx - xn * Gy;
    }
    __shared__ float sg[8][6];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const float v = warp_sum(g[c]);
        if (l == 0) sg[w][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float a = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += sg[i][threadIdx.x];
        d.dego_part[(size_t)blockIdx.x * 6 + threadIdx.x] = a;
    }
}

__global__ void __launch_bounds__(192) k_depth_ego_final(Win d)
{
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    double s = 0.0;
    for (int i = l; i < d.pix_tiles; i += 32) s += (double)d.dego_part[(size_t)i * 6 + c];
    s = warp_sum(s);
    if (l == 0 && d.dego) d.dego[c] = (float)s;
}

// ---------------------------------------------------------------------------
// launchers

static int event_grid(int64_t n, int sm_count)
{
    const int64_t blocks = (n + kEventThreads - 1) / kEventThreads;
    const int64_t cap = (int64_t)sm_count * 8;
    return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

cudaError_t launch_flow(const Win& d, cudaStream_t st)
{
    const size_t HW = (size_t)d.W * d.H;
    const int grid = (int)((HW + 255) / 256 < 4096 ? (HW + 255) / 256 : 4096);
    KernelScope ks("k_flow", st);
    k_flow<<<grid, 256, 0, st>>>(d.W, d.H, d.rho, d.ego, d.fx, d.fy, d.cx, d.cy, d.dt, const_cast<float2*>(d.flow));
    return cudaGetLastError();
}

cudaError_t launch_splat(const Win& d, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaSuccess;
    const int g = event_grid(d.n, sm_count);
    KernelScope ks("k_splat", st);
    if (d.B <= 1) k_splat<1><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 10) k_splat<10><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 20) k_splat<20><<<g, kEventThreads, 0, st>>>(d);
    else k_splat<32><<<g, kEventThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(const Win& d, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaSuccess;
    const int g = event_grid(d.n, sm_count);
    KernelScope ks("k_adjoint", st);
    if (d.B <= 1) k_adjoint<1><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 10) k_adjoint<10><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 20) k_adjoint<20><<<g, kEventThreads, 0, st>>>(d);
    else k_adjoint<32><<<g, kEventThreads, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_loss(const Win& d, cudaStream_t st)
{
    {
        KernelScope ks("k_loss_partial", st);
        k_loss_partial<<<dim3(d.loss_tiles, d.R), 256, 0, st>>>(d);
    }
    {
        KernelScope ks("k_loss_final", st);
        k_loss_final<<<1, 1024, 0, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_depth_ego(const Win& d, cudaStream_t st)
{
    {
        KernelScope ks("k_depth_ego", st);
        k_depth_ego<<<d.pix_tiles, 256, 0, st>>>(d);
    }
    {
        KernelScope ks("k_depth_ego_final", st);
        k_depth_ego_final<<<1, 192, 0, st>>>(d);
    }
    return cudaGetLastError();
}

}  // namespace cmk
