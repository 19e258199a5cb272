// cm_geo.cu -- the geometry-consistency loss (Sec. 3.2, Eq. 3) and its
// gradient to both views' inverse depths and the camera motion between them.
//
// Every pixel x of view 0 (depth 1/rho0) is moved by the camera motion (the
// rigid transform of cm_pose.cuh, P = R X + t); its forward-projected depth is
// a = P2 and its projection x' = x + d (the displacement d of cm_pose.cuh)
// lands in view 1, where the interpolated depth b is the bilinear sample of
// 1/rho1 at x' (corner indices clamped).  Valid pixels: P2 > 0 and x' inside
// the closed image box.  L_geo = (1/|V|) sum_V |a - b| / (a + b).
// The projection is kept as the pixel plus the FP32 displacement of
// cm_pose.cuh (cell u + floor(d.x), fractional part d.x - floor(d.x)), and b
// and the sign of a - b are computed with correctly rounded operations
// (geo_pixel), so the valid set, the sample cells and the branch of |a - b|
// are fixed functions of the inputs; sums are fixed-order (per-tile partials,
// FP64 final).
#include <cmath>
#include <cstdint>

#include "../../include/cm.h"
#include "cm_launch.h"
#include "cm_pose.cuh"

namespace cmk {

namespace {

constexpr int kGeoThreads = 256;
constexpr int kGeoPerThread = 4;
constexpr int kGeoTile = kGeoThreads * kGeoPerThread;
constexpr int kGeoPartials = 12;  // dL/dt (3) and dL/dR = sum dL/dP X^T (9)
static_assert(kGeoPartials == 12, "the backward reduces its partials with warp_sum12");

struct GeoArgs {
    int32_t W, H;
    float fx, fy, cx, cy, dt;
    const float* rho0;  // [H][W] view 0
    const float* rho1;  // [H][W] view 1
    const float* ego;   // [6] camera motion from view 0 to view 1
};

// scratch: [tiles][2] forward partials (sum, count), the valid count and the
// loss, then [tiles][12] backward partials
struct GeoScratch {
    float* fwd;
    int32_t* count;
    float* bwd;
};

GeoScratch geo_scratch(void* base, int tiles)
{
    char* p = static_cast<char*>(base);
    GeoScratch s;
    s.fwd = reinterpret_cast<float*>(p);
    s.count = reinterpret_cast<int32_t*>(p + (size_t)tiles * 2 * sizeof(float));
    s.bwd = reinterpret_cast<float*>(p + (size_t)tiles * 2 * sizeof(float) + 16);
    return s;
}

// one pixel of view 0: the decisions and the two depths
struct GeoPixel {
    bool valid;
    int ix, iy, ix1, iy1;
    float ax, ay, a, b, sg;
    float D00, D10, D01, D11;
};

__device__ __forceinline__ GeoPixel geo_pixel(const GeoArgs& g, const Pose& p, const PixelPoint& q, int u, int v)
{
    GeoPixel r;
    float P2;
    const float2 d = displacement(p, q, g.fx, g.fy, P2);
    // x' = (u + d.x, v + d.y) kept as the pixel plus the offset d: the cell is
    // u + floor(d.x) and the fractional part d.x - floor(d.x) (capped below 1),
    // without rounding x' to the coarser grid of its absolute coordinate
    r.valid = P2 > 0.0f && d.x >= (float)(-u) && d.x <= (float)(g.W - 1 - u) && d.y >= (float)(-v) &&
              d.y <= (float)(g.H - 1 - v);
    if (!r.valid) return r;
    constexpr float kBelowOne = 0x1.fffffep-1f;
    const float fx0 = floorf(d.x), fy0 = floorf(d.y);
    r.ix = u + (int)fx0;
    r.iy = v + (int)fy0;
    r.ix1 = min(r.ix + 1, g.W - 1);
    r.iy1 = min(r.iy + 1, g.H - 1);
    // b and the sign of a - b (the branch of |a - b|)
    r.ax = fminf(__fsub_rn(d.x, fx0), kBelowOne);
    r.ay = fminf(__fsub_rn(d.y, fy0), kBelowOne);
    r.D00 = __frcp_rn(__ldg(g.rho1 + (size_t)r.iy * g.W + r.ix));
    r.D10 = __frcp_rn(__ldg(g.rho1 + (size_t)r.iy * g.W + r.ix1));
    r.D01 = __frcp_rn(__ldg(g.rho1 + (size_t)r.iy1 * g.W + r.ix));
    r.D11 = __frcp_rn(__ldg(g.rho1 + (size_t)r.iy1 * g.W + r.ix1));
    const float bx = __fsub_rn(1.0f, r.ax), by = __fsub_rn(1.0f, r.ay);
    const float w00 = __fmul_rn(bx, by), w10 = __fmul_rn(r.ax, by), w01 = __fmul_rn(bx, r.ay);
    const float w11 = __fmul_rn(r.ax, r.ay);
    r.b = __fmaf_rn(w11, r.D11, __fmaf_rn(w01, r.D01, __fmaf_rn(w10, r.D10, __fmul_rn(w00, r.D00))));
    r.a = P2;
    r.sg = r.a > r.b ? 1.0f : (r.a < r.b ? -1.0f : 0.0f);
    return r;
}

// adds a to row[x0] and b to row[x1] (x1 = x0 + 1, or x0 at the right border):
// one 8-byte reduction when the pair is contiguous and 8-byte aligned (the row
// base of a W-wide image, element 0 of the image 8-byte aligned)
__device__ __forceinline__ void push_row(float* row, int x0, int x1, float a, float b)
{
    float* q = row + x0;
    if (x1 == x0 + 1 && (reinterpret_cast<uintptr_t>(q) & 7) == 0) {
        red_add_v2(q, a, b);
    } else {
        atomicAdd(q, a);
        atomicAdd(row + x1, b);
    }
}

__device__ __forceinline__ void pixel_uv32(uint32_t i, int W, int& u, int& v)
{
    const uint32_t q = i / (uint32_t)W;
    v = (int)q;
    u = (int)(i - q * (uint32_t)W);
}

__global__ void __launch_bounds__(kGeoThreads) k_geo_forward(GeoArgs g, float* __restrict__ part, int ntiles)
{
    __shared__ Pose pose;
    __shared__ float red[kGeoThreads / 32][2];
    if (threadIdx.x == 0) pose = pose_of(g.ego, g.dt);
    __syncthreads();
    const uint32_t HW = (uint32_t)g.W * (uint32_t)g.H;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        float sum = 0.0f, cnt = 0.0f;
#pragma unroll
        for (int k = 0; k < kGeoPerThread; ++k) {
            const uint32_t i = (uint32_t)tile * kGeoTile + k * kGeoThreads + threadIdx.x;
            if (i >= HW) continue;
            int u, v;
            pixel_uv32(i, g.W, u, v);
            const GeoPixel r = geo_pixel(g, pose, pixel_point(u, v, __ldg(g.rho0 + i), g.fx, g.fy, g.cx, g.cy), u, v);
            if (!r.valid) continue;
            sum += r.sg * (r.a - r.b) / (r.a + r.b);
            cnt += 1.0f;
        }
        sum = warp_sum(sum);
        cnt = warp_sum(cnt);
        if (l == 0) {
            red[w][0] = sum;
            red[w][1] = cnt;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            float s = 0.0f;
            for (int k = 0; k < kGeoThreads / 32; ++k) s += red[k][threadIdx.x];
            part[(size_t)tile * 2 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// L = sum / |V| (fixed order, FP64); the count is kept for the backward
__global__ void __launch_bounds__(64) k_geo_forward_final(const float* __restrict__ part, int ntiles,
                                                          int32_t* __restrict__ count, float* __restrict__ loss)
{
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    __shared__ double tot[2];
    double s = 0.0;
    // lane l adds tiles l, l + 32, ... in that order, eight loads in flight
    for (int i0 = l; i0 < ntiles; i0 += 32 * 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i0 + 32 * u < ntiles ? part[(size_t)(i0 + 32 * u) * 2 + c] : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)v[u];
    }
    s = warp_sum(s);
    if (l == 0) tot[c] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long n = (long long)llrint(tot[1]);
        count[0] = (int32_t)n;
        loss[0] = n > 0 ? (float)(tot[0] / (double)n) : 0.0f;
    }
}

__global__ void __launch_bounds__(kGeoThreads) k_geo_backward(GeoArgs g, const float* __restrict__ dloss,
                                                              const int32_t* __restrict__ count,
                                                              float* __restrict__ drho0, float* __restrict__ drho1,
                                                              float* __restrict__ part, int ntiles)
{
    __shared__ Pose pose;
    __shared__ float red[kGeoThreads / 32][kGeoPartials];
    if (threadIdx.x == 0) pose = pose_of(g.ego, g.dt);
    __syncthreads();
    const int n = __ldg(count);
    const float gl = n > 0 ? __ldg(dloss) / (float)n : 0.0f;
    const uint32_t HW = (uint32_t)g.W * (uint32_t)g.H;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const Pose& p = pose;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        float c[kGeoPartials];
#pragma unroll
        for (int m = 0; m < kGeoPartials; ++m) c[m] = 0.0f;
#pragma unroll
        for (int k = 0; k < kGeoPerThread; ++k) {
            const uint32_t i = (uint32_t)tile * kGeoTile + k * kGeoThreads + threadIdx.x;
            if (i >= HW) continue;
            int u, v;
            pixel_uv32(i, g.W, u, v);
            const PixelPoint q = pixel_point(u, v, __ldg(g.rho0 + i), g.fx, g.fy, g.cx, g.cy);
            const GeoPixel r = geo_pixel(g, p, q, u, v);
            if (!r.valid) {
                drho0[i] = 0.0f;
                continue;
            }
            const float a = r.a, b = r.b, s2 = (a + b) * (a + b);
            const float dfa = gl * r.sg * 2.0f * b / s2, dfb = -gl * r.sg * 2.0f * a / s2;
            const float dbx = (1.0f - r.ay) * (r.D10 - r.D00) + r.ay * (r.D11 - r.D01);
            const float dby = (1.0f - r.ax) * (r.D01 - r.D00) + r.ax * (r.D11 - r.D10);
            float X[3], P[3];
            transform(p, q, X, P);
            const float iz = 1.0f / P[2];
            // x' = fx P0/P2 + cx, y' = fy P1/P2 + cy, a = P2
            const float dP[3] = {dfb * dbx * g.fx * iz, dfb * dby * g.fy * iz,
                                 dfa - dfb * (dbx * g.fx * P[0] + dby * g.fy * P[1]) * iz * iz};
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                c[rr] += dP[rr];
#pragma unroll
                for (int ss = 0; ss < 3; ++ss) c[3 + 3 * rr + ss] += dP[rr] * X[ss];
            }
            // dL/dZ in closed form (q = R m, P = Z q + t): da/dZ = q2 and
            // dx'/dZ = fx (q0 t2 - t0 q2) / P2^2, with no difference of the
            // two nearly equal terms P0/P2 and xn
            const float q0 = p.R[0] * q.xn + p.R[1] * q.yn + p.R[2];
            const float q1 = p.R[3] * q.xn + p.R[4] * q.yn + p.R[5];
            const float q2 = p.R[6] * q.xn + p.R[7] * q.yn + p.R[8];
            const float dZ = dfa * q2 + dfb * (dbx * g.fx * (q0 * p.t[2] - p.t[0] * q2) +
                                               dby * g.fy * (q1 * p.t[2] - p.t[1] * q2)) * iz * iz;
            drho0[i] = -q.Z * q.Z * dZ;
            // b = sum_c w_c / rho1_c
            const float bx = 1.0f - r.ax, by = 1.0f - r.ay;
            push_row(drho1 + (size_t)r.iy * g.W, r.ix, r.ix1, -dfb * bx * by * r.D00 * r.D00,
                     -dfb * r.ax * by * r.D10 * r.D10);
            push_row(drho1 + (size_t)r.iy1 * g.W, r.ix, r.ix1, -dfb * bx * r.ay * r.D01 * r.D01,
                     -dfb * r.ax * r.ay * r.D11 * r.D11);
        }
        warp_sum12(c);
        if ((l & 7) == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j) red[w][3 * (l >> 3) + j] = c[j];
        }
        __syncthreads();
        if (threadIdx.x < kGeoPartials) {
            float s = 0.0f;
            for (int k = 0; k < kGeoThreads / 32; ++k) s += red[k][threadIdx.x];
            part[(size_t)tile * kGeoPartials + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kGeoPartials * 32) k_geo_backward_final(GeoArgs g, const float* __restrict__ part,
                                                                          int ntiles, float* __restrict__ dego)
{
    __shared__ double sum[kGeoPartials];
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    double s = 0.0;
    // lane l adds tiles l, l + 32, ... in that order, eight loads in flight
    for (int i0 = l; i0 < ntiles; i0 += 32 * 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = i0 + 32 * u < ntiles ? part[(size_t)(i0 + 32 * u) * kGeoPartials + c] : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)v[u];
    }
    s = warp_sum(s);
    if (l == 0) sum[c] = s;
    __syncthreads();
    if (threadIdx.x == 0) pose_grad(sum, g.ego, g.dt, dego);
}

bool geo_args(const cm_camera* cam, const float* rho0, const float* rho1, const float* ego, float dt, GeoArgs& g)
{
    if (!cam || !rho0 || !rho1 || !ego) return false;
    if (cam->width < 2 || cam->height < 2 || cam->width > 32767 || cam->height > 32767) return false;
    if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy)) return false;
    if (!std::isfinite(cam->cx) || !std::isfinite(cam->cy) || !std::isfinite(dt)) return false;
    g = GeoArgs{cam->width, cam->height, cam->fx, cam->fy, cam->cx, cam->cy, dt, rho0, rho1, ego};
    return true;
}

int geo_tiles(const cm_camera* cam) { return (int)(((size_t)cam->width * cam->height + kGeoTile - 1) / kGeoTile); }

size_t geo_bytes(int tiles) { return (size_t)tiles * 2 * sizeof(float) + 16 + (size_t)tiles * kGeoPartials * sizeof(float); }

int geo_grid(int tiles)
{
    const int cap = sm_count_current() * 8;
    return tiles < cap ? (tiles < 1 ? 1 : tiles) : cap;
}

}  // namespace

}  // namespace cmk

extern "C" {

int cm_geo_scratch_query(const cm_camera* cam, size_t* bytes)
{
    if (!cam || !bytes || cam->width < 2 || cam->height < 2) return CM_EINVAL;
    *bytes = cmk::geo_bytes(cmk::geo_tiles(cam));
    return CM_OK;
}

int cm_geo_forward(const cm_camera* cam, const float* inv_depth0, const float* inv_depth1, const float* ego6,
                   float dt, void* scratch, size_t scratch_bytes, float* loss_out, void* stream)
{
    cmk::GeoArgs g;
    if (!loss_out || !scratch || !cmk::geo_args(cam, inv_depth0, inv_depth1, ego6, dt, g)) return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return CM_EINVAL;
    const int tiles = cmk::geo_tiles(cam);
    if (scratch_bytes < cmk::geo_bytes(tiles)) return CM_ENOMEM;
    const cmk::GeoScratch sc = cmk::geo_scratch(scratch, tiles);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        cmk::KernelScope ks("k_geo_forward", s);
        cmk::k_geo_forward<<<cmk::geo_grid(tiles), cmk::kGeoThreads, 0, s>>>(g, sc.fwd, tiles);
    }
    {
        cmk::KernelScope ks("k_geo_forward_final", s);
        cmk::k_geo_forward_final<<<1, 64, 0, s>>>(sc.fwd, tiles, sc.count, loss_out);
    }
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_ECUDA;
}

int cm_geo_backward(const cm_camera* cam, const float* inv_depth0, const float* inv_depth1, const float* ego6,
                    float dt, const float* dloss, float* dinv_depth0, float* dinv_depth1, float* dego6, void* scratch,
                    size_t scratch_bytes, void* stream)
{
    cmk::GeoArgs g;
    if (!dloss || !dinv_depth0 || !dinv_depth1 || !dego6 || !scratch ||
        !cmk::geo_args(cam, inv_depth0, inv_depth1, ego6, dt, g))
        return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return CM_EINVAL;
    const int tiles = cmk::geo_tiles(cam);
    if (scratch_bytes < cmk::geo_bytes(tiles)) return CM_ENOMEM;
    const cmk::GeoScratch sc = cmk::geo_scratch(scratch, tiles);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(dinv_depth1, 0, (size_t)cam->width * cam->height * sizeof(float), s) != cudaSuccess)
        return CM_ECUDA;
    {
        cmk::KernelScope ks("k_geo_backward", s);
        cmk::k_geo_backward<<<cmk::geo_grid(tiles), cmk::kGeoThreads, 0, s>>>(g, dloss, sc.count, dinv_depth0,
                                                                               dinv_depth1, sc.bwd, tiles);
    }
    {
        cmk::KernelScope ks("k_geo_backward_final", s);
        cmk::k_geo_backward_final<<<1, cmk::kGeoPartials * 32, 0, s>>>(g, sc.bwd, tiles, dego6);
    }
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_ECUDA;
}

}  // extern "C"
