// cm_eq2.cu -- the discrete flow of Eq. 2 with one pose per bin (Sec. 3.2),
// and its adjoint through the projection, the rigid transform and Rodrigues'
// formula.
//
// Bin i moves the camera with velocity v_i and angular velocity w_i for dt
// seconds: a pixel's point X = (xn, yn, 1) / rho maps to P = R X + t with
// R = Rodrigues(k), k = -w dt, t = -v dt, and its flow is `scale` times the
// displacement fx (P0/P2 - xn), fy (P1/P2 - yn) (scale = number of bins gives
// px per window, the unit of the iterative warp).
//
// The FP32 operation sequence of the rotation and of the displacement d is
// stated in cm_pose.cuh; the flow is (scale * d.x, scale * d.y).
// The adjoint is FP32 per pixel with fixed-order FP64 final sums; the
// derivative of Rodrigues' formula is taken in FP64 once per bin.
#include <cmath>
#include <cstdint>

#include "../../include/cm.h"
#include "cm_launch.h"
#include "cm_pose.cuh"

namespace cmk {

namespace {

constexpr int kEq2Threads = 256;
constexpr int kEq2Partials = 12;  // dL/dt (3) and dL/dR = sum dL/dP X^T (9), per bin and tile
static_assert(kEq2Partials == 12, "the adjoint reduces its partials with warp_sum12");

struct Eq2Args {
    int32_t W, H, nb;
    float fx, fy, cx, cy, dt, scale;
    const float* rho;   // [H][W]
    const float* ego;   // [nb][6]
};

// flow of every bin at every pixel; the block's poses are built once in shared
// memory, packed for the displacement (the pixel loop is instruction-bound)
__global__ void __launch_bounds__(kEq2Threads) k_flow_eq2(Eq2Args a, float2* __restrict__ flow)
{
    __shared__ PoseD poses[CM_MAX_BINS];
    if (threadIdx.x < a.nb) poses[threadIdx.x] = pack_displacement(pose_of(a.ego + 6 * threadIdx.x, a.dt));
    __syncthreads();
    const uint32_t HW = (uint32_t)a.W * (uint32_t)a.H;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += gridDim.x * blockDim.x) {
        const uint32_t v = i / (uint32_t)a.W, u = i - v * (uint32_t)a.W;
        const PixelPoint q = pixel_point((int)u, (int)v, __ldg(a.rho + i), a.fx, a.fy, a.cx, a.cy);
        for (int b = 0; b < a.nb; ++b) {
            float P2;
            const float2 d = displacement(poses[b], q, a.fx, a.fy, P2);
            flow[(size_t)b * HW + i] = make_float2(__fmul_rn(a.scale, d.x), __fmul_rn(a.scale, d.y));
        }
    }
}

// Pixels per thread of the adjoint: a thread keeps its pixels' points in
// registers and reads each bin's pose from shared memory once for all of them.
constexpr int kEq2PerThread = 4;
constexpr int kEq2Tile = kEq2Threads * kEq2PerThread;

// Adjoint per tile of kEq2Tile pixels (kEq2PerThread per thread, strided by
// the block size): dL/d(rho) per pixel (summed over the bins), and per bin the
// tile's twelve sums dL/dt, dL/dR (one warp reduction per bin and warp, one
// barrier per tile).
__global__ void __launch_bounds__(kEq2Threads, 3) k_flow_eq2_grad(Eq2Args a, const float2* __restrict__ dflow,
                                                                  float* __restrict__ drho, float* __restrict__ part,
                                                                  int ntiles)
{
    __shared__ Pose poses[CM_MAX_BINS];
    // per warp, bin and component: the warp's sum
    __shared__ float red[kEq2Threads / 32][CM_MAX_BINS][kEq2Partials];
    if (threadIdx.x < a.nb) poses[threadIdx.x] = pose_of(a.ego + 6 * threadIdx.x, a.dt);
    __syncthreads();
    const uint32_t HW = (uint32_t)a.W * (uint32_t)a.H;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        PixelPoint q[kEq2PerThread];
        float dr[kEq2PerThread];
#pragma unroll
        for (int k = 0; k < kEq2PerThread; ++k) {
            const uint32_t i = (uint32_t)tile * kEq2Tile + k * kEq2Threads + threadIdx.x;
            dr[k] = 0.0f;
            q[k] = PixelPoint{0.0f, 0.0f, 0.0f};
            if (i < HW) {
                const uint32_t v = i / (uint32_t)a.W, u = i - v * (uint32_t)a.W;
                q[k] = pixel_point((int)u, (int)v, __ldg(a.rho + i), a.fx, a.fy, a.cx, a.cy);
            }
        }
        for (int b = 0; b < a.nb; ++b) {
            const Pose p = poses[b];
            float2 g[kEq2PerThread];
#pragma unroll
            for (int k = 0; k < kEq2PerThread; ++k) {
                const uint32_t i = (uint32_t)tile * kEq2Tile + k * kEq2Threads + threadIdx.x;
                g[k] = i < HW ? __ldg(dflow + (size_t)b * HW + i) : make_float2(0.0f, 0.0f);
            }
            float c[kEq2Partials];
#pragma unroll
            for (int m = 0; m < kEq2Partials; ++m) c[m] = 0.0f;
#pragma unroll
            for (int k = 0; k < kEq2PerThread; ++k) {
                const uint32_t i = (uint32_t)tile * kEq2Tile + k * kEq2Threads + threadIdx.x;
                if (i >= HW) continue;
                float X[3], P[3];
                transform(p, q[k], X, P);
                const float iz = recip(P[2]);  // hardware reciprocal: the adjoint is ALU-bound
                const float Gx = a.scale * g[k].x * a.fx, Gy = a.scale * g[k].y * a.fy;
                const float dP[3] = {Gx * iz, Gy * iz, -(Gx * P[0] + Gy * P[1]) * iz * iz};
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    c[r] += dP[r];
#pragma unroll
                    for (int s = 0; s < 3; ++s) c[3 + 3 * r + s] += dP[r] * X[s];
                }
                // dL/d(rho) = -Z^2 dL/dZ.  With m = (xn, yn, 1), P = Z R m + t and
                // e0 = P0 - xn P2 = Z s0 + u0 (s0 = sum_c (A_0c - xn A_2c) m_c,
                // A = R - I, u0 = t0 - xn t2):  d(fx e0/P2)/dZ = fx (s0 t2 - u0 q2) / P2^2,
                // q2 = (R m)_2, and likewise for y.  Written this way the two
                // nearly equal terms of the direct chain (xn P2 against P0) never
                // meet, so the derivative keeps FP32 relative precision (it is 0
                // for a pure rotation, as it should be).
                const PixelPoint& pq = q[k];
                const float q2 = p.R[6] * pq.xn + p.R[7] * pq.yn + p.R[8];
                const float s0 = (p.Ad[0] - pq.xn * p.R[6]) * pq.xn + (p.R[1] - pq.xn * p.R[7]) * pq.yn +
                                 (p.R[2] - pq.xn * p.Ad[2]);
                const float s1 = (p.R[3] - pq.yn * p.R[6]) * pq.xn + (p.Ad[1] - pq.yn * p.R[7]) * pq.yn +
                                 (p.R[5] - pq.yn * p.Ad[2]);
                const float u0 = p.t[0] - pq.xn * p.t[2], u1 = p.t[1] - pq.yn * p.t[2];
                const float dZ = (Gx * (s0 * p.t[2] - u0 * q2) + Gy * (s1 * p.t[2] - u1 * q2)) * iz * iz;
                dr[k] -= pq.Z * pq.Z * dZ;
            }
            warp_sum12(c);
            if ((l & 7) == 0) {
#pragma unroll
                for (int j = 0; j < 3; ++j) red[w][b][3 * (l >> 3) + j] = c[j];
            }
        }
#pragma unroll
        for (int k = 0; k < kEq2PerThread; ++k) {
            const uint32_t i = (uint32_t)tile * kEq2Tile + k * kEq2Threads + threadIdx.x;
            if (i < HW) drho[i] = dr[k];
        }
        __syncthreads();
        // the tile's partial of every (bin, component): its warps' sums in a fixed order
        for (int j = threadIdx.x; j < a.nb * kEq2Partials; j += blockDim.x) {
            const int b = j / kEq2Partials, m = j - b * kEq2Partials;
            float s = 0.0f;
            for (int k = 0; k < kEq2Threads / 32; ++k) s += red[k][b][m];
            part[((size_t)tile * a.nb + b) * kEq2Partials + m] = s;
        }
        __syncthreads();
    }
}

// per bin (one block): fixed-order FP64 sums of the tiles' partials, then
// dL/dv = -dt dL/dt and dL/dw_c = -dt sum dL/dR_ab dR_ab/dk_c
__global__ void __launch_bounds__(kEq2Partials * 32) k_flow_eq2_final(Eq2Args a, const float* __restrict__ part,
                                                                      int ntiles, float* __restrict__ dego)
{
    __shared__ double sum[kEq2Partials];
    const int b = blockIdx.x, c = threadIdx.x >> 5, l = threadIdx.x & 31;
    double s = 0.0;
    for (int i0 = l; i0 < ntiles; i0 += 32 * 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = i0 + 32 * u < ntiles ? part[((size_t)(i0 + 32 * u) * a.nb + b) * kEq2Partials + c] : 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)v[u];
    }
    s = warp_sum(s);
    if (l == 0) sum[c] = s;
    __syncthreads();
    if (threadIdx.x == 0) pose_grad(sum, a.ego + 6 * b, a.dt, dego + 6 * b);
}


bool eq2_args(const cm_camera* cam, const float* rho, const float* ego, int32_t nb, float dt, float scale, Eq2Args& a)
{
    if (!cam || !rho || !ego || nb < 1 || nb > CM_MAX_BINS) return false;
    if (cam->width < 2 || cam->height < 2 || cam->width > 32767 || cam->height > 32767) return false;
    if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy)) return false;
    if (!std::isfinite(cam->cx) || !std::isfinite(cam->cy) || !std::isfinite(dt) || !std::isfinite(scale)) return false;
    a = Eq2Args{cam->width, cam->height, nb, cam->fx, cam->fy, cam->cx, cam->cy, dt, scale, rho, ego};
    return true;
}

int eq2_tiles(const cm_camera* cam) { return (int)(((size_t)cam->width * cam->height + kEq2Tile - 1) / kEq2Tile); }

// blocks of a launch over `units` units of work: at most `per_sm` resident
// blocks on every SM, the units distributed over them in whole rounds
int grid_for(int units, int per_sm)
{
    const int cap = sm_count_current() * per_sm;
    return units < cap ? (units < 1 ? 1 : units) : cap;
}

}  // namespace

}  // namespace cmk

extern "C" {

int cm_flow_eq2(const cm_camera* cam, const float* inv_depth, const float* ego6, int32_t nb, float dt_bin,
                float scale, float* flow_out, void* stream)
{
    cmk::Eq2Args a;
    if (!flow_out || !cmk::eq2_args(cam, inv_depth, ego6, nb, dt_bin, scale, a)) return CM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tiles = (int)(((size_t)cam->width * cam->height + cmk::kEq2Threads - 1) / cmk::kEq2Threads);
    cmk::KernelScope ks("k_flow_eq2", s);
    cmk::k_flow_eq2<<<cmk::grid_for(tiles, 8), cmk::kEq2Threads, 0, s>>>(a, reinterpret_cast<float2*>(flow_out));
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_ECUDA;
}

int cm_flow_eq2_scratch_query(const cm_camera* cam, int32_t nb, size_t* bytes)
{
    if (!cam || !bytes || nb < 1 || nb > CM_MAX_BINS || cam->width < 2 || cam->height < 2) return CM_EINVAL;
    *bytes = (size_t)cmk::eq2_tiles(cam) * nb * cmk::kEq2Partials * sizeof(float);
    return CM_OK;
}

int cm_flow_eq2_backward(const cm_camera* cam, const float* inv_depth, const float* ego6, int32_t nb, float dt_bin,
                         float scale, const float* dflow, float* dinv_depth, float* dego6, void* scratch,
                         size_t scratch_bytes, void* stream)
{
    cmk::Eq2Args a;
    if (!dflow || !dinv_depth || !dego6 || !scratch || !cmk::eq2_args(cam, inv_depth, ego6, nb, dt_bin, scale, a))
        return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return CM_EINVAL;
    size_t need = 0;
    cm_flow_eq2_scratch_query(cam, nb, &need);
    if (scratch_bytes < need) return CM_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tiles = cmk::eq2_tiles(cam);
    float* part = static_cast<float*>(scratch);
    {
        cmk::KernelScope ks("k_flow_eq2_grad", s);
        cmk::k_flow_eq2_grad<<<cmk::grid_for(tiles, 3), cmk::kEq2Threads, 0, s>>>(
            a, reinterpret_cast<const float2*>(dflow), dinv_depth, part, tiles);
    }
    {
        cmk::KernelScope ks("k_flow_eq2_final", s);
        cmk::k_flow_eq2_final<<<nb, cmk::kEq2Partials * 32, 0, s>>>(a, part, tiles, dego6);
    }
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_ECUDA;
}

}  // extern "C"
