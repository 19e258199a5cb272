// cm_device.cuh -- device-side building blocks of the contrast-maximisation
// kernels: the window descriptor, the FP32 trajectory arithmetic and the
// bilinear sample / splat primitives.
//
// Position precision.  The floor of a trajectory position decides the flow
// cell that is sampled, the pixels a splat touches, whether a corner has a
// nonzero weight and whether the event stays inside the image; the
// eps-regularised ratio of Eq. 1 makes the loss sensitive to those decisions,
// and the second derivative of the bilinear weights makes every gradient term
// sensitive to the position itself.  A trajectory point is therefore kept as
// the event's own pixel (xk, yk), an exact integer, plus an FP32 offset
// (dx, dy) from it: the offset is at most the distance the event travels in a
// window (tens of pixels), so its rounding unit is 30-100x finer than that of
// the absolute coordinate of a 346- or 640-pixel sensor.  The cell is
// xk + floor(dx) and the fractional part dx - floor(dx).  The steps
// (Sec. 3.1 iterative warp with bilinearly sampled flow; Sec. 3.3):
//   tau     = (t - t0) / span                      span = t1 - t0
//   b       = clamp(floor(tau * B), 0, B - 1)
//   tau_j   = j / B,  h = 1 / B
//   forward:  d_{b+1} = (tau_{b+1} - tau) u_b[x_k],   d_{j+1} = d_j + h u_j(x_k + d_j)
//   backward: d_b     = -(tau - tau_b) u_b[x_k],      d_{j-1} = d_j - h u_{j-1}(x_k + d_j)
//   u(x): bilinear sample of the flow in the cell of x, corner indices clamped
// The operations are written as explicit correctly rounded single-precision
// intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn) so that the compiler
// cannot contract or reorder them: the points are a fixed function of the
// inputs, the same in every kernel that recomputes them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cmk {

constexpr int kRefEnd = 0;
constexpr int kRefAll = 1;
constexpr int kEventThreads = 256;

// Flow quad: the four flow values a bilinear sample in cell (ix, iy) reads,
// corner indices clamped to the image, a = (u00, u10), b = (u01, u11).  One
// 32-byte load of a quad replaces four 8-byte gathers, and the L2 serves random
// requests at the same rate whatever their width up to a 32-byte sector.  The
// same record layout accumulates dL/dflow: a push adds its four corner terms to
// its cell's record with two 16-byte vector reductions (instead of four 8-byte
// ones), and a per-pixel fold sums every record corner that names a pixel.
struct __align__(32) FQ {
    float4 a, b;
};

// One window: events, flow, IWE and gradient buffers, statistics.
struct Win {
    const int16_t* x;
    const int16_t* y;
    const float* t;
    const int8_t* p;
    int64_t n;
    int32_t W, H, B, R;
    int32_t ref_mode, nfb;
    float t0, span, eps;
    float dt;                // window length (depth input)
    float fx, fy, cx, cy;    // intrinsics (depth input)
    const float2* flow;      // [nfb][H][W]
    float4* iwe;             // iwe_split == 0: [R][H][W] (C+, S+, C-, S-);
                             // iwe_split == 1: [R][2][H][W] float2 (C, S), one plane per polarity
    int32_t iwe_split;
    float2* dflow;           // [nfb][H][W]; nullptr: dL/dflow of a depth window is not stored
    const FQ* fq;            // [nfb][H][W] flow quads, or nullptr (then samples gather from flow)
    FQ* dq;                  // [nfb][H][W] quad accumulators of dL/dflow, or nullptr (then pushes reduce into dflow)
    float2* warp;            // [B+1][n] trajectory points stored by the splat for the adjoint, or nullptr
                             // (then the adjoint recomputes them)
    float* norm;             // [R]: 1 / (R (N_nz(r) + eps))
    float* loss_r;           // [R]
    int32_t* nnz_r;          // [R]
    float* loss;             // [1]
    const float* dloss;      // [1]
    float2* loss_part;       // [R][loss_tiles]: (sum of T^2, non-empty count)
    int32_t loss_tiles;
    int32_t pix_tiles;
    const float* rho;        // [H][W] inverse depth
    const float* ego;        // [6]
    float* drho;             // [H][W]
    float* dego;             // [6]
    float* dego_part;        // [gradient tiles][6] (pix_tiles; loss_tiles on the batched path)
    int32_t* sync;           // [4] batched path: completion counters of the loss and gradient reductions
    int32_t* gsync;          // completion counter of the grouping's count pass: in memory that starts at
                             // zero (the plan's, or a workspace's zeroed once); the last block resets it
    // spatial grouping (batched path; tile_cnt == nullptr: events are used in their given order)
    int32_t* tile_cnt;       // tiles: [ntiles + 1] events per 32x32 tile, turned into tile starts by the scan;
                             // bands: [nty][super-chunks] events per band and super-chunk, turned into
                             // stable write offsets by the scan
    int32_t* tile_cur;       // [ntiles] scatter cursors (tiles only)
    int16_t* rx;             // [n] events grouped by tile
    int16_t* ry;
    float* rt;
    int8_t* rp;
    int32_t ntx, nty;        // tiles per row and per column (bands: 1 and the number of bands)
    int32_t band_rows;       // 0: 32x32 tiles; else rows per band (stable grouping by band)
    int32_t smem_tiles;      // 1: the window's events are splatted and pushed by the shared-memory tile
                             // kernels (grouped by kSmemTile tiles), not by the per-chunk ones
    int32_t tile_px;         // side of the grouping tiles (kBinTile or kSmemTile)
    int32_t* item_start;     // smem_tiles: [ntiles + 1] first work item of each tile, the total last
};

constexpr int kBinTile = 32;   // px, side of the tiles events are grouped by (schedule bin 1)
constexpr int kSmemTile = 32;  // px, side of the tiles of the shared-memory strategy (schedule bin 3)
constexpr int kMaxRefs = 33;  // references of a window at most (B + 1), for per-reference shared arrays

__device__ __forceinline__ size_t plane_size(const Win& d) { return (size_t)d.W * (size_t)d.H; }

// column u and row v of pixel i of a W-wide image, in 32-bit arithmetic (an
// image holds fewer than 2^31 pixels: W, H <= 32767); a 64-bit integer
// division is a long software sequence on the GPU
__device__ __forceinline__ void pixel_uv(size_t i, int W, int& u, int& v)
{
    const uint32_t ii = (uint32_t)i, w = (uint32_t)W;
    const uint32_t q = ii / w;
    v = (int)q;
    u = (int)(ii - q * w);
}

__device__ __forceinline__ const float2* field(const Win& d, int j)
{
    return d.flow + (d.nfb == 1 ? (size_t)0 : (size_t)j * plane_size(d));
}

__device__ __forceinline__ const float2* field_ptr(const Win& d, int j) { return field(d, j); }

// flow-field plane used by the push across bin j (one field for all bins, or one per bin)
__device__ __forceinline__ size_t plane_of(const Win& d, int j) { return d.nfb == 1 ? (size_t)0 : (size_t)j; }

__device__ __forceinline__ float2* field_grad(const Win& d, int j)
{
    return d.dflow + (d.nfb == 1 ? (size_t)0 : (size_t)j * plane_size(d));
}

__device__ __forceinline__ float tau_of(float t, float t0, float span)
{
    return __fdiv_rn(__fsub_rn(t, t0), span);
}

__device__ __forceinline__ int bin_of(float tau, int B)
{
    float q = floorf(__fmul_rn(tau, (float)B));
    q = fminf(fmaxf(q, 0.0f), (float)(B - 1));
    return (int)q;
}

__device__ __forceinline__ float edge_tau(int j, int B) { return __fdiv_rn((float)j, (float)B); }

// average timestamp of an event at normalised time tau for reference edge j
__device__ __forceinline__ float tbar_of(int j, int B, float tau)
{
    return __fsub_rn(1.0f, fabsf(__fsub_rn(edge_tau(j, B), tau)));
}

// the point (xk + dx, yk + dy) lies in the closed image box [0, W-1] x [0, H-1]
// (the bounds -xk and W-1-xk are exact in FP32)
__device__ __forceinline__ bool inside(int xk, int yk, float dx, float dy, int W, int H)
{
    return dx >= (float)(-xk) && dx <= (float)(W - 1 - xk) && dy >= (float)(-yk) && dy <= (float)(H - 1 - yk);
}

// Bilinear cell, fractional parts and the four weights of a point.
struct Bil {
    int ix, iy;
    float ax, ay, bx, by;
    float w00, w10, w01, w11;
};

// cell and weights of the point (xk + dx, yk + dy).  The fractional part
// dx - floor(dx) is exact except for -1 < dx < 0, where it can round up to 1;
// it is capped at the largest float below 1 (a change of at most 2^-24 px), so
// that 0 <= a < 1 always holds and the cell is always xk + floor(dx).
__device__ __forceinline__ Bil bil(int xk, int yk, float dx, float dy)
{
    constexpr float kBelowOne = 0x1.fffffep-1f;
    Bil s;
    const float fx0 = floorf(dx), fy0 = floorf(dy);
    s.ix = xk + (int)fx0;
    s.iy = yk + (int)fy0;
    s.ax = fminf(__fsub_rn(dx, fx0), kBelowOne);
    s.ay = fminf(__fsub_rn(dy, fy0), kBelowOne);
    s.bx = __fsub_rn(1.0f, s.ax);
    s.by = __fsub_rn(1.0f, s.ay);
    s.w00 = __fmul_rn(s.bx, s.by);
    s.w10 = __fmul_rn(s.ax, s.by);
    s.w01 = __fmul_rn(s.bx, s.ay);
    s.w11 = __fmul_rn(s.ax, s.ay);
    return s;
}

// the same for a point given by its fractional parts in a known cell
// (0 <= ax, ay < 1; the sort path's payload)
__device__ __forceinline__ Bil bil_frac(float ax, float ay)
{
    Bil s;
    s.ix = 0;
    s.iy = 0;
    s.ax = ax;
    s.ay = ay;
    s.bx = __fsub_rn(1.0f, ax);
    s.by = __fsub_rn(1.0f, ay);
    s.w00 = __fmul_rn(s.bx, s.by);
    s.w10 = __fmul_rn(s.ax, s.by);
    s.w01 = __fmul_rn(s.bx, s.ay);
    s.w11 = __fmul_rn(s.ax, s.ay);
    return s;
}

// Loads of data that other blocks of the same kernel may write while it runs
// (the persistent step kernel of the batched plan, NC = false) go through L2
// (ld.global.cg); loads of data fixed for the kernel's lifetime may take the
// non-coherent read-only path (NC = true, __ldg).
template <bool NC, class T>
__device__ __forceinline__ T ld_in(const T* p)
{
    if constexpr (NC) return __ldg(p);
    else return __ldcg(p);
}

// The four flow values around a cell (corner indices clamped to the image).
struct Quad {
    float2 u00, u10, u01, u11;
};

template <bool NC = true>
__device__ __forceinline__ Quad load_quad(const float2* __restrict__ U, int W, int H, const Bil& s)
{
    const int ix1 = min(s.ix + 1, W - 1), iy1 = min(s.iy + 1, H - 1);
    Quad q;
    q.u00 = ld_in<NC>(U + (size_t)s.iy * W + s.ix);
    q.u10 = ld_in<NC>(U + (size_t)s.iy * W + ix1);
    q.u01 = ld_in<NC>(U + (size_t)iy1 * W + s.ix);
    q.u11 = ld_in<NC>(U + (size_t)iy1 * W + ix1);
    return q;
}

__device__ __forceinline__ float2 interp(const Bil& s, const Quad& q)
{
    float ux = __fmul_rn(s.w00, q.u00.x);
    ux = __fmaf_rn(s.w10, q.u10.x, ux);
    ux = __fmaf_rn(s.w01, q.u01.x, ux);
    ux = __fmaf_rn(s.w11, q.u11.x, ux);
    float uy = __fmul_rn(s.w00, q.u00.y);
    uy = __fmaf_rn(s.w10, q.u10.y, uy);
    uy = __fmaf_rn(s.w01, q.u01.y, uy);
    uy = __fmaf_rn(s.w11, q.u11.y, uy);
    return make_float2(ux, uy);
}

// Trajectory points at the computed edges, as offsets from the event's pixel.
// Traj keeps them in registers (indices are compile-time after unrolling);
// SmemTraj in the block's shared memory, [edge][thread] (consecutive threads
// in consecutive banks), for the adjoint, which keeps every point live through
// its reverse sweeps while it waits on its gathers: registers it does not spend
// on the points are occupancy.
template <int MAXB>
struct Traj {
    float x_[MAXB + 1];
    float y_[MAXB + 1];
    float ex, ey;  // the point at the window end (edge B), kept in scalars so that
                   // selecting it never needs a run-time array index
    __device__ __forceinline__ float& x(int j) { return x_[j]; }
    __device__ __forceinline__ float& y(int j) { return y_[j]; }
};

template <int MAXB>
struct SmemTraj {
    float2* ps;  // this thread's column of a [MAXB + 1][kEventThreads] float2 array
    float ex, ey;
    __device__ __forceinline__ float& x(int j) { return ps[j * kEventThreads].x; }
    __device__ __forceinline__ float& y(int j) { return ps[j * kEventThreads].y; }
};

// Per-event quantities shared by the forward and backward kernels.
struct EventAt {
    int xk, yk, b, pol2;
    float tau;
};

template <bool NC = true>
__device__ __forceinline__ bool load_event(const Win& d, int64_t k, EventAt& e)
{
    e.xk = NC ? d.x[k] : __ldcg(d.x + k);
    e.yk = NC ? d.y[k] : __ldcg(d.y + k);
    if ((unsigned)e.xk >= (unsigned)d.W || (unsigned)e.yk >= (unsigned)d.H) return false;
    e.tau = tau_of(ld_in<NC>(d.t + k), d.t0, d.span);
    e.b = bin_of(e.tau, d.B);
    e.pol2 = (NC ? d.p[k] : __ldcg(d.p + k)) > 0 ? 0 : 2;
    return true;
}

// one 32-byte load of a flow quad (NC: read-only for the kernel's lifetime;
// else through L2, for quads built by another block of the same kernel)
template <bool NC = true>
__device__ __forceinline__ Quad load_fq(const FQ* p)
{
    Quad q;
    if constexpr (NC) {
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(q.u00.x), "=f"(q.u00.y), "=f"(q.u10.x), "=f"(q.u10.y), "=f"(q.u01.x), "=f"(q.u01.y),
              "=f"(q.u11.x), "=f"(q.u11.y)
            : "l"(p));
    } else {
        asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(q.u00.x), "=f"(q.u00.y), "=f"(q.u10.x), "=f"(q.u10.y), "=f"(q.u01.x), "=f"(q.u01.y),
                       "=f"(q.u11.x), "=f"(q.u11.y)
                     : "l"(p));
    }
    return q;
}

__device__ __forceinline__ size_t cell_index(const Win& d, int j, int x, int y)
{
    return (d.nfb == 1 ? (size_t)0 : (size_t)j * plane_size(d)) + (size_t)y * d.W + x;
}

// the four flow values around a cell of field j: one quad load, else four gathers
template <bool NC = true>
__device__ __forceinline__ Quad quad_at(const Win& d, int j, const Bil& s)
{
    if (d.fq) return load_fq<NC>(d.fq + cell_index(d, j, s.ix, s.iy));
    return load_quad<NC>(field(d, j), d.W, d.H, s);
}

template <bool NC = true>
__device__ __forceinline__ float2 flow_at_pixel(const Win& d, int j, int x, int y)
{
    if (d.fq) return ld_in<NC>(reinterpret_cast<const float2*>(d.fq + cell_index(d, j, x, y)));
    return ld_in<NC>(field(d, j) + (size_t)y * d.W + x);
}

// S2 + S3: the trajectory of one event through all computed edges (forward
// chain b+1..B; with all edges as references also the backward chain b..0)
// and the global mask.  Returns false when any computed point leaves the image.
template <int MAXB, bool NC = true, class TR>
__device__ __forceinline__ bool trajectory(const Win& d, const EventAt& e, TR& P)
{
    const int W = d.W, H = d.H, B = d.B, b = e.b, xk = e.xk, yk = e.yk;
    const float h = __fdiv_rn(1.0f, (float)B);
    const float2 u0 = flow_at_pixel<NC>(d, b, xk, yk);
    bool ok = true;
    const float dtf = __fsub_rn(edge_tau(b + 1, B), e.tau);
#pragma unroll
    for (int j = 1; j <= MAXB; ++j) {
        if (j <= B && j > b) {
            if (j == b + 1) {
                P.x(j) = __fmul_rn(dtf, u0.x);
                P.y(j) = __fmul_rn(dtf, u0.y);
            } else if (ok) {
                const Bil s = bil(xk, yk, P.x(j - 1), P.y(j - 1));
                const float2 u = interp(s, quad_at<NC>(d, j - 1, s));
                P.x(j) = __fmaf_rn(h, u.x, P.x(j - 1));
                P.y(j) = __fmaf_rn(h, u.y, P.y(j - 1));
            } else {
                P.x(j) = P.x(j - 1);
                P.y(j) = P.y(j - 1);
            }
            ok = ok && inside(xk, yk, P.x(j), P.y(j), W, H);
            P.ex = P.x(j);
            P.ey = P.y(j);
        }
    }
    if (d.ref_mode == kRefAll) {
        const float dtb = __fsub_rn(e.tau, edge_tau(b, B));
#pragma unroll
        for (int j = MAXB - 1; j >= 0; --j) {
            if (j <= b) {
                if (j == b) {
                    P.x(j) = __fmul_rn(-dtb, u0.x);
                    P.y(j) = __fmul_rn(-dtb, u0.y);
                } else if (ok) {
                    const Bil s = bil(xk, yk, P.x(j + 1), P.y(j + 1));
                    const float2 u = interp(s, quad_at<NC>(d, j, s));
                    P.x(j) = __fmaf_rn(-h, u.x, P.x(j + 1));
                    P.y(j) = __fmaf_rn(-h, u.y, P.y(j + 1));
                } else {
                    P.x(j) = P.x(j + 1);
                    P.y(j) = P.y(j + 1);
                }
                ok = ok && inside(xk, yk, P.x(j), P.y(j), W, H);
            }
        }
    }
    return ok;
}

// 8-byte vector reduction (no return value) into global memory.  No memory
// clobber: a kernel never reads the buffer it reduces into, so the reductions
// need no ordering against its other loads.
__device__ __forceinline__ void red_add_v2(float* addr, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b));
}

// 32-byte stores (32-byte aligned address): one instruction where two 16-byte
// stores would queue in the load/store unit
__device__ __forceinline__ void st_v8(void* p, float4 a, float4 b)
{
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

// Reciprocal by the hardware approximation (rcp.approx.ftz.f32, at most 1 ulp
// from the correctly rounded value; C + eps is a normal number).  The loss pass
// and the adjoint both take T = S * recip(C + eps) and A = 2 T recip(C + eps),
// so the adjoint recomputes exactly the loss pass's values.
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 16-byte vector reduction (16-byte aligned address), same conventions
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float e)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(e));
}

// S4: bilinear splat of one point (weight w to C_p, w * tbar to S_p) into one
// IWE plane; corners with a zero weight are skipped (they lie outside the
// image or carry nothing).
__device__ __forceinline__ void splat_point(float4* plane, int W, const Bil& s, float tbar, int pol2)
{
    float* q = reinterpret_cast<float*>(plane + (size_t)s.iy * W + s.ix) + pol2;
    red_add_v2(q, s.w00, __fmul_rn(s.w00, tbar));
    if (s.ax > 0.0f) red_add_v2(q + 4, s.w10, __fmul_rn(s.w10, tbar));
    if (s.ay > 0.0f) red_add_v2(q + 4 * (size_t)W, s.w01, __fmul_rn(s.w01, tbar));
    if (s.ax > 0.0f && s.ay > 0.0f) red_add_v2(q + 4 * (size_t)W + 4, s.w11, __fmul_rn(s.w11, tbar));
}

// One row of a splat into polarity planes of (C, S) pairs: the left corner at
// float2 index gi of the image, the right one behind it when `two`.  A pair
// that starts on a 16-byte boundary takes one 16-byte reduction, else two
// 8-byte ones (the L2 serves both widths at the same request rate).
__device__ __forceinline__ void splat_row(float2* img, size_t gi, bool two, float wl, float wr, float tbar)
{
    float* q = reinterpret_cast<float*>(img + gi);
    if (two && !(gi & 1)) {
        red_add_v4(q, wl, __fmul_rn(wl, tbar), wr, __fmul_rn(wr, tbar));
        return;
    }
    red_add_v2(q, wl, __fmul_rn(wl, tbar));
    if (two) red_add_v2(q + 2, wr, __fmul_rn(wr, tbar));
}

// S4 into the polarity-plane layout: plane 2r + polarity
__device__ __forceinline__ void splat_point_split(const Win& d, int r, const Bil& s, float tbar, int pol2)
{
    const size_t gi = (size_t)(2 * r + (pol2 >> 1)) * plane_size(d) + (size_t)s.iy * d.W + s.ix;
    float2* img = reinterpret_cast<float2*>(d.iwe);
    const bool two = s.ax > 0.0f;
    splat_row(img, gi, two, s.w00, s.w10, tbar);
    if (s.ay > 0.0f) splat_row(img, gi + d.W, two, s.w01, s.w11, tbar);
}

// Where the splat (S4) and the flow-gradient scatter (S6) go.
//
// RedSink adds into the IWE / dL/dflow with 8-byte vector reductions (the order
// of the additions is not fixed).  EmitSink writes one entry per splat point or
// push instead: a key (plane * HW + the cell of the point's top-left corner) and
// the payload (ax, ay, a, b), the point's fractional parts in that cell and two
// values; entry k * stride + slot belongs to event k, so the
// entries have a fixed order.  The sort path orders them by key (stable) and a
// per-pixel gather sums each pixel's entries in that order: bit-reproducible.
struct RedSink {
    __device__ __forceinline__ void splat(const Win& d, int r, const Bil& s, float tbar, int pol2, int64_t) const
    {
        if (d.iwe_split) splat_point_split(d, r, s, tbar, pol2);
        else splat_point(d.iwe + (size_t)r * plane_size(d), d.W, s, tbar, pol2);
    }
    // a push sampled in cell s: hs * w_c * lambda to the four corners
    __device__ __forceinline__ void scatter(const Win& d, int field, int, const Bil& s, float hx, float hy,
                                            int64_t) const
    {
        const int W = d.W;
        if (d.dq) {
            float* q = reinterpret_cast<float*>(d.dq + cell_index(d, field, s.ix, s.iy));
            red_add_v4(q, s.w00 * hx, s.w00 * hy, s.w10 * hx, s.w10 * hy);
            if (s.ay > 0.0f) red_add_v4(q + 4, s.w01 * hx, s.w01 * hy, s.w11 * hx, s.w11 * hy);
            return;
        }
        float* g = reinterpret_cast<float*>(field_grad(d, field) + (size_t)s.iy * W + s.ix);
        red_add_v2(g, s.w00 * hx, s.w00 * hy);
        if (s.ax > 0.0f) red_add_v2(g + 2, s.w10 * hx, s.w10 * hy);
        if (s.ay > 0.0f) red_add_v2(g + 2 * (size_t)W, s.w01 * hx, s.w01 * hy);
        if (s.ax > 0.0f && s.ay > 0.0f) red_add_v2(g + 2 * (size_t)W + 2, s.w11 * hx, s.w11 * hy);
    }
    // the first push of a chain, sampled at the event's own pixel
    __device__ __forceinline__ void point(const Win& d, int field, int, int xk, int yk, float vx, float vy,
                                          int64_t) const
    {
        if (d.dq) {
            red_add_v2(reinterpret_cast<float*>(d.dq + cell_index(d, field, xk, yk)), vx, vy);
            return;
        }
        red_add_v2(reinterpret_cast<float*>(field_grad(d, field) + (size_t)yk * d.W + xk), vx, vy);
    }
};

struct EmitSink {
    uint32_t* key;
    float4* pay;
    int32_t stride;  // entries per event: R for the splat, B + 1 for the adjoint (one per edge)

    __device__ __forceinline__ void splat(const Win& d, int r, const Bil& s, float tbar, int pol2, int64_t k) const
    {
        const int64_t e = k * stride + r;
        key[e] = (uint32_t)((size_t)(2 * r + (pol2 >> 1)) * plane_size(d) + (size_t)s.iy * d.W + s.ix);
        pay[e] = make_float4(s.ax, s.ay, 1.0f, tbar);
    }
    __device__ __forceinline__ void scatter(const Win& d, int field, int edge, const Bil& s, float hx, float hy,
                                            int64_t k) const
    {
        const int64_t e = k * stride + edge;
        key[e] = (uint32_t)(plane_of(d, field) * plane_size(d) + (size_t)s.iy * d.W + s.ix);
        pay[e] = make_float4(s.ax, s.ay, hx, hy);
    }
    __device__ __forceinline__ void point(const Win& d, int field, int edge, int xk, int yk, float vx, float vy,
                                          int64_t k) const
    {
        const int64_t e = k * stride + edge;
        key[e] = (uint32_t)(plane_of(d, field) * plane_size(d) + (size_t)yk * d.W + xk);
        pay[e] = make_float4(0.0f, 0.0f, vx, vy);
    }
};

// Edge j of an event in bin b is a computed trajectory point: the forward
// chain b+1..B, and with all edges as references also the backward chain 0..b.
__device__ __forceinline__ bool computed_edge(const Win& d, int j, int b)
{
    return j <= d.B && (j > b || d.ref_mode == kRefAll);
}

// Stored warps: the splat writes every computed point of event k (its offset
// from the event's pixel) to d.warp[j][k] (coalesced across a warp); the
// adjoint reads them back instead
// of recomputing the trajectory, and takes the mask from them (a point outside
// the image stays outside in every later point of its chain, so the test over
// all stored points repeats the decision of the trajectory exactly).
template <int MAXB, class TR>
__device__ __forceinline__ void store_traj(const Win& d, const EventAt& e, TR& P, int64_t k)
{
#pragma unroll
    for (int j = 0; j <= MAXB; ++j)
        if (computed_edge(d, j, e.b)) d.warp[(size_t)j * d.n + k] = make_float2(P.x(j), P.y(j));
}

template <int MAXB, bool NC = true, class TR>
__device__ __forceinline__ bool load_traj(const Win& d, const EventAt& e, TR& P, int64_t k)
{
    bool ok = true;
#pragma unroll
    for (int j = 0; j <= MAXB; ++j) {
        if (computed_edge(d, j, e.b)) {
            const float2 q = ld_in<NC>(d.warp + (size_t)j * d.n + k);
            P.x(j) = q.x;
            P.y(j) = q.y;
            ok = ok && inside(e.xk, e.yk, q.x, q.y, d.W, d.H);
            if (j == d.B) {
                P.ex = q.x;
                P.ey = q.y;
            }
        }
    }
    return ok;
}

template <int MAXB, bool NC = true, class Sink, class TR>
__device__ __forceinline__ void splat_points(const Win& d, int64_t k, const Sink& sink, TR& P)
{
    EventAt e;
    if (!load_event<NC>(d, k, e)) return;
    const bool ok = trajectory<MAXB, NC>(d, e, P);
    if (d.warp) store_traj<MAXB>(d, e, P, k);
    if (!ok) return;
    if (d.ref_mode == kRefAll) {
#pragma unroll
        for (int j = 0; j <= MAXB; ++j)
            if (j <= d.B) sink.splat(d, j, bil(e.xk, e.yk, P.x(j), P.y(j)), tbar_of(j, d.B, e.tau), e.pol2, k);
    } else {
        sink.splat(d, 0, bil(e.xk, e.yk, P.ex, P.ey), tbar_of(d.B, d.B, e.tau), e.pol2, k);
    }
}

template <int MAXB, class Sink = RedSink>
__device__ __forceinline__ void splat_event(const Win& d, int64_t k, const Sink& sink = Sink())
{
    Traj<MAXB> P;
    splat_points<MAXB>(d, k, sink, P);
}

// the same with the points in shared memory: smem is the block's
// [MAXB + 1][kEventThreads] float2 array (16-byte aligned)
template <int MAXB, bool NC = true, class Sink = RedSink>
__device__ __forceinline__ void splat_event_smem(const Win& d, int64_t k, float* smem, const Sink& sink = Sink())
{
    SmemTraj<MAXB> P;
    P.ps = reinterpret_cast<float2*>(smem) + threadIdx.x;
    splat_points<MAXB, NC>(d, k, sink, P);
}

// dL/dw_c of one corner from its count and timestamp sum, with the loss
// pass's T = S/(C+eps) and A = 2T/(C+eps): phi = kappa * A * (tbar - T)
__device__ __forceinline__ float phi_of(float C, float S, float eps, float kap, float tbar)
{
    const float rc = recip(C + eps);
    const float T = S * rc;
    return kap * (2.0f * T * rc) * (tbar - T);
}

// phi of the two corners of one row in polarity-plane layout (left at float2
// index gi, right behind it when `two`).  One 16-byte gather of the aligned
// pair holding the left corner, plus an 8-byte one for the right corner when
// the row starts at an odd index.  No branch: every lane issues its gathers
// together, so the row costs one L2 latency (a divergent choice between the two
// forms would serialise them).  The aligned pair never leaves the image: the
// last float2 of the buffer has an odd index.
template <bool NC = true>
__device__ __forceinline__ void phi_row(const float2* img, size_t gi, bool two, float eps, float kap, float tbar,
                                        float& pl, float& pr)
{
    const bool odd = (gi & 1) != 0;
    const float4 g = ld_in<NC>(reinterpret_cast<const float4*>(img + (gi & ~(size_t)1)));
    float2 h = make_float2(0.0f, 0.0f);
    if (two && odd) h = ld_in<NC>(img + gi + 1);
    const float2 l = odd ? make_float2(g.z, g.w) : make_float2(g.x, g.y);
    const float2 r = odd ? h : make_float2(g.z, g.w);
    pl = phi_of(l.x, l.y, eps, kap, tbar);
    pr = two ? phi_of(r.x, r.y, eps, kap, tbar) : 0.0f;
}

// position adjoint a = sum_c grad(w_c) phi_c at reference r, edge j; corners
// outside the image have phi = 0.  SPLIT: the image is in the polarity-plane
// layout (Win::iwe_split == 1), a compile-time choice so that the event kernels
// carry the code of one layout only.
template <bool SPLIT, bool NC = true>
__device__ __forceinline__ float2 ref_adjoint(const Win& d, int r, int j, const Bil& s, float tau, int pol2, float dl)
{
    const size_t HW = plane_size(d);
    const int W = d.W, H = d.H;
    const float kap = dl * ld_in<NC>(d.norm + r);
    const float tb = tbar_of(j, d.B, tau);
    const float eps = d.eps;
    const size_t i00 = (size_t)s.iy * W + s.ix;
    const bool inx = s.ix + 1 <= W - 1, iny = s.iy + 1 <= H - 1;
    float p00, p10 = 0.0f, p01 = 0.0f, p11 = 0.0f;
    if (SPLIT) {
        const float2* img = reinterpret_cast<const float2*>(d.iwe);
        const size_t gi = (size_t)(2 * r + (pol2 >> 1)) * HW + i00;
        phi_row<NC>(img, gi, inx, eps, kap, tb, p00, p10);
        phi_row<NC>(img, iny ? gi + W : gi, inx, eps, kap, tb, p01, p11);  // unconditional: both rows in flight together
        if (!iny) p01 = p11 = 0.0f;
    } else {
        const float2* G = reinterpret_cast<const float2*>(d.iwe + (size_t)r * HW) + (pol2 >> 1);
        auto at = [&](size_t i) {
            const float2 g = ld_in<NC>(G + 2 * i);
            return phi_of(g.x, g.y, eps, kap, tb);
        };
        p00 = at(i00);
        if (inx) p10 = at(i00 + 1);
        if (iny) p01 = at(i00 + W);
        if (inx && iny) p11 = at(i00 + W + 1);
    }
    float2 a;
    a.x = s.by * (p10 - p00) + s.ay * (p11 - p01);
    a.y = s.bx * (p01 - p00) + s.ax * (p11 - p10);
    return a;
}

// One push of the adjoint back across a step x' = x + hs u(x) sampled at x,
// in cell s (hs = +h forward chain, -h backward chain): scatter hs w_c lambda
// into the gradient of field `field` and return lambda + hs J(x)^T lambda.
template <bool NC = true, class Sink>
__device__ __forceinline__ float2 push_back(const Win& d, const Sink& sink, int field, int edge, const Bil& s,
                                            float hs, float2 lam, int64_t k)
{
    const Quad q = quad_at<NC>(d, field, s);
    const float hx = hs * lam.x, hy = hs * lam.y;
    sink.scatter(d, field, edge, s, hx, hy, k);
    const float jxx = s.by * (q.u10.x - q.u00.x) + s.ay * (q.u11.x - q.u01.x);
    const float jxy = s.bx * (q.u01.x - q.u00.x) + s.ax * (q.u11.x - q.u10.x);
    const float jyx = s.by * (q.u10.y - q.u00.y) + s.ay * (q.u11.y - q.u01.y);
    const float jyy = s.bx * (q.u01.y - q.u00.y) + s.ax * (q.u11.y - q.u10.y);
    float2 out;
    out.x = lam.x + hs * (jxx * lam.x + jyx * lam.y);
    out.y = lam.y + hs * (jxy * lam.x + jyy * lam.y);
    return out;
}

// S6: per-event adjoint.  The trajectory is recomputed (or read back when the
// splat stored it); the position adjoint of each reference point comes from
// the (C, S) pairs gathered at its corners (phi_of), and the adjoint is
// carried back along both chains of pushes, scattering dL/dflow.  The points
// live in registers (Traj) or, given a block's [MAXB + 1][kEventThreads] float2
// shared array `smem`, in shared memory (SmemTraj).
template <int MAXB, bool SPLIT, bool NC = true, class Sink, class TR>
__device__ __forceinline__ void adjoint_points(const Win& d, int64_t k, float dl, const Sink& sink, TR& P)
{
    EventAt e;
    if (!load_event<NC>(d, k, e)) return;
    if (!(d.warp ? load_traj<MAXB, NC>(d, e, P, k) : trajectory<MAXB, NC>(d, e, P))) return;
    const int B = d.B, b = e.b;
    const float h = __fdiv_rn(1.0f, (float)B);
    const bool all = d.ref_mode == kRefAll;
    // forward chain: edges B .. b+1
    float2 lam = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = MAXB; j >= 1; --j) {
        if (j <= B && j > b) {
            if (all || j == B) {
                const float2 a =
                    ref_adjoint<SPLIT, NC>(d, all ? j : 0, j, bil(e.xk, e.yk, P.x(j), P.y(j)), e.tau, e.pol2, dl);
                lam.x += a.x;
                lam.y += a.y;
            }
            if (j > b + 1) {
                lam = push_back<NC>(d, sink, j - 1, j, bil(e.xk, e.yk, P.x(j - 1), P.y(j - 1)), h, lam, k);
            } else {
                const float dtf = __fsub_rn(edge_tau(b + 1, B), e.tau);
                sink.point(d, b, j, e.xk, e.yk, dtf * lam.x, dtf * lam.y, k);
            }
        }
    }
    if (!all) return;
    // backward chain: edges 0 .. b
    lam = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j <= MAXB - 1; ++j) {
        if (j <= b) {
            const float2 a = ref_adjoint<SPLIT, NC>(d, j, j, bil(e.xk, e.yk, P.x(j), P.y(j)), e.tau, e.pol2, dl);
            lam.x += a.x;
            lam.y += a.y;
            if (j < b) {
                lam = push_back<NC>(d, sink, j, j, bil(e.xk, e.yk, P.x(j + 1), P.y(j + 1)), -h, lam, k);
            } else {
                const float dtb = __fsub_rn(e.tau, edge_tau(b, B));
                sink.point(d, b, j, e.xk, e.yk, -dtb * lam.x, -dtb * lam.y, k);
            }
        }
    }
}

template <int MAXB, class Sink = RedSink, bool SPLIT = false>
__device__ __forceinline__ void adjoint_event(const Win& d, int64_t k, float dl, const Sink& sink = Sink())
{
    Traj<MAXB> P;
    adjoint_points<MAXB, SPLIT>(d, k, dl, sink, P);
}

// the same with the points in shared memory: smem is the block's
// [MAXB + 1][kEventThreads] float2 array (16-byte aligned)
template <int MAXB, class Sink = RedSink, bool SPLIT = false, bool NC = true>
__device__ __forceinline__ void adjoint_event_smem(const Win& d, int64_t k, float dl, float* smem,
                                                   const Sink& sink = Sink())
{
    SmemTraj<MAXB> P;
    P.ps = reinterpret_cast<float2*>(smem) + threadIdx.x;
    adjoint_points<MAXB, SPLIT, NC>(d, k, dl, sink, P);
}

// warp-level sum (fixed shuffle tree: deterministic)
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// True in exactly one block: the last of `total` tile completions counted on
// `counter`.  Every thread fences its own writes before the block's arrival is
// counted, and the last block fences again before reading the others' writes;
// it then resets the counter for the next use.  The caller's reduction over
// the tiles runs in a fixed order, so the result does not depend on which
// block arrives last.
__device__ __forceinline__ bool last_tile_done(int32_t* counter, int total)
{
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(counter, 1);
        is_last = prev == total - 1;
        if (is_last) atomicExch(counter, 0);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last != 0;
}

// ---------------------------------------------------------------------------
// Per-pixel passes, written once for the single-window and the batched
// kernels.  A pass over one image is split into `ntiles` tiles; tile `tile`
// covers pixels tile*blockDim + threadIdx.x, stepping by ntiles*blockDim.

// S1: rigid motion field (Sec. 3.2, Eq. 2 in its instantaneous form), FP32
// with the operation order of the trajectory contract:
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

__device__ __forceinline__ void flow_tile(const Win& d, int tile, int ntiles)
{
    const int W = d.W;
    const size_t HW = plane_size(d);
    float2* flow = const_cast<float2*>(d.flow);
    for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < HW; i += (size_t)ntiles * blockDim.x) {
        int u, v;
        pixel_uv(i, W, u, v);
        flow[i] = motion_field(u, v, __ldg(d.rho + i), d.ego, d.fx, d.fy, d.cx, d.cy, d.dt);
    }
}

// S1 for the flow quads: writes record (u, v) from the flow at the cell's four
// corners (clamped to the image): the motion field evaluated there for depth
// input, the given field for flow input.  Returns the flow at (u, v).  Every
// corner value is the same FP32 function of its own pixel as in flow_tile, so
// a quad holds exactly the values four gathers would read.
__device__ __forceinline__ float2 build_quad(const Win& d, int u, int v)
{
    const int u1 = min(u + 1, d.W - 1), v1 = min(v + 1, d.H - 1);
    const size_t r0 = (size_t)v * d.W, r1 = (size_t)v1 * d.W;
    float2 f00, f10, f01, f11;
    if (d.rho) {
        f00 = motion_field(u, v, __ldg(d.rho + r0 + u), d.ego, d.fx, d.fy, d.cx, d.cy, d.dt);
        f10 = motion_field(u1, v, __ldg(d.rho + r0 + u1), d.ego, d.fx, d.fy, d.cx, d.cy, d.dt);
        f01 = motion_field(u, v1, __ldg(d.rho + r1 + u), d.ego, d.fx, d.fy, d.cx, d.cy, d.dt);
        f11 = motion_field(u1, v1, __ldg(d.rho + r1 + u1), d.ego, d.fx, d.fy, d.cx, d.cy, d.dt);
    } else {
        f00 = __ldg(d.flow + r0 + u);
        f10 = __ldg(d.flow + r0 + u1);
        f01 = __ldg(d.flow + r1 + u);
        f11 = __ldg(d.flow + r1 + u1);
    }
    st_v8(const_cast<FQ*>(d.fq) + r0 + u, make_float4(f00.x, f00.y, f10.x, f10.y), make_float4(f01.x, f01.y, f11.x, f11.y));
    return f00;
}

// dL/dflow at pixel (x, y) from the quad accumulators (one field): the sum of
// every record corner whose clamped index is this pixel.  Corner 00 of its own
// cell; corner 10 of cell x-1 (and of its own cell on the right border);
// corner 01 of cell y-1 (and of its own cell on the bottom border); corner 11
// of the cells combining both.
__device__ __forceinline__ float2 fold_dq(const Win& d, int x, int y)
{
    const int W = d.W, H = d.H;
    const float4* Q = reinterpret_cast<const float4*>(d.dq);
    auto at = [&](int qx, int qy, int half) { return Q[2 * ((size_t)qy * W + qx) + half]; };
    const float4 own = at(x, y, 0);
    float gx = own.x, gy = own.y;
    if (x >= 1) {
        const float4 t = at(x - 1, y, 0);
        gx += t.z;
        gy += t.w;
    }
    if (x == W - 1) {
        gx += own.z;
        gy += own.w;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (k == 0 ? y < 1 : y != H - 1) continue;
        const int qy = k == 0 ? y - 1 : y;
        const float4 t = at(x, qy, 1);
        gx += t.x;
        gy += t.y;
        if (x >= 1) {
            const float4 l = at(x - 1, qy, 1);
            gx += l.z;
            gy += l.w;
        }
        if (x == W - 1) {
            gx += t.z;
            gy += t.w;
        }
    }
    return make_float2(gx, gy);
}

// dL/dflow of one tile's pixels from the quad accumulators (flow-input windows)
__device__ __forceinline__ void fold_tile(const Win& d, int tile, int ntiles)
{
    const int W = d.W;
    const size_t HW = plane_size(d);
    for (size_t i = (size_t)tile * blockDim.x + threadIdx.x; i < HW; i += (size_t)ntiles * blockDim.x) {
        int u, v;
        pixel_uv(i, W, u, v);
        d.dflow[i] = fold_dq(d, u, v);
    }
}

// S5 pass 1 over one tile of reference r: T = S/(C+eps) for both polarities;
// the sum of T^2 and the non-empty count go to out[0].  Read-only: the adjoint
// recomputes T and A = 2T/(C+eps) from (C, S) at the corners it gathers, with
// the same operations (phi_of).  Ends with __syncthreads (the caller may loop).
__device__ __forceinline__ void loss_tile(const Win& d, int r, int tile, int ntiles, float2* out)
{
    const size_t HW = plane_size(d);
    const float eps = d.eps;
    float s = 0.0f;
    int cnt = 0;
    const size_t stride = (size_t)ntiles * blockDim.x;
    // (C+, S+, C-, S-) of pixel i in either layout
    const float4* plane = d.iwe + (size_t)r * HW;
    const float2* pos = reinterpret_cast<const float2*>(d.iwe) + (size_t)2 * r * HW;
    const float2* neg = pos + HW;
    const bool split = d.iwe_split != 0;
    auto ld = [&](size_t i) {
        if (!split) return plane[i];
        const float2 a = pos[i], b = neg[i];
        return make_float4(a.x, a.y, b.x, b.y);
    };
    auto one = [&](float4 q) {
        const float tp = q.y * recip(q.x + eps), tm = q.w * recip(q.z + eps);
        s = fmaf(tp, tp, s);
        s = fmaf(tm, tm, s);
        cnt += (q.x > 0.0f || q.z > 0.0f) ? 1 : 0;
    };
    size_t i = (size_t)tile * blockDim.x + threadIdx.x;
    // four independent loads in flight per thread (the pass is latency-bound otherwise)
    for (; i + 3 * stride < HW; i += 4 * stride) {
        const float4 q0 = ld(i), q1 = ld(i + stride), q2 = ld(i + 2 * stride), q3 = ld(i + 3 * stride);
        one(q0);
        one(q1);
        one(q2);
        one(q3);
    }
    for (; i < HW; i += stride) one(ld(i));
    __shared__ float ss[32];
    __shared__ int sc[32];
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
        *out = make_float2(a, (float)c);
    }
    __syncthreads();
}

// S5 pass 1 over one pixel tile of a window and every reference, for the
// polarity-plane layout (iwe_split == 1): the sum of T^2 and the non-empty
// count of reference r over the tile go to loss_part[r][tile].  Same per-pixel
// operations as loss_tile.  Two references per round and four pixel pairs
// per polarity (PAIRS: 16-byte loads, for planes 16-byte aligned: HW even):
// sixteen loads in flight per thread.  Padding slots read (0, 0), which adds
// exactly nothing.  Ends with __syncthreads (the caller may loop).
template <bool PAIRS>
__device__ __forceinline__ void loss_tile_planes(const Win& d, int tile, int ntiles)
{
    constexpr int K = 4, RK = 2;
    const uint32_t HW = (uint32_t)plane_size(d);
    const float eps = d.eps;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ float ss[kMaxRefs][32];
    __shared__ int sc[kMaxRefs][32];
    const uint32_t stride = (uint32_t)ntiles * blockDim.x, first = (uint32_t)tile * blockDim.x + threadIdx.x;
    const float2* planes = reinterpret_cast<const float2*>(d.iwe);
    const uint32_t n = PAIRS ? HW >> 1 : HW;  // loads per plane
    for (int r0 = 0; r0 < d.R; r0 += RK) {
        float s[RK];
        int cnt[RK];
#pragma unroll
        for (int q = 0; q < RK; ++q) {
            s[q] = 0.0f;
            cnt[q] = 0;
        }
        auto one = [&](int q, float cp, float sp, float cm, float sm) {
            const float tp = sp * recip(cp + eps), tm = sm * recip(cm + eps);
            s[q] = fmaf(tp, tp, s[q]);
            s[q] = fmaf(tm, tm, s[q]);
            cnt[q] += (cp > 0.0f || cm > 0.0f) ? 1 : 0;
        };
        for (uint32_t j0 = first; j0 < n; j0 += K * stride) {
            float4 a[RK][K], b[RK][K];
#pragma unroll
            for (int q = 0; q < RK; ++q) {
                const float2* pos = planes + (size_t)2 * (r0 + q) * HW;
                const float2* neg = pos + HW;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const uint32_t j = j0 + k * stride;
                    const bool in = j < n && r0 + q < d.R;
                    if (PAIRS) {
                        a[q][k] = in ? reinterpret_cast<const float4*>(pos)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                        b[q][k] = in ? reinterpret_cast<const float4*>(neg)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                    } else {
                        const float2 x = in ? pos[j] : make_float2(0.f, 0.f), y = in ? neg[j] : make_float2(0.f, 0.f);
                        a[q][k] = make_float4(x.x, x.y, 0.f, 0.f);
                        b[q][k] = make_float4(y.x, y.y, 0.f, 0.f);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < RK; ++q)
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    one(q, a[q][k].x, a[q][k].y, b[q][k].x, b[q][k].y);
                    if (PAIRS) one(q, a[q][k].z, a[q][k].w, b[q][k].z, b[q][k].w);
                }
        }
#pragma unroll
        for (int q = 0; q < RK; ++q) {
            const float sq = warp_sum(s[q]);
            const int cq = warp_sum(cnt[q]);
            if (l == 0 && r0 + q < d.R) {
                ss[r0 + q][w] = sq;
                sc[r0 + q][w] = cq;
            }
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < d.R) {
        const int r = threadIdx.x;
        float a = 0.0f;
        int c = 0;
        for (int i = 0; i < nw; ++i) {
            a += ss[r][i];
            c += sc[r][i];
        }
        d.loss_part[(size_t)r * ntiles + tile] = make_float2(a, (float)c);
    }
    __syncthreads();
}

// S5 pass 2 for one window (one block): fixed-order reduction of the tiles,
// L_r, N_nz(r), 1/(R(N_nz + eps)) and the loss.
__device__ __forceinline__ void loss_final_window(const Win& d)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ double lr[64];
    for (int r = w; r < d.R; r += nw) {
        const float2* part = d.loss_part + (size_t)r * d.loss_tiles;
        double s = 0.0, c = 0.0;
        // lane l adds tiles l, l+32, ... in that order, with eight loads in flight
        // (this single block is the pass's serial tail)
        for (int i0 = l; i0 < d.loss_tiles; i0 += 32 * 8) {
            float2 q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) q[u] = i0 + 32 * u < d.loss_tiles ? part[i0 + 32 * u] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s += (double)q[u].x;
                c += (double)q[u].y;
            }
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

// S7 over one tile: dL/d(rho) per pixel and the tile's six dL/d(ego) sums
// (to d.dego_part[tile][6]).  Ends with __syncthreads.
__device__ __forceinline__ void depth_ego_tile(const Win& d, int tile, int ntiles)
{
    const int W = d.W;
    const size_t HW = plane_size(d);
    const float vx = __ldg(d.ego + 0), vy = __ldg(d.ego + 1), vz = __ldg(d.ego + 2);
    const float ifx = 1.0f / d.fx, ify = 1.0f / d.fy;
    const float sx = d.dt * d.fx, sy = d.dt * d.fy;
    float g[6] = {0, 0, 0, 0, 0, 0};
    // dL/dflow at pixel i: folded from the quad accumulators (and stored) when
    // the pushes went there, else read
    auto dfl = [&](size_t i) -> float2 {
        if (!d.dq) return d.dflow[i];
        int u, v;
        pixel_uv(i, W, u, v);
        const float2 f = fold_dq(d, u, v);
        if (d.dflow) d.dflow[i] = f;
        return f;
    };
    auto one = [&](size_t i, float r, float2 df) {
        int u, v;
        pixel_uv(i, W, u, v);
        const float xn = ((float)u - d.cx) * ifx, yn = ((float)v - d.cy) * ify;
        const float Gx = sx * df.x, Gy = sy * df.y;
        if (d.drho) d.drho[i] = Gx * (xn * vz - vx) + Gy * (yn * vz - vy);
        g[0] -= r * Gx;
        g[1] -= r * Gy;
        g[2] += r * (xn * Gx + yn * Gy);
        g[3] += xn * yn * Gx + (1.0f + yn * yn) * Gy;
        g[4] -= (1.0f + xn * xn) * Gx + xn * yn * Gy;
        g[5] += yn * Gx - xn * Gy;
    };
    // four pixels' loads in flight, added in the order i, i + stride, ...
    constexpr int K = 4;
    const size_t stride = (size_t)ntiles * blockDim.x;
    for (size_t i0 = (size_t)tile * blockDim.x + threadIdx.x; i0 < HW; i0 += K * stride) {
        float r[K];
        float2 f[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t i = i0 + k * stride;
            if (i < HW) {
                r[k] = __ldg(d.rho + i);
                f[k] = dfl(i);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i0 + k * stride < HW) one(i0 + k * stride, r[k], f[k]);
    }
    __shared__ float sg[32][6];
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
        d.dego_part[(size_t)tile * 6 + threadIdx.x] = a;
    }
    __syncthreads();
}

// S7 final for one window: warps 0..5 reduce the ntiles tiles of one component each.
__device__ __forceinline__ void depth_ego_final_window(const Win& d, int ntiles)
{
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (c >= 6) return;
    double s = 0.0;
    // lane l adds tiles l, l+32, ... in that order, with eight loads in flight
    for (int i0 = l; i0 < ntiles; i0 += 32 * 8) {
        float q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) q[u] = i0 + 32 * u < ntiles ? d.dego_part[(size_t)(i0 + 32 * u) * 6 + c] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) s += (double)q[u];
    }
    s = warp_sum(s);
    if (l == 0 && d.dego) d.dego[c] = (float)s;
}

}  // namespace cmk
