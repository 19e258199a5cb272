// cm_kernels.cu -- the kernels of one window: flow from depth (S1), warp +
// splat (S2-S4), loss reduction (S5), adjoint (S6), depth / ego gradient (S7),
// and their host-side launchers.
#include "cm_bands.cuh"
#include "cm_device.cuh"
#include "cm_launch.h"

namespace cmk {

// ---------------------------------------------------------------------------
// S1 (grid-stride over the pixels of one window)
__global__ void __launch_bounds__(256) k_flow(Win d) { flow_tile(d, blockIdx.x, gridDim.x); }

// ---------------------------------------------------------------------------
// the event kernels keep their trajectory points in shared memory up to 10
// bins: 64 registers and four blocks per SM.  With more bins they keep them
// in registers: two blocks per SM either way, and at 20 bins the register
// form measured faster (a one-window plan at 1280x720: 2.61 against 2.74 ms).
template <int MAXB>
constexpr bool kPointsInSmem = MAXB <= 10;
template <int MAXB>
constexpr int kEventBlocksPerSm = MAXB <= 10 ? 4 : 2;

// S2-S4: one thread per event (grid-stride)
template <int MAXB>
__global__ void __launch_bounds__(kEventThreads, kEventBlocksPerSm<MAXB>) k_splat(Win d)
{
    __shared__ __align__(16) float pts[kPointsInSmem<MAXB> ? 2 * (MAXB + 1) * kEventThreads : 1];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x) {
        if (kPointsInSmem<MAXB>) splat_event_smem<MAXB>(d, k, pts);
        else splat_event<MAXB>(d, k);
    }
}

// S6: one thread per event (grid-stride).  SPLIT: the images are polarity
// planes (Win::iwe_split == 1)
template <int MAXB, bool SPLIT>
__global__ void __launch_bounds__(kEventThreads, kEventBlocksPerSm<MAXB>) k_adjoint(Win d)
{
    __shared__ __align__(16) float pts[kPointsInSmem<MAXB> ? 2 * (MAXB + 1) * kEventThreads : 1];
    const float dl = __ldg(d.dloss);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x) {
        if (kPointsInSmem<MAXB>) adjoint_event_smem<MAXB, RedSink, SPLIT>(d, k, dl, pts);
        else adjoint_event<MAXB, RedSink, SPLIT>(d, k, dl);
    }
}

// ---------------------------------------------------------------------------
// The plane layout of one window (the batched plan's): zero the polarity
// planes and the quad accumulators of dL/dflow, build the flow quads (the
// motion field for depth input).  Grid-stride over 32-byte chunks and pixels.
__global__ void __launch_bounds__(256) k_prep(Win d)
{
    const size_t HW = plane_size(d);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t nf4 = (size_t)d.R * HW, n32 = nf4 / 2;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < n32; c += stride) st_v8(d.iwe + 2 * c, z4, z4);
    if ((nf4 & 1) && blockIdx.x == 0 && threadIdx.x == 0) d.iwe[nf4 - 1] = z4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += stride) {
        st_v8(d.dq + i, z4, z4);
        int u, v;
        pixel_uv(i, d.W, u, v);
        build_quad(d, u, v);
    }
}

// S5 pass 1 over the polarity planes: a tile is 2048 pixels of every reference
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_loss_planes(Win d)
{
    loss_tile_planes<PAIRS>(d, blockIdx.x, gridDim.x);
    // the block completing the last tile reduces the tiles (fixed order)
    if (last_tile_done(d.sync + 0, gridDim.x)) loss_final_window(d);
}

// dL/dflow folded from the quad accumulators (flow input)
__global__ void __launch_bounds__(256) k_fold(Win d) { fold_tile(d, blockIdx.x, gridDim.x); }

// Band grouping of one window's events (cm_bands.cuh): pass 1 counts every
// super-chunk's events per band (the block finishing the last super-chunk
// turns the table into stable offsets), pass 2 places them.
__global__ void __launch_bounds__(kEventThreads) k_band_count(Win d)
{
    __shared__ int hist[kMaxBands];
    const int nsc = super_chunks(d);
    for (int sc = blockIdx.x; sc < nsc; sc += gridDim.x) {
        const long long e0 = (long long)sc * kSuperChunk;
        const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
        band_count(d, sc, e0, e1, hist);
    }
}

__global__ void __launch_bounds__(kEventThreads) k_band_scatter(Win d)
{
    const int nsc = super_chunks(d);
    for (int sc = blockIdx.x; sc < nsc; sc += gridDim.x) {
        const long long e0 = (long long)sc * kSuperChunk;
        const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
        band_scatter(d, sc, e0, e1);
    }
}

// ---------------------------------------------------------------------------
// S5: loss.  Pass 1 (grid = loss_tiles x R), pass 2 (one block).
__global__ void __launch_bounds__(256) k_loss_partial(Win d)
{
    loss_tile(d, blockIdx.y, blockIdx.x, gridDim.x, d.loss_part + (size_t)blockIdx.y * d.loss_tiles + blockIdx.x);
}

__global__ void __launch_bounds__(1024) k_loss_final(Win d) { loss_final_window(d); }

// S7: dL/d(rho) per pixel and the six dL/d(ego) sums (fixed-order reduction)
__global__ void __launch_bounds__(256) k_depth_ego(Win d) { depth_ego_tile(d, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(192) k_depth_ego_final(Win d) { depth_ego_final_window(d, d.pix_tiles); }

// the same for the plane layout, the six sums reduced by the block completing
// the last tile
__global__ void __launch_bounds__(256) k_depth_ego_planes(Win d)
{
    depth_ego_tile(d, blockIdx.x, gridDim.x);
    if (last_tile_done(d.sync + 1, gridDim.x)) {
        __syncthreads();
        depth_ego_final_window(d, gridDim.x);
    }
}

// ---------------------------------------------------------------------------
// launchers

// The event kernels' grids.  The adjoint runs the blocks that fit on the SMs
// at once (their launch bounds), so that its grid-stride loop keeps the
// events in flight contiguous: with events grouped by band they then gather
// from one strip of the images (a larger grid runs in waves, each resident
// block striding over the whole window; 1.64 against 1.42 ms at 1280x720 with
// 2M events).  The splat, whose reductions need no reply, measured faster
// with eight blocks per SM in waves (0.96 against 1.06 ms there).
static int event_grid(int64_t n, int sm_count, int blocks_per_sm)
{
    const int64_t blocks = (n + kEventThreads - 1) / kEventThreads;
    const int64_t cap = (int64_t)sm_count * blocks_per_sm;
    return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

cudaError_t launch_flow(const Win& d, cudaStream_t st)
{
    const size_t HW = (size_t)d.W * d.H;
    const int grid = (int)((HW + 255) / 256 < 4096 ? (HW + 255) / 256 : 4096);
    KernelScope ks("k_flow", st);
    k_flow<<<grid, 256, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_splat(const Win& d, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaSuccess;
    KernelScope ks("k_splat", st);
    const int g = event_grid(d.n, sm_count, 8);
    if (d.B <= 1) k_splat<1><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 10) k_splat<10><<<g, kEventThreads, 0, st>>>(d);
    else if (d.B <= 20) k_splat<20><<<g, kEventThreads, 0, st>>>(d);
    else k_splat<32><<<g, kEventThreads, 0, st>>>(d);
    return cudaGetLastError();
}

template <bool SPLIT>
static void adjoint_for(const Win& d, int sm, cudaStream_t st)
{
    if (d.B <= 1) k_adjoint<1, SPLIT><<<event_grid(d.n, sm, kEventBlocksPerSm<1>), kEventThreads, 0, st>>>(d);
    else if (d.B <= 10) k_adjoint<10, SPLIT><<<event_grid(d.n, sm, kEventBlocksPerSm<10>), kEventThreads, 0, st>>>(d);
    else if (d.B <= 20) k_adjoint<20, SPLIT><<<event_grid(d.n, sm, kEventBlocksPerSm<20>), kEventThreads, 0, st>>>(d);
    else k_adjoint<32, SPLIT><<<event_grid(d.n, sm, kEventBlocksPerSm<32>), kEventThreads, 0, st>>>(d);
}

cudaError_t launch_adjoint(const Win& d, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaSuccess;
    KernelScope ks("k_adjoint", st);
    if (d.iwe_split) adjoint_for<true>(d, sm_count, st);
    else adjoint_for<false>(d, sm_count, st);
    return cudaGetLastError();
}

static int pixel_grid(size_t n, int cap)
{
    const size_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > (size_t)cap ? cap : g));
}

cudaError_t launch_prep(const Win& d, int sm_count, cudaStream_t st)
{
    KernelScope ks("k_prep", st);
    k_prep<<<pixel_grid((size_t)d.R * d.W * d.H / 2, sm_count * 8), 256, 0, st>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_loss_planes(const Win& d, cudaStream_t st)
{
    {
        KernelScope ks("k_loss_planes", st);
        if (((size_t)d.W * d.H) & 1) k_loss_planes<false><<<d.loss_tiles, 256, 0, st>>>(d);
        else k_loss_planes<true><<<d.loss_tiles, 256, 0, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_bands(const Win& d, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaSuccess;
    const int nsc = super_chunks(d);
    const int g = nsc < sm_count * 4 ? nsc : sm_count * 4;
    {
        KernelScope ks("k_band_count", st);
        k_band_count<<<g, kEventThreads, 0, st>>>(d);
    }
    {
        KernelScope ks("k_band_scatter", st);
        k_band_scatter<<<g, kEventThreads, 0, st>>>(d);
    }
    return cudaGetLastError();
}

cudaError_t launch_fold(const Win& d, cudaStream_t st)
{
    KernelScope ks("k_fold", st);
    k_fold<<<d.pix_tiles, 256, 0, st>>>(d);
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

cudaError_t launch_depth_ego_planes(const Win& d, cudaStream_t st)
{
    KernelScope ks("k_depth_ego_planes", st);
    k_depth_ego_planes<<<d.pix_tiles, 256, 0, st>>>(d);
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
