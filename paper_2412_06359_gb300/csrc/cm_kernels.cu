// cm_kernels.cu -- the kernels of one window: flow from depth (S1), warp +
// splat (S2-S4), loss reduction (S5), adjoint (S6), depth / ego gradient (S7),
// and their host-side launchers.
#include "cm_device.cuh"
#include "cm_launch.h"

namespace cmk {

// ---------------------------------------------------------------------------
// S1 (grid-stride over the pixels of one window)
__global__ void __launch_bounds__(256) k_flow(Win d) { flow_tile(d, blockIdx.x, gridDim.x); }

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
// S5: loss.  Pass 1 (grid = loss_tiles x R), pass 2 (one block).
__global__ void __launch_bounds__(256) k_loss_partial(Win d)
{
    loss_tile(d, blockIdx.y, blockIdx.x, gridDim.x, d.loss_part + (size_t)blockIdx.y * d.loss_tiles + blockIdx.x);
}

__global__ void __launch_bounds__(1024) k_loss_final(Win d) { loss_final_window(d); }

// S7: dL/d(rho) per pixel and the six dL/d(ego) sums (fixed-order reduction)
__global__ void __launch_bounds__(256) k_depth_ego(Win d) { depth_ego_tile(d, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(192) k_depth_ego_final(Win d) { depth_ego_final_window(d, d.pix_tiles); }

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
    k_flow<<<grid, 256, 0, st>>>(d);
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
