// cm_static.cu -- cm_loss_grad_static: the loss and flow gradient of one
// window with every intermediate buffer in a fixed, file-scope device array,
// so that the call allocates nothing.
//
// Who needs this.  Some callers cannot allocate device memory at the point
// where they evaluate the loss: a real-time control or on-board learning loop
// (such as the drone loop this loss was designed for) that must not pay an
// allocator's latency, or risk an out-of-memory failure, in the middle of its
// cycle; a plug-in hosted by a framework that owns all device memory through
// its own pool and forbids raw cudaMalloc; code whose memory was budgeted once,
// up front.  The regular entry points need a caller-provided workspace;
// this one needs none.
//
// The scratch array below is CM_STATIC_SCRATCH_BYTES (32 MiB).  The first call
// on each device reserves it there (see scratch_address) and the device keeps it
// until the process exits.  All calls share the one array and it keeps whatever the last call left
// in it; each call clears the part that must start at zero (the images of warped
// events) before using it.  Two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array and give wrong results:
// order them on one stream or synchronise between them.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/cm.h"
#include "cm_launch.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[CM_STATIC_SCRATCH_BYTES];

// device address of g_static_scratch, looked up once per device (host code may
// not use the symbol itself: on the host it names a stand-in, not device memory)
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// The first lookup on a device is also where the array is reserved: with
// CUDA's lazy module loading this module (it holds no kernels, only the array)
// is loaded on that device when its symbol is first asked for, so a device
// without 32 MiB free fails here, with CM_ENOMEM.
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CM_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e == cudaErrorMemoryAllocation) {
            (void)cudaGetLastError();
            return CM_ENOMEM;
        }
        if (e != cudaSuccess || !p) return CM_ECUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return CM_OK;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// the checks of the workspace entry points, then what this entry point does
// not support (stored warps, the sort path)
bool valid_args(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t nfb, const cm_loss_cfg* cfg,
                const float* dloss, const float* loss_out, const float* dflow_out)
{
    if (cmk::check_camera(cam) != CM_OK || cmk::check_cfg(cfg) != CM_OK || cmk::check_events(ev) != CM_OK)
        return false;
    if (!flow || !dloss || !loss_out || !dflow_out) return false;
    if (cfg->store_warps != 0) return false;
    if (cfg->splat != CM_SPLAT_AUTO && cfg->splat != CM_SPLAT_ATOMIC) return false;
    if (nfb != 1 && nfb != cfg->nbins) return false;
    return true;
}

}  // namespace

extern "C" int cm_loss_grad_static(const cm_camera* cam, const cm_events* ev, const float* flow,
                                   int32_t n_flow_bins, const cm_loss_cfg* cfg, const float* dloss,
                                   float* loss_out, float* dflow_out, void* stream)
{
    if (!valid_args(cam, ev, flow, n_flow_bins, cfg, dloss, loss_out, dflow_out)) return CM_EINVAL;
    const size_t HW = (size_t)cam->width * cam->height;
    const int R = cfg->ref_mode == CM_REF_END ? 1 : cfg->nbins + 1;
    size_t tiles = (HW + 2047) / 2048;
    tiles = tiles < 1 ? 1 : (tiles > 256 ? 256 : tiles);
    // scratch layout: IWE | loss partials | 1/(R(N+eps)) | L_r | N_nz
    const size_t o_iwe = 0;
    const size_t o_part = up256(o_iwe + (size_t)R * HW * sizeof(float4));
    const size_t o_norm = up256(o_part + (size_t)R * tiles * sizeof(float2));
    const size_t o_lr = up256(o_norm + (size_t)R * sizeof(float));
    const size_t o_nnz = up256(o_lr + (size_t)R * sizeof(float));
    const size_t need = up256(o_nnz + (size_t)R * sizeof(int32_t));
    if (need > (size_t)CM_STATIC_SCRATCH_BYTES) return CM_ENOMEM;  // the window does not fit the fixed scratch

    void* base = nullptr;
    int st = scratch_address(&base);
    if (st != CM_OK) return st;
    char* s = static_cast<char*>(base);

    cmk::Win d;
    std::memset(&d, 0, sizeof(d));
    d.x = ev->x;
    d.y = ev->y;
    d.t = ev->t;
    d.p = ev->p;
    d.n = ev->n;
    d.t0 = ev->t0;
    d.span = ev->t1 - ev->t0;
    d.W = cam->width;
    d.H = cam->height;
    d.B = cfg->nbins;
    d.R = R;
    d.ref_mode = cfg->ref_mode;
    d.nfb = n_flow_bins;
    d.eps = cfg->eps > 0.0f ? cfg->eps : 1e-9f;
    d.flow = reinterpret_cast<const float2*>(flow);
    d.iwe = reinterpret_cast<float4*>(s + o_iwe);
    d.loss_part = reinterpret_cast<float2*>(s + o_part);
    d.loss_tiles = (int32_t)tiles;
    d.norm = reinterpret_cast<float*>(s + o_norm);
    d.loss_r = reinterpret_cast<float*>(s + o_lr);
    d.nnz_r = reinterpret_cast<int32_t*>(s + o_nnz);
    d.loss = loss_out;
    d.dloss = dloss;
    d.dflow = reinterpret_cast<float2*>(dflow_out);

    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    const int sms = cmk::sm_count_current();
    if (cudaMemsetAsync(d.iwe, 0, (size_t)R * HW * sizeof(float4), cs) != cudaSuccess) return CM_ECUDA;
    if (cmk::launch_splat(d, sms, cs) != cudaSuccess) return CM_ECUDA;
    if (cmk::launch_loss(d, cs) != cudaSuccess) return CM_ECUDA;
    if (cudaMemsetAsync(d.dflow, 0, (size_t)n_flow_bins * HW * sizeof(float2), cs) != cudaSuccess) return CM_ECUDA;
    if (cmk::launch_adjoint(d, sms, cs) != cudaSuccess) return CM_ECUDA;
    return CM_OK;
}
