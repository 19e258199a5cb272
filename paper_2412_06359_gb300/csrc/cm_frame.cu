// cm_frame.cu -- the network's input frame: the events of a window counted per
// pixel and polarity ((2, H, W), supp. Table 4), i.e. the splat of S4 with zero
// flow at the event's own pixel, counts only.  Counts are integers below 2^24,
// so the unordered float reductions give the same bits on every run.
#include <cstdint>

#include "../../include/cm.h"
#include "cm_launch.h"

namespace cmk {

namespace {

__global__ void __launch_bounds__(kEventThreads) k_event_frame(const int16_t* __restrict__ x,
                                                                const int16_t* __restrict__ y,
                                                                const int8_t* __restrict__ p, int64_t n, int W, int H,
                                                                float* __restrict__ frame)
{
    const size_t HW = (size_t)W * H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int xk = __ldg(x + k), yk = __ldg(y + k);
        if ((unsigned)xk >= (unsigned)W || (unsigned)yk >= (unsigned)H) continue;
        float* c = frame + (__ldg(p + k) > 0 ? 0 : HW) + (size_t)yk * W + xk;
        asm volatile("red.global.add.f32 [%0], %1;" ::"l"(c), "f"(1.0f));
    }
}

}  // namespace

}  // namespace cmk

extern "C" {

int cm_event_frame(const cm_camera* cam, const cm_events* ev, float* frame_out, void* stream)
{
    if (!cam || !ev || !frame_out || ev->n < 0 || (ev->n > 0 && (!ev->x || !ev->y || !ev->p))) return CM_EINVAL;
    if (cam->width < 2 || cam->height < 2 || cam->width > 32767 || cam->height > 32767) return CM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)2 * cam->width * cam->height * sizeof(float);
    if (cudaMemsetAsync(frame_out, 0, bytes, s) != cudaSuccess) return CM_ECUDA;
    if (ev->n == 0) return CM_OK;
    const int64_t blocks = (ev->n + cmk::kEventThreads - 1) / cmk::kEventThreads;
    const int cap = cmk::sm_count_current() * 16;
    cmk::KernelScope ks("k_event_frame", s);
    cmk::k_event_frame<<<(int)(blocks < cap ? blocks : cap), cmk::kEventThreads, 0, s>>>(
        ev->x, ev->y, ev->p, ev->n, cam->width, cam->height, frame_out);
    return cudaGetLastError() == cudaSuccess ? CM_OK : CM_ECUDA;
}

}  // extern "C"
