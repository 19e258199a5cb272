// cm_launch.h -- host-side launchers shared between the translation units of
// libcm.so (internal; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "../../include/cm.h"
#include "cm_device.cuh"

namespace cmk {

cudaError_t launch_flow(const Win& d, cudaStream_t st);
cudaError_t launch_splat(const Win& d, int sm_count, cudaStream_t st);
cudaError_t launch_adjoint(const Win& d, int sm_count, cudaStream_t st);
cudaError_t launch_loss(const Win& d, cudaStream_t st);
cudaError_t launch_depth_ego(const Win& d, cudaStream_t st);
cudaError_t launch_depth_ego_planes(const Win& d, cudaStream_t st);  // fused final reduction (d.sync[1] zero)
// the polarity-plane layout of one window (iwe_split, flow quads, quad accumulators)
cudaError_t launch_prep(const Win& d, int sm_count, cudaStream_t st);
cudaError_t launch_loss_planes(const Win& d, cudaStream_t st);  // d.loss_tiles blocks over every reference,
                                                                // fused final reduction (d.sync[0] zero)
cudaError_t launch_fold(const Win& d, cudaStream_t st);         // dL/dflow from the quad accumulators
// events grouped by band of rows into d.rx, d.ry, d.rt, d.rp (d.tile_cnt: the
// [bands][super-chunks] table; d.sync[2]: its completion counter, zero)
cudaError_t launch_bands(const Win& d, int sm_count, cudaStream_t st);

// number of SMs of the current device (cached per device)
int sm_count_current();

// argument checks of the C ABI (cm_api.cu): CM_OK or CM_EINVAL
int check_camera(const cm_camera* cam);  // sizes 2..32767, finite fx, fy > 0, finite cx, cy
int check_cfg(const cm_loss_cfg* cfg);   // bins, reference mode, splat, store_warps, finite eps
int check_events(const cm_events* ev);   // n >= 0, arrays given when n > 0, finite t0 < t1 with a finite span

// Tracing scope around one kernel launch: counts the launch and, when
// profiling is on and the stream is not being captured, brackets it with CUDA
// events on the launch stream (cm_profile.cu).
class KernelScope {
public:
    KernelScope(const char* name, cudaStream_t s, int launches = 1);
    ~KernelScope();
    KernelScope(const KernelScope&) = delete;
    KernelScope& operator=(const KernelScope&) = delete;

private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t a_;
};

// add kernel launches made outside KernelScope (graph replays)
void count_launches(long long n);

// for CUDA-graph replays: whether per-kernel timing is on, an event from the
// profiler's pool, and a recorded (start, stop) pair to be collected
bool profiling_on();
cudaEvent_t profile_take_event();
void profile_push(const char* name, cudaEvent_t a, cudaEvent_t b);

}  // namespace cmk
