// cm_launch.h -- host-side launchers shared between the translation units of
// libcm.so (internal; not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "cm_device.cuh"

namespace cmk {

cudaError_t launch_flow(const Win& d, cudaStream_t st);
cudaError_t launch_splat(const Win& d, int sm_count, cudaStream_t st);
cudaError_t launch_adjoint(const Win& d, int sm_count, cudaStream_t st);
cudaError_t launch_loss(const Win& d, cudaStream_t st);
cudaError_t launch_depth_ego(const Win& d, cudaStream_t st);

// number of SMs of the current device (cached per device)
int sm_count_current();

}  // namespace cmk
