// cm_l2probe.cu -- measured ceiling of the request-bound event kernels.
//
// The splat and the adjoint issue random vector reductions and random loads
// into images that live in L2; their rate of requests, not their bytes, bounds
// them.  This probe measures the two rates on the GPU it runs on (random 8-byte
// reductions, random 8-byte loads over a caller buffer), so that a roofline of
// those kernels can be stated against a measured peak, the way the copy
// bandwidth is the peak of the streaming passes.
#include <cstdint>

#include "../../include/cm.h"
#include "cm_launch.h"

namespace cmk {

namespace {

// spreads consecutive (thread, step) pairs over the slots (two xor-shift /
// odd-multiply rounds)
__device__ __forceinline__ uint32_t scatter_hash(uint32_t x)
{
    x ^= x >> 15;
    x *= 0x2c1b3c6du;
    x ^= x >> 12;
    x *= 0x297a2d39u;
    x ^= x >> 15;
    return x;
}

__global__ void __launch_bounds__(256) k_probe_red(float2* buf, uint32_t nslots, int iters)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        const uint32_t s = scatter_hash(t * 1031u + (uint32_t)i) % nslots;
        red_add_v2(&buf[s].x, 1.0f, 0.5f);
    }
}

__global__ void __launch_bounds__(256) k_probe_load(const float2* buf, uint32_t nslots, int iters, float* flag)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    for (int i = 0; i < iters; ++i) {
        const uint32_t s = scatter_hash(t * 1031u + (uint32_t)i) % nslots;
        const float2 v = __ldg(buf + s);
        acc += v.x + v.y;
    }
    if (acc < 0.0f) *flag = acc;  // never true (the buffer holds non-negative sums); keeps the loads
}

}  // namespace

}  // namespace cmk

extern "C" {

int cm_measure_l2_rates(void* buf, size_t bytes, void* stream, double* red_per_s, double* load_per_s)
{
    if (!buf || bytes < ((size_t)16 << 20) || !red_per_s || !load_per_s) return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(buf) % 256) return CM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t slots = (bytes - 256) / sizeof(float2);
    const uint32_t nslots = (uint32_t)(slots > 0x7fffffffu ? 0x7fffffffu : slots);
    float2* img = static_cast<float2*>(buf);
    float* flag = reinterpret_cast<float*>(static_cast<char*>(buf) + bytes - 256);
    const int blocks = cmk::sm_count_current() * 8, threads = 256, iters = 64;
    const double ops = (double)blocks * threads * iters;
    if (cudaMemsetAsync(buf, 0, bytes, s) != cudaSuccess) return CM_ECUDA;
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return CM_ECUDA;
    if (cudaEventCreate(&z) != cudaSuccess) {
        cudaEventDestroy(a);
        return CM_ECUDA;
    }
    double best[2] = {0.0, 0.0};
    int st = CM_OK;
    for (int which = 0; which < 2 && st == CM_OK; ++which) {
        for (int rep = 0; rep < 4 && st == CM_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(a, s);
            if (which == 0) cmk::k_probe_red<<<blocks, threads, 0, s>>>(img, nslots, iters);
            else cmk::k_probe_load<<<blocks, threads, 0, s>>>(img, nslots, iters, flag);
            cudaEventRecord(z, s);
            float ms = 0.0f;
            if (cudaEventSynchronize(z) != cudaSuccess || cudaEventElapsedTime(&ms, a, z) != cudaSuccess) {
                st = CM_ECUDA;
                break;
            }
            const double rate = ops / (ms * 1e-3);
            if (rep > 0 && rate > best[which]) best[which] = rate;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (st == CM_OK && cudaGetLastError() != cudaSuccess) st = CM_ECUDA;
    *red_per_s = best[0];
    *load_per_s = best[1];
    return st;
}

}  // extern "C"
