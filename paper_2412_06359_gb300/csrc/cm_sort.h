// cm_sort.h -- the deterministic sort-by-pixel path (cm_sort.cu), internal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cm_device.cuh"

namespace cmk {

inline size_t plane_size_host(const Win& d) { return (size_t)d.W * (size_t)d.H; }

// device buffers of the sort path (inside a workspace)
struct SortBufs {
    uint32_t* ka;   // [entries] keys (emitted here), ping-pong with kb
    uint32_t* kb;
    uint32_t* va;   // [entries] entry indices, ping-pong with vb
    uint32_t* vb;
    float4* pay;    // [entries] (x, y, a, b)
    uint32_t* hist; // [256 x tiles] digit counts, scanned in place
    uint32_t* part; // chunk sums of the scan
    uint32_t* start;// [planes x HW + 1] first sorted position of every key
};

// element counts of each buffer for windows of up to max_events events
struct SortSizes {
    size_t entries, hist, part, start;
};

SortSizes sort_sizes(int64_t max_events, int R, int B, int nfb, size_t HW);

// S2-S4 into d.iwe (every pixel written; no zeroing needed)
cudaError_t sort_splat(const Win& d, SortBufs& sb, int sm_count, cudaStream_t st);
// S6 into d.dflow (every pixel of every field written)
cudaError_t sort_adjoint(const Win& d, SortBufs& sb, int sm_count, cudaStream_t st);

}  // namespace cmk
