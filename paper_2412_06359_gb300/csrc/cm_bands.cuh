// cm_bands.cuh -- grouping a window's events by band of image rows, keeping
// their time order within each band (a counting sort over super-chunks of
// kSuperChunk events), used by the batched plan and the single-window calls:
// events in flight then touch one strip of the images, whose lines stay in L2,
// while the events of a warp still share their bin.
#pragma once

#include "cm_device.cuh"

namespace cmk {

// block-wide exclusive scan (any blockDim multiple of 32 up to 1024); returns
// the block total through *total
__device__ __forceinline__ int block_scan_excl(int v, int* total)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        ws[lane] = t;
    }
    __syncthreads();
    const int before = (w > 0 ? ws[w - 1] : 0) + x - v;
    *total = ws[nw - 1];
    __syncthreads();
    return before;
}

// Binning works on super-chunks of kSuperChunk events of one window: a block
// counts its super-chunk's events per band in shared memory and touches the
// global counters once per band, not once per event.
constexpr int kSuperChunk = 4096;
constexpr int kBandRows = 32;       // rows per band of the stable band grouping
constexpr int kMaxBands = 128;      // windows with more bands (H > 4096) are not grouped

__device__ __forceinline__ int band_of(const Win& d, int y) { return min(max(y, 0), d.H - 1) / d.band_rows; }

__host__ __device__ __forceinline__ int super_chunks(const Win& d) { return (int)((d.n + kSuperChunk - 1) / kSuperChunk); }

constexpr int kRounds = kSuperChunk / kEventThreads;  // 256-event rounds of a super-chunk
static_assert(kRounds * kEventThreads == kSuperChunk, "a super-chunk is whole rounds of a block");

// band grouping, pass 1 for super-chunk sc = [e0, e1): its events per band,
// column sc of the band-major [band][super-chunk] table (warp-aggregated
// shared-memory counts; the rows of all rounds are loaded first, so the block
// waits on memory once).  The block completing a window's last super-chunk
// scans the whole table in band-major order: entry (b, sc) becomes the first
// slot of super-chunk sc's events of band b, so the bands keep the order of
// the super-chunks.
__device__ __forceinline__ void band_count(const Win& d, int sc, long long e0, long long e1, int* hist)
{
    const int nb = d.nty, nsc = super_chunks(d), lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    int16_t yr[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long k = e0 + r * kEventThreads + threadIdx.x;
        yr[r] = k < e1 ? d.y[k] : (int16_t)0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long k = e0 + r * kEventThreads + threadIdx.x;
        const int b = k < e1 ? band_of(d, yr[r]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(hist + b, __popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) d.tile_cnt[(size_t)i * nsc + sc] = hist[i];
    if (last_tile_done(d.gsync, nsc)) {
        const int total = nb * nsc;
        int carry = 0;
        for (int base = 0; base < total; base += blockDim.x) {
            const int i = base + threadIdx.x;
            const int v = i < total ? __ldcg(d.tile_cnt + i) : 0;  // other blocks' columns, from L2
            int tot = 0;
            const int ex = block_scan_excl(v, &tot);
            if (i < total) d.tile_cnt[i] = carry + ex;
            carry += tot;
        }
        __syncthreads();
    }
}

// band grouping, pass 2 for super-chunk sc: its events (all rounds loaded
// first) go to the slots of their band that the count pass reserved for this
// super-chunk, so the bands keep the order of the super-chunks; within one
// super-chunk's share of a band (4096 consecutive events, a small part of the
// window's time span) a warp takes a run of slots per band through one
// shared-memory atomic (lanes in order), the warps and rounds in any order
__device__ __forceinline__ void band_scatter(const Win& d, int sc, long long e0, long long e1)
{
    __shared__ int cur[kMaxBands];
    const int nb = d.nty, nsc = super_chunks(d), lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) cur[i] = d.tile_cnt[(size_t)i * nsc + sc];
    int16_t xr[kRounds], yr[kRounds];
    float tr[kRounds];
    int8_t pr[kRounds];
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long k = e0 + r * kEventThreads + threadIdx.x;
        const bool ok = k < e1;
        xr[r] = ok ? d.x[k] : (int16_t)0;
        yr[r] = ok ? d.y[k] : (int16_t)0;
        tr[r] = ok ? __ldg(d.t + k) : 0.0f;
        pr[r] = ok ? d.p[k] : (int8_t)0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
        const long long k = e0 + r * kEventThreads + threadIdx.x;
        const bool ok = k < e1;
        const int b = ok ? band_of(d, yr[r]) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (ok && lane == leader) first = atomicAdd(cur + b, __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (ok) {
            const int pos = first + __popc(peers & ((1u << lane) - 1u));
            d.rx[pos] = xr[r];
            d.ry[pos] = yr[r];
            d.rt[pos] = tr[r];
            d.rp[pos] = pr[r];
        }
    }
    __syncthreads();
}

}  // namespace cmk
