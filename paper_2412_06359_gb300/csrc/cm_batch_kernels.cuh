// cm_batch_kernels.cuh -- the device side of the batched plan (cm_batch.cu):
// the window table's header, and the kernels of its phases (prep with the
// band count, grouping, splat, loss, adjoint, gradient, and the
// shared-memory tile variants of the splat and the adjoint).  Every kernel
// covers a range of windows of the table; see cm_batch.cu for the host side.
#pragma once

#include "cm_bands.cuh"
#include "cm_device.cuh"

namespace cmk {

struct BatchHdr {
    int32_t nwin;
    int32_t p_nseg;          // persistent step: segments of the queue
    int32_t p_total;         // persistent step: work items of the queue
    int32_t pad;
    long long total_chunks;  // event chunks of kEventThreads events
    int32_t total_ltiles;    // loss / gradient tiles (loss_tiles per window)
    int32_t total_ptiles;    // pixel tiles (pix_tiles per window)
};

// largest w in [lo, hi) with s[w] <= c (s non-decreasing; empty windows skipped)
__device__ __forceinline__ int find_ll(const long long* s, int lo, int hi, long long c)
{
    hi -= 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(s + mid) <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_i(const int* s, int lo, int hi, int c)
{
    hi -= 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(s + mid) <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int clamp_end(const BatchHdr* h, int w1) { return w1 < h->nwin ? w1 : h->nwin; }

// Each kernel covers windows [w0, w1) of the table (clamped to the windows in
// use).  Pixel passes walk per-window tiles, event passes chunks of 256 events.

__device__ __forceinline__ int tile_of(const Win& d, int x, int y)
{
    const int tx = min(max(x, 0), d.W - 1) / d.tile_px, ty = min(max(y, 0), d.H - 1) / d.tile_px;
    return ty * d.ntx + tx;
}

// Binning works on super-chunks of kSuperChunk events of one window: a block
// counts its super-chunk's events per tile in shared memory and touches the
// global counters once per tile, not once per event.
constexpr int kMaxBinTiles = 4096;  // windows with more tiles are not grouped
constexpr int kTileItemEvents = 4096;  // events of one work item of the shared-memory tile kernels

__device__ __forceinline__ void count_tiles(const Win& d, long long e0, long long e1, int* hist)
{
    const int nt = d.ntx * d.nty;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) atomicAdd(hist + tile_of(d, d.x[k], d.y[k]), 1);
    __syncthreads();
}

// zero the images of warped events and the quad accumulators of dL/dflow,
// build the flow quads (the motion field for depth input), reset the
// completion counters.  With `bands`, the blocks first run pass 1 of the band
// grouping (the count per band and super-chunk); it needs no zeroed state (the
// table's columns are written whole and its completion counter returns to zero
// when the last block has scanned the table), so it is not reset here.
// one pixel tile ti of the prep pass of window d: zero its share of the images
// and of the quad accumulators, build its flow quads, reset the completion
// counters (tile 0) and the tile grouping's counts
// the images of tile ti's share zeroed by the TMA engine: bulk copies
// (cp.async.bulk, 16-byte aligned, sizes in multiples of 16 bytes) from a
// zeroed shared-memory buffer (zsm: its shared address, kZeroBytes long),
// issued by thread 0, so the zero fill takes no store instructions of the
// SMs that the event kernels share (0.2-0.3% on the 64-window step); the
// caller waits for them before the block exits
constexpr unsigned kZeroBytes = 16384;

__device__ __forceinline__ void zero_images_bulk(const Win& d, int ti, unsigned zsm)
{
    if (threadIdx.x != 0) return;
    const size_t total = (size_t)d.R * plane_size(d) * sizeof(float4);
    size_t per = (total + d.pix_tiles - 1) / d.pix_tiles;
    per = (per + 15) / 16 * 16;
    const size_t a = (size_t)ti * per;
    const size_t b = a + per < total ? a + per : total;
    char* base = reinterpret_cast<char*>(d.iwe);
    for (size_t o = a; o < b; o += kZeroBytes) {
        const unsigned n = (unsigned)(b - o < kZeroBytes ? b - o : kZeroBytes);
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(base + o), "r"(zsm), "r"(n)
                     : "memory");
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

template <bool BULK = false>
__device__ __forceinline__ void prep_tile(const Win& d, int ti, unsigned zsm = 0)
{
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ti == 0 && threadIdx.x < 2) d.sync[threadIdx.x] = 0;
    // the tile grouping counts in a later kernel: its counter can be reset here
    if (ti == 0 && threadIdx.x == 2 && d.tile_cnt && !d.band_rows) *d.gsync = 0;
    const size_t HW = plane_size(d);
    const size_t stride = (size_t)d.pix_tiles * blockDim.x;
    // the window's images as one flat run of 32-byte chunks (the slab is 32-byte aligned)
    const size_t nf4 = (size_t)d.R * HW, n32 = nf4 / 2;
    if (BULK) {
        zero_images_bulk(d, ti, zsm);
    } else {
        for (size_t c = (size_t)ti * blockDim.x + threadIdx.x; c < n32; c += stride) st_v8(d.iwe + 2 * c, z4, z4);
        if ((nf4 & 1) && ti == 0 && threadIdx.x == 0) d.iwe[nf4 - 1] = z4;
    }
    for (size_t i = (size_t)ti * blockDim.x + threadIdx.x; i < HW; i += stride) {
        st_v8(d.dq + i, z4, z4);
        int u, v;
        pixel_uv(i, d.W, u, v);
        build_quad(d, u, v);
    }
    if (d.tile_cnt && !d.band_rows) {
        const int nt = d.ntx * d.nty;
        for (int i = ti * blockDim.x + threadIdx.x; i <= nt; i += (int)stride) {
            d.tile_cnt[i] = 0;
            if (i < nt) d.tile_cur[i] = 0;
        }
    }
}

__global__ void __launch_bounds__(kEventThreads) k_prep_batch(const BatchHdr* h, const Win* tab, const int* pstart,
                                                              const long long* sstart, int bands, int w0, int w1)
{
    __shared__ int hist[kMaxBands];
    __shared__ __align__(128) float4 zbuf[kZeroBytes / sizeof(float4)];
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    for (int i = threadIdx.x; i < (int)(kZeroBytes / sizeof(float4)); i += blockDim.x) zbuf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    // the zeros written through the generic proxy, read by the bulk copies through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const unsigned zsm = (unsigned)__cvta_generic_to_shared(zbuf);
    if (bands) {
        const long long cb = sstart[w0], ce = sstart[w1];
        for (long long c = cb + blockIdx.x; c < ce; c += gridDim.x) {
            const int w = find_ll(sstart, w0, w1, c);
            const Win d = tab[w];
            if (!d.tile_cnt || !d.band_rows) continue;
            const long long e0 = (c - sstart[w]) * kSuperChunk;
            const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
            band_count(d, (int)(c - sstart[w]), e0, e1, hist);
        }
    }
    const int tb = pstart[w0], te = pstart[w1];
    for (int tile = tb + blockIdx.x; tile < te; tile += gridDim.x) {
        const int w = find_i(pstart, w0, w1, tile);
        prep_tile<true>(tab[w], tile - pstart[w], zsm);
    }
    // the block's bulk zeroing complete (written) before it exits
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// binning, pass 1: events per tile (or per band and super-chunk); the block
// finishing a window's last super-chunk turns the counts into tile starts and
// the cursors (or into stable band offsets)
__global__ void __launch_bounds__(kEventThreads) k_bin_count_batch(const BatchHdr* h, const Win* tab,
                                                                    const long long* sstart, int w0, int w1)
{
    __shared__ int hist[kMaxBinTiles];
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const long long cb = sstart[w0], ce = sstart[w1];
    for (long long c = cb + blockIdx.x; c < ce; c += gridDim.x) {
        const int w = find_ll(sstart, w0, w1, c);
        const Win d = tab[w];
        if (!d.tile_cnt) continue;
        const long long e0 = (c - sstart[w]) * kSuperChunk;
        const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
        if (d.band_rows) {
            band_count(d, (int)(c - sstart[w]), e0, e1, hist);
            continue;
        }
        count_tiles(d, e0, e1, hist);
        const int nt0 = d.ntx * d.nty;
        for (int i = threadIdx.x; i < nt0; i += blockDim.x)
            if (hist[i]) atomicAdd(d.tile_cnt + i, hist[i]);
        const int chunks = (int)((d.n + kSuperChunk - 1) / kSuperChunk);
        if (last_tile_done(d.gsync, chunks)) {
            const int nt = d.ntx * d.nty;
            int carry = 0;
            for (int base = 0; base < nt; base += blockDim.x) {
                const int i = base + threadIdx.x;
                const int v = i < nt ? d.tile_cnt[i] : 0;
                int tot = 0;
                const int ex = block_scan_excl(v, &tot);
                if (i < nt) {
                    d.tile_cnt[i] = carry + ex;
                    d.tile_cur[i] = carry + ex;
                }
                carry += tot;
            }
            if (threadIdx.x == 0) d.tile_cnt[nt] = carry;
            __syncthreads();
            if (d.smem_tiles) {
                // work items of at most kTileItemEvents events per tile
                carry = 0;
                for (int base = 0; base < nt; base += blockDim.x) {
                    const int i = base + threadIdx.x;
                    const int v = i < nt ? (d.tile_cnt[i + 1] - d.tile_cnt[i] + kTileItemEvents - 1) / kTileItemEvents : 0;
                    int tot = 0;
                    const int ex = block_scan_excl(v, &tot);
                    if (i < nt) d.item_start[i] = carry + ex;
                    carry += tot;
                }
                if (threadIdx.x == 0) d.item_start[nt] = carry;
                __syncthreads();
            }
        }
    }
}

// binning, pass 2: a block reserves, per tile, one range of slots for its
// super-chunk's events (one global atomic per tile) and places them there (or
// places them at their stable band slots).  The scatter and the pixel passes
// are held to 64 registers: in the batched step their blocks share the SMs
// with the event kernels' (64 registers, four blocks per SM), and at 128 / 80
// registers they took the register file of two event blocks each (1267
// against 1279-1285 Mev/s for the 64-window step at 6 x 2).
__global__ void __launch_bounds__(kEventThreads, 4) k_bin_scatter_batch(const BatchHdr* h, const Win* tab,
                                                                      const long long* sstart, int w0, int w1)
{
    __shared__ int hist[kMaxBinTiles];
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const long long cb = sstart[w0], ce = sstart[w1];
    for (long long c = cb + blockIdx.x; c < ce; c += gridDim.x) {
        const int w = find_ll(sstart, w0, w1, c);
        const Win d = tab[w];
        if (!d.tile_cnt) continue;
        const long long e0 = (c - sstart[w]) * kSuperChunk;
        const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
        if (d.band_rows) {
            band_scatter(d, (int)(c - sstart[w]), e0, e1);
            continue;
        }
        count_tiles(d, e0, e1, hist);
        const int nt = d.ntx * d.nty;
        for (int i = threadIdx.x; i < nt; i += blockDim.x)
            if (hist[i]) hist[i] = atomicAdd(d.tile_cur + i, hist[i]);  // the block's first slot in tile i
        __syncthreads();
        for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
            const int16_t x = d.x[k], y = d.y[k];
            const int pos = atomicAdd(hist + tile_of(d, x, y), 1);
            d.rx[pos] = x;
            d.ry[pos] = y;
            d.rt[pos] = __ldg(d.t + k);
            d.rp[pos] = d.p[k];
        }
        __syncthreads();
    }
}

// events of a grouped window are read in tile order
__device__ __forceinline__ void use_grouped(Win& d)
{
    if (d.tile_cnt) {
        d.x = d.rx;
        d.y = d.ry;
        d.t = d.rt;
        d.p = d.rp;
    }
}

// the event kernels keep their trajectory points in shared memory up to 10
// bins: 64 registers and four blocks per SM.  With more bins they keep them
// in registers: two blocks per SM either way, and at 20 bins the register
// form measured faster (a one-window plan at 1280x720: 2.61 against 2.74 ms).
template <int MAXB>
constexpr bool kPointsSmem = MAXB <= 10;

template <int MAXB>
__global__ void __launch_bounds__(kEventThreads, MAXB <= 10 ? 4 : 2) k_splat_batch(const BatchHdr* h, const Win* tab,
                                                                const long long* cstart, int w0, int w1)
{
    __shared__ __align__(16) float pts[kPointsSmem<MAXB> ? 2 * (MAXB + 1) * kEventThreads : 1];
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const long long cb = cstart[w0], ce = cstart[w1];
    for (long long c = cb + blockIdx.x; c < ce; c += gridDim.x) {
        const int w = find_ll(cstart, w0, w1, c);
        Win d = tab[w];
        use_grouped(d);
        const long long k = (c - cstart[w]) * kEventThreads + threadIdx.x;
        if (k >= d.n || d.smem_tiles) continue;
        if (kPointsSmem<MAXB>) splat_event_smem<MAXB>(d, k, pts);
        else splat_event<MAXB>(d, k);
    }
}

template <int MAXB>
__global__ void __launch_bounds__(kEventThreads, MAXB <= 10 ? 4 : 2) k_adjoint_batch(const BatchHdr* h, const Win* tab,
                                                                  const long long* cstart, int w0, int w1)
{
    __shared__ __align__(16) float pts[kPointsSmem<MAXB> ? 2 * (MAXB + 1) * kEventThreads : 1];
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const long long cb = cstart[w0], ce = cstart[w1];
    for (long long c = cb + blockIdx.x; c < ce; c += gridDim.x) {
        const int w = find_ll(cstart, w0, w1, c);
        Win d = tab[w];
        use_grouped(d);
        const long long k = (c - cstart[w]) * kEventThreads + threadIdx.x;
        if (k >= d.n || d.smem_tiles) continue;
        // polarity-plane images
        if (kPointsSmem<MAXB>) adjoint_event_smem<MAXB, RedSink, true>(d, k, __ldg(d.dloss), pts);
        else adjoint_event<MAXB, RedSink, true>(d, k, __ldg(d.dloss));
    }
}

// ---------------------------------------------------------------------------
// Shared-memory tile accumulation (schedule bin 3).  The events of each window
// are grouped by 32x32-pixel tile and one block (512 threads, one per SM)
// takes one work item at a time: a tile's events, in runs of at most
// kTileItemEvents (a hot tile is several items).  The splat accumulates the
// (C, S) pairs of every point that lands in the item's tile, for the first
// kTileRefs references, in shared memory ([r][polarity][32][32] float2), and
// flushes the tile once: one 16-byte reduction per pixel pair that received
// anything.  The adjoint accumulates its pushes into the tile's per-cell
// records of dL/dflow ([32][32] of 32 bytes) the same way.  Points and pushes
// that land outside the tile reduce straight into global memory.
constexpr int kTileRefs = 12;      // references held in shared memory (12 x 16 KB)
constexpr int kTileThreads = 512;  // threads of a tile block (one block per SM)
// Sum the same-address updates of a warp before the shared atomic
// (__match_any_sync groups, the lowest lane of each collects by shuffles).
// Measured slower than leaving same-address lanes to the shared-memory atomic
// unit, which serialises them itself (64 windows, 640x480: 216 against 410
// Mev/s; motion-consistent windows, many events per pixel: 70 against 177), so
// it is off; kept to re-measure on other workloads.
constexpr bool kTileAggregate = false;

// warp-aggregated shared-memory add of N values at base + key * N (key < 0:
// nothing to add); every active lane of the warp calls it together
template <int N>
__device__ __forceinline__ void smem_add_agg(float* base, int key, const float (&v)[N])
{
    if (!kTileAggregate) {
        if (key >= 0) {
#pragma unroll
            for (int q = 0; q < N; ++q)
                if (v[q] != 0.0f) atomicAdd(base + (size_t)key * N + q, v[q]);
        }
        return;
    }
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(act, key);
    const int leader = __ffs(peers) - 1;
    const unsigned others = peers & ~(1u << leader);
    const int mine = lane == leader && key >= 0 ? __popc(others) : 0;
    const int rounds = __reduce_max_sync(act, (unsigned)mine);
    float acc[N];
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = v[q];
    for (int i = 0; i < rounds; ++i) {
        const int src = i < mine ? __fns(others, 0, i + 1) : lane;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const float o = __shfl_sync(act, v[q], src);
            if (i < mine) acc[q] += o;
        }
    }
    if (lane == leader && key >= 0) {
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (acc[q] != 0.0f) atomicAdd(base + (size_t)key * N + q, acc[q]);
    }
}

struct TileSink {
    float* img;  // splat: [rt][2][32][32] float2 (as floats)
    FQ* rec;     // adjoint: [32][32] cell records
    int x0, y0, rt;

    __device__ __forceinline__ int local(int x, int y) const
    {
        const int lx = x - x0, ly = y - y0;
        return (unsigned)lx < (unsigned)kSmemTile && (unsigned)ly < (unsigned)kSmemTile ? ly * kSmemTile + lx : -1;
    }
    // S4: the four corners of a point; those in the tile (references < rt) to
    // shared memory, the others straight to the polarity planes
    __device__ __forceinline__ void splat(const Win& d, int r, const Bil& s, float tbar, int pol2, int64_t) const
    {
        const size_t plane = (size_t)(2 * r + (pol2 >> 1)) * plane_size(d);
        float2* gimg = reinterpret_cast<float2*>(d.iwe);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cx = s.ix + (c & 1), cy = s.iy + (c >> 1);
            const float w = c == 0 ? s.w00 : (c == 1 ? s.w10 : (c == 2 ? s.w01 : s.w11));
            const bool has = (c & 1 ? s.ax > 0.0f : true) && (c >> 1 ? s.ay > 0.0f : true);
            const int li = has && r < rt ? local(cx, cy) : -1;
            const float v[2] = {w, __fmul_rn(w, tbar)};
            smem_add_agg<2>(img, li < 0 ? -1 : ((2 * r + (pol2 >> 1)) * kSmemTile * kSmemTile + li), v);
            if (has && li < 0) red_add_v2(reinterpret_cast<float*>(gimg + plane + (size_t)cy * d.W + cx), v[0], v[1]);
        }
    }
    // S6: a push sampled in cell s: hs * w_c * lambda to the cell's record
    __device__ __forceinline__ void scatter(const Win& d, int field, int, const Bil& s, float hx, float hy,
                                            int64_t) const
    {
        const int li = local(s.ix, s.iy);
        const float v[8] = {s.w00 * hx, s.w00 * hy, s.w10 * hx, s.w10 * hy,
                            s.w01 * hx, s.w01 * hy, s.w11 * hx, s.w11 * hy};
        smem_add_agg<8>(reinterpret_cast<float*>(rec), li, v);
        if (li < 0) {
            float* q = reinterpret_cast<float*>(d.dq + cell_index(d, field, s.ix, s.iy));
            red_add_v4(q, v[0], v[1], v[2], v[3]);
            if (s.ay > 0.0f) red_add_v4(q + 4, v[4], v[5], v[6], v[7]);
        }
    }
    // the first push of a chain, sampled at the event's own pixel (in the tile)
    __device__ __forceinline__ void point(const Win& d, int field, int, int xk, int yk, float vx, float vy,
                                          int64_t) const
    {
        const int li = local(xk, yk);
        const float v[8] = {vx, vy, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        smem_add_agg<8>(reinterpret_cast<float*>(rec), li, v);
        if (li < 0) red_add_v2(reinterpret_cast<float*>(d.dq + cell_index(d, field, xk, yk)), vx, vy);
    }
};

// work item `it` of window d: its tile's origin and its events [e0, e1) in the
// grouped copy (a tile's events in runs of kTileItemEvents)
__device__ __forceinline__ void tile_item(const Win& d, int it, int& x0, int& y0, long long& e0, long long& e1)
{
    const int nt = d.ntx * d.nty;
    int lo = 0, hi = nt - 1;  // the last tile t with item_start[t] <= it
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d.item_start[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    const int t = lo;
    x0 = (t % d.ntx) * kSmemTile;
    y0 = (t / d.ntx) * kSmemTile;
    e0 = d.tile_cnt[t] + (long long)(it - d.item_start[t]) * kTileItemEvents;
    e1 = e0 + kTileItemEvents < d.tile_cnt[t + 1] ? e0 + kTileItemEvents : d.tile_cnt[t + 1];
}

template <int MAXB>
__global__ void __launch_bounds__(kTileThreads, 1) k_splat_tiles_batch(const BatchHdr* h, const Win* tab, int w0,
                                                                        int w1)
{
    extern __shared__ float4 tile_smem[];
    float* img = reinterpret_cast<float*>(tile_smem);
    w1 = clamp_end(h, w1);
    for (int w = w0; w < w1; ++w) {
        Win d = tab[w];
        if (!d.smem_tiles) continue;
        use_grouped(d);
        const int items = d.item_start[d.ntx * d.nty];
        const int rt = min(d.R, kTileRefs), n = rt * 2 * kSmemTile * kSmemTile;
        const float2* acc = reinterpret_cast<const float2*>(img);
        float2* gimg = reinterpret_cast<float2*>(d.iwe);
        const size_t HW = plane_size(d);
        for (int it = blockIdx.x; it < items; it += gridDim.x) {
            int x0, y0;
            long long e0, e1;
            tile_item(d, it, x0, y0, e0, e1);
            for (int i = threadIdx.x; i < n; i += blockDim.x) reinterpret_cast<float2*>(img)[i] = make_float2(0.f, 0.f);
            __syncthreads();
            const TileSink sink{img, nullptr, x0, y0, rt};
            for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
                Traj<MAXB> P;
                splat_points<MAXB>(d, k, sink, P);
            }
            __syncthreads();
            // flush: one 16-byte reduction per pixel pair of the tile that received anything
            constexpr int T = kSmemTile, T2 = kSmemTile * kSmemTile;
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int q = i / (T2 / 2), li = 2 * (i % (T2 / 2)), lx = li % T, ly = li / T;
                const float2 a = acc[q * T2 + li], b = acc[q * T2 + li + 1];
                const int X = x0 + lx, Y = y0 + ly;
                if (Y >= d.H || X >= d.W) continue;
                const size_t gi = (size_t)q * HW + (size_t)Y * d.W + X;
                const bool two = X + 1 < d.W;
                if (a.x == 0.0f && (!two || b.x == 0.0f)) continue;
                float* g = reinterpret_cast<float*>(gimg + gi);
                if (two && !(gi & 1)) {
                    red_add_v4(g, a.x, a.y, b.x, b.y);
                } else {
                    if (a.x != 0.0f) red_add_v2(g, a.x, a.y);
                    if (two && b.x != 0.0f) red_add_v2(g + 2, b.x, b.y);
                }
            }
            __syncthreads();
        }
    }
}

template <int MAXB>
__global__ void __launch_bounds__(kTileThreads, 1) k_adjoint_tiles_batch(const BatchHdr* h, const Win* tab, int w0,
                                                                          int w1)
{
    extern __shared__ float4 tile_smem[];
    FQ* rec = reinterpret_cast<FQ*>(tile_smem);
    float4* r4 = reinterpret_cast<float4*>(rec);
    constexpr int T = kSmemTile, T2 = kSmemTile * kSmemTile;
    w1 = clamp_end(h, w1);
    for (int w = w0; w < w1; ++w) {
        Win d = tab[w];
        if (!d.smem_tiles) continue;
        use_grouped(d);
        const int items = d.item_start[d.ntx * d.nty];
        const float dl = __ldg(d.dloss);
        for (int it = blockIdx.x; it < items; it += gridDim.x) {
            int x0, y0;
            long long e0, e1;
            tile_item(d, it, x0, y0, e0, e1);
            for (int i = threadIdx.x; i < 2 * T2; i += blockDim.x) r4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            const TileSink sink{nullptr, rec, x0, y0, 0};
            for (long long k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
                Traj<MAXB> P;
                adjoint_points<MAXB, true>(d, k, dl, sink, P);
            }
            __syncthreads();
            // flush the cell records that received anything
            for (int i = threadIdx.x; i < T2; i += blockDim.x) {
                const int X = x0 + i % T, Y = y0 + i / T;
                if (Y >= d.H || X >= d.W) continue;
                const float4 a = r4[2 * i], b = r4[2 * i + 1];
                float* g = reinterpret_cast<float*>(d.dq + (size_t)Y * d.W + X);
                if (a.x != 0.0f || a.y != 0.0f || a.z != 0.0f || a.w != 0.0f) red_add_v4(g, a.x, a.y, a.z, a.w);
                if (b.x != 0.0f || b.y != 0.0f || b.z != 0.0f || b.w != 0.0f) red_add_v4(g + 4, b.x, b.y, b.z, b.w);
            }
            __syncthreads();
        }
    }
}

// loss pass 1 per tile; the block completing a window's last tile runs pass 2
__global__ void __launch_bounds__(256, 4) k_loss_batch(const BatchHdr* h, const Win* tab, const int* lstart, int w0,
                                                    int w1)
{
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const int tb = lstart[w0], te = lstart[w1];
    for (int tile = tb + blockIdx.x; tile < te; tile += gridDim.x) {
        const int w = find_i(lstart, w0, w1, tile);
        const Win d = tab[w];
        const int ti = tile - lstart[w];
        if (d.iwe_split) {
            if (plane_size(d) & 1)
                loss_tile_planes<false>(d, ti, d.loss_tiles);
            else
                loss_tile_planes<true>(d, ti, d.loss_tiles);
        } else {
            for (int r = 0; r < d.R; ++r) loss_tile(d, r, ti, d.loss_tiles, d.loss_part + (size_t)r * d.loss_tiles + ti);
        }
        if (last_tile_done(d.sync + 0, d.loss_tiles)) loss_final_window(d);
    }
}

// dL/dflow folded from the quad accumulators, and the depth / ego gradient per
// tile (the loss pass's tiles); the block completing a window's last tile
// reduces the six ego sums
__global__ void __launch_bounds__(256, 4) k_grad_batch(const BatchHdr* h, const Win* tab, const int* lstart, int w0,
                                                    int w1)
{
    w1 = clamp_end(h, w1);
    if (w0 >= w1) return;
    const int tb = lstart[w0], te = lstart[w1];
    for (int tile = tb + blockIdx.x; tile < te; tile += gridDim.x) {
        const int w = find_i(lstart, w0, w1, tile);
        const Win d = tab[w];
        if (!d.rho) {
            if (d.dq) fold_tile(d, tile - lstart[w], d.loss_tiles);  // flow input: dL/dflow only
            continue;
        }
        depth_ego_tile(d, tile - lstart[w], d.loss_tiles);
        if (last_tile_done(d.sync + 1, d.loss_tiles)) {
            __syncthreads();
            depth_ego_final_window(d, d.loss_tiles);
        }
    }
}


// ---------------------------------------------------------------------------
// The persistent step (schedule persist > 0): one kernel runs every phase of
// every window.  Each block takes work items from a device queue (one atomic
// counter), in the order of the plan's segment table: a segment is one phase
// of one window (its pixel tiles, super-chunks, event chunks or loss tiles),
// and the table staggers the windows (window w + 1's first phase comes
// `persist` phases after window w's), so a few windows are in flight at a
// time, the GPU stays full across a window's phase boundaries, and no launch
// or graph edge separates the phases.  Before its item's work a block waits,
// thread 0 spinning on the window's per-phase completion counters (an acquire
// load; bounded: after about 4 s it sets the plan's error word and skips the
// work), for the phases the item depends on; after the work it adds one to
// its own phase's counter (release).  Every dependency is an earlier phase of
// the same window, so it was taken from the queue earlier by a block that is
// running: the waits always end, whatever the grid size.  Data one item
// writes and a later item reads (images, quads, grouped events, statistics)
// are read through L2 (the coherent load path, NC = false).
enum PPhase { kPPrep = 0, kPBandCount = 1, kPBandScatter = 2, kPSplat = 3, kPLoss = 4, kPAdjoint = 5, kPGrad = 6 };
constexpr int kPCounters = 8;  // per window: the seven phase counters and one spare

struct PSeg {
    int32_t w, phase, start, count;  // items [start, start + count) of phase `phase` of window w
};

constexpr long long kSpinLimit = 1LL << 22;  // polls of at most ~1 us each

// thread 0: wait until *c >= target; false when the plan's error word is set or
// the wait gives up (then it sets the error word)
__device__ __forceinline__ bool wait_count(const int* c, int target, int* err)
{
    unsigned ns = 32;
    for (long long it = 0;; ++it) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if (v >= target) return true;
        int e;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(e) : "l"(err) : "memory");
        if (e) return false;
        if (it >= kSpinLimit) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
    }
}

__device__ __forceinline__ int chunks_of(const Win& d) { return (int)((d.n + kEventThreads - 1) / kEventThreads); }

// the dependencies of an item of phase ph of window d (counters dn): every
// earlier phase whose output it reads, directly or through a phase between
// them.  A phase with no items (the event phases of an empty window) passes
// its wait at once, so a later phase waits on the phases before it as well:
// the loss pass of an empty window must still find its images zeroed.
__device__ __forceinline__ bool wait_deps(const Win& d, int ph, const int* dn, int* err)
{
    const bool grouped = d.tile_cnt && d.band_rows;
    if (ph == kPBandCount) return true;
    if (ph == kPBandScatter) return wait_count(dn + kPBandCount, super_chunks(d), err);
    const int chunks = chunks_of(d);
    bool ok = ph == kPPrep || wait_count(dn + kPPrep, d.pix_tiles, err);
    if (ok && ph >= kPSplat && grouped) ok = wait_count(dn + kPBandScatter, super_chunks(d), err);
    if (ok && ph > kPSplat) ok = wait_count(dn + kPSplat, chunks, err);
    if (ok && ph > kPLoss) ok = wait_count(dn + kPLoss, d.loss_tiles, err);
    if (ok && ph > kPAdjoint) ok = wait_count(dn + kPAdjoint, chunks, err);
    return ok;
}

// q[0]: the queue head, q[1]: the error word; done: [windows][kPCounters];
// both zero at the start of the launch
// trajectory points in shared memory up to 10 bins (the phases' other shared
// arrays take 19 KB of the static 48 KB)
template <int MAXB>
constexpr bool kPersistPointsSmem = MAXB <= 10;

template <int MAXB>
__global__ void __launch_bounds__(kEventThreads, MAXB <= 10 ? 3 : 2)
    k_step_persistent(const BatchHdr* h, const Win* tab, const PSeg* seg, int* q, int* done)
{
    const int nseg = h->p_nseg, total = h->p_total;
    __shared__ __align__(16) float pts[kPersistPointsSmem<MAXB> ? 2 * (MAXB + 1) * kEventThreads : 1];
    __shared__ int hist[kMaxBands];
    __shared__ int s_item, s_ok;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(q, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= total) break;
        int lo = 0, hi = nseg - 1;  // the last segment with start <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&seg[mid].start) <= it) lo = mid;
            else hi = mid - 1;
        }
        const int w = __ldg(&seg[lo].w), ph = __ldg(&seg[lo].phase), sub = it - __ldg(&seg[lo].start);
        Win d = tab[w];
        int* dn = done + (size_t)w * kPCounters;
        if (threadIdx.x == 0) s_ok = wait_deps(d, ph, dn, q + 1);
        __syncthreads();
        if (s_ok) {
            switch (ph) {
            case kPPrep: prep_tile(d, sub); break;
            case kPBandCount:
            case kPBandScatter: {
                const long long e0 = (long long)sub * kSuperChunk;
                const long long e1 = e0 + kSuperChunk < d.n ? e0 + kSuperChunk : d.n;
                if (ph == kPBandCount) band_count(d, sub, e0, e1, hist);
                else band_scatter(d, sub, e0, e1);
                break;
            }
            case kPSplat:
            case kPAdjoint: {
                use_grouped(d);
                const long long k = (long long)sub * kEventThreads + threadIdx.x;
                if (k < d.n) {
                    if (ph == kPSplat) {
                        if (kPersistPointsSmem<MAXB>) splat_event_smem<MAXB, false>(d, k, pts);
                        else {
                            Traj<MAXB> P;
                            splat_points<MAXB, false>(d, k, RedSink(), P);
                        }
                    } else {
                        const float dl = __ldg(d.dloss);
                        if (kPersistPointsSmem<MAXB>) adjoint_event_smem<MAXB, RedSink, true, false>(d, k, dl, pts);
                        else {
                            Traj<MAXB> P;
                            adjoint_points<MAXB, true, false>(d, k, dl, RedSink(), P);
                        }
                    }
                }
                break;
            }
            case kPLoss:
                if (plane_size(d) & 1) loss_tile_planes<false>(d, sub, d.loss_tiles);
                else loss_tile_planes<true>(d, sub, d.loss_tiles);
                if (last_tile_done(d.sync + 0, d.loss_tiles)) loss_final_window(d);
                break;
            case kPGrad:
                if (!d.rho) {
                    if (d.dq) fold_tile(d, sub, d.loss_tiles);
                } else {
                    depth_ego_tile(d, sub, d.loss_tiles);
                    if (last_tile_done(d.sync + 1, d.loss_tiles)) {
                        __syncthreads();
                        depth_ego_final_window(d, d.loss_tiles);
                    }
                }
                break;
            default: break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(dn + ph, 1);
        }
    }
}

}  // namespace cmk
