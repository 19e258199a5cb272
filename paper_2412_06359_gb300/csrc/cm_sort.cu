// cm_sort.cu -- the deterministic path: sort-by-pixel segmented reduction.
//
// The splat (S4) and the flow-gradient scatter of the adjoint (S6) emit one
// entry per splat point or push (EmitSink in cm_device.cuh): a key, plane * HW
// plus the cell of the point's top-left bilinear corner, and a payload
// (x, y, a, b).  Entry k * stride + slot belongs to event k, so the entries
// start in a fixed order.  A stable LSD radix sort orders them by key; the
// start of every key's run is found; then one thread per output pixel adds,
// in a fixed order, the contributions of the four cells whose corners cover it
// (the cell itself, its left, upper and upper-left neighbours), each cell's
// entries in sorted order.  Every sum has the same operands in the same order
// on every run: the images of warped events and dL/dflow are bit-reproducible.
//
// Radix sort: 8-bit digits, as many passes as the largest key needs.  A pass
// (1) counts each tile's digits, (2) scans the digit-major count table, and
// (3) scatters each entry to its digit's offset plus its rank among the tile's
// entries with the same digit: tiles are walked in rounds of 256 consecutive
// entries, a warp ranks equal digits with __match_any_sync, warps add the counts
// of the warps before them, so equal keys keep their order (stable).
#include <cstdint>

#include "cm_device.cuh"
#include "cm_launch.h"
#include "cm_sort.h"

namespace cmk {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsThreads * kRsRounds;
constexpr int kRadix = 256;
constexpr int kScanChunk = 4096;

__global__ void __launch_bounds__(kRsThreads) k_fill_keys(uint32_t* key, int64_t n, uint32_t v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = v;
}

template <int MAXB>
__global__ void __launch_bounds__(kEventThreads) k_splat_emit(Win d, EmitSink s)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x)
        splat_event<MAXB>(d, k, s);
}

template <int MAXB>
__global__ void __launch_bounds__(kEventThreads) k_adjoint_emit(Win d, EmitSink s)
{
    const float dl = __ldg(d.dloss);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d.n; k += (int64_t)gridDim.x * blockDim.x)
        adjoint_event<MAXB>(d, k, dl, s);
}

// (1) per-tile digit counts, digit-major: hist[digit * nblk + tile]
__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint32_t* key, int64_t n, int shift, uint32_t* hist,
                                                        int nblk)
{
    __shared__ uint32_t cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t e = base + r * kRsThreads + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(key[e] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// block-wide exclusive scan of one value per thread (256 threads); returns the
// block total through *total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t ws[kRsThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kRsThreads / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kRsThreads / 32) ws[lane] = t;
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? ws[w - 1] : 0) + x - v;
    if (total) *total = ws[kRsThreads / 32 - 1];
    __syncthreads();
    return before;
}

// (2a) sums of chunks of kScanChunk values
__global__ void __launch_bounds__(kRsThreads) k_scan_reduce(const uint32_t* a, int64_t n, uint32_t* part)
{
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanChunk; i += kRsThreads)
        if (base + i < n) s += a[base + i];
    uint32_t tot = 0;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// (2b) exclusive scan of the chunk sums (one block)
__global__ void __launch_bounds__(kRsThreads) k_scan_top(uint32_t* part, int n)
{
    uint32_t carry = 0;
    for (int base = 0; base < n; base += kRsThreads) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < n ? part[i] : 0;
        uint32_t tot = 0;
        const uint32_t ex = block_exclusive_scan(v, &tot);
        if (i < n) part[i] = carry + ex;
        carry += tot;
    }
}

// (2c) exclusive scan inside each chunk, offset by the chunk's prefix
__global__ void __launch_bounds__(kRsThreads) k_scan_down(uint32_t* a, int64_t n, const uint32_t* part)
{
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    constexpr int per = kScanChunk / kRsThreads;
    uint32_t v[per];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
        const int64_t i = base + (int64_t)threadIdx.x * per + j;
        v[j] = i < n ? a[i] : 0;
        s += v[j];
    }
    uint32_t run = part[blockIdx.x] + block_exclusive_scan(s, nullptr);
#pragma unroll
    for (int j = 0; j < per; ++j) {
        const int64_t i = base + (int64_t)threadIdx.x * per + j;
        if (i < n) a[i] = run;
        run += v[j];
    }
}

// (3) stable scatter of one pass
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint32_t* kin, const uint32_t* vin, int64_t n,
                                                           int shift, const uint32_t* hist, int nblk, uint32_t* kout,
                                                           uint32_t* vout)
{
    __shared__ uint32_t run[kRadix];
    __shared__ uint16_t wc[kRsThreads / 32][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = hist[(size_t)threadIdx.x * nblk + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
        for (int i = 0; i < kRsThreads / 32; ++i) wc[i][threadIdx.x] = 0;
        __syncthreads();
        const int64_t e = base + r * kRsThreads + threadIdx.x;
        const bool valid = e < n;
        const uint32_t k = valid ? kin[e] : 0u;
        const uint32_t dg = valid ? (k >> shift) & (kRadix - 1) : (uint32_t)kRadix;
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) wc[w][dg] = (uint16_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[dg] + rank;
            for (int i = 0; i < w; ++i) pos += wc[i][dg];
            kout[pos] = k;
            vout[pos] = vin ? vin[e] : (uint32_t)e;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int i = 0; i < kRsThreads / 32; ++i) tot += wc[i][threadIdx.x];
        run[threadIdx.x] += tot;
    }
}

// start[c] = first sorted position with key >= c, for c = 0 .. kmax (keys equal
// to kmax are the unused slots and sort last)
__global__ void __launch_bounds__(kRsThreads) k_cell_start(const uint32_t* key, int64_t n, uint32_t kmax,
                                                           uint32_t* start)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cur = i < n ? (int64_t)min(key[i], kmax) : (int64_t)kmax;
        const int64_t prev = i == 0 ? -1 : (int64_t)min(key[i - 1], kmax);
        for (int64_t c = prev + 1; c <= cur; ++c) start[c] = (uint32_t)i;
    }
}

// one output pixel of one plane: the fixed-order sum over the entries of the
// four cells whose bilinear corners cover it
__global__ void __launch_bounds__(kRsThreads) k_cell_gather(const uint32_t* start, const uint32_t* vals,
                                                            const float4* pay, int W, int H, int nplanes, float* out,
                                                            int qdiv, int pstride)
{
    const size_t HW = (size_t)W * H;
    const size_t total = HW * nplanes;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / HW);
        const size_t p = t - (size_t)q * HW;
        int x, y;
        pixel_uv(p, W, x, y);
        const uint32_t* st = start + (size_t)q * HW;
        float a = 0.0f, b = 0.0f;
        // cell (x, y) as corner 00, (x-1, y) as 10, (x, y-1) as 01, (x-1, y-1) as 11
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cx = x - (c & 1), cy = y - (c >> 1);
            if (cx < 0 || cy < 0) continue;
            const size_t cell = (size_t)cy * W + cx;
            const uint32_t i0 = st[cell], i1 = st[cell + 1];
            for (uint32_t i = i0; i < i1; ++i) {
                const float4 v = pay[vals[i]];
                const Bil s = bil_frac(v.x, v.y);
                const float wgt = c == 0 ? s.w00 : (c == 1 ? s.w10 : (c == 2 ? s.w01 : s.w11));
                a = __fadd_rn(a, __fmul_rn(wgt, v.z));
                b = __fadd_rn(b, __fmul_rn(wgt, v.w));
            }
        }
        float* o = out + ((size_t)(q / qdiv) * HW + p) * pstride + (q % qdiv) * 2;
        o[0] = a;
        o[1] = b;
    }
}

int grid_for(int64_t n, int per_block, int cap)
{
    const int64_t g = (n + per_block - 1) / per_block;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

int key_bits(uint32_t kmax)
{
    int b = 0;
    while (b < 32 && (kmax >> b) != 0) ++b;
    return b;
}

// sort the n entries in sb (keys in sb.ka, values implicit) and add them into out
cudaError_t sort_and_gather(const Win& d, SortBufs& sb, int64_t n, uint32_t kmax, int nplanes, float* out, int qdiv,
                            int pstride, cudaStream_t st)
{
    if (n <= 0) return cudaErrorInvalidValue;  // callers only sort non-empty entry lists
    const int nblk = (int)((n + kRsTile - 1) / kRsTile);
    const int64_t L = (int64_t)kRadix * nblk;
    const int nchunk = (int)((L + kScanChunk - 1) / kScanChunk);
    uint32_t* kin = sb.ka;
    uint32_t* kout = sb.kb;
    uint32_t* vin = nullptr;  // identity values on the first pass
    uint32_t* vout = sb.va;
    const int passes = (key_bits(kmax) + 7) / 8;
    for (int ps = 0; ps < passes; ++ps) {
        const int shift = 8 * ps;
        {
            KernelScope ks("k_rs_hist", st);
            k_rs_hist<<<nblk, kRsThreads, 0, st>>>(kin, n, shift, sb.hist, nblk);
        }
        {
            KernelScope ks("k_rs_scan", st, 3);
            k_scan_reduce<<<nchunk, kRsThreads, 0, st>>>(sb.hist, L, sb.part);
            k_scan_top<<<1, kRsThreads, 0, st>>>(sb.part, nchunk);
            k_scan_down<<<nchunk, kRsThreads, 0, st>>>(sb.hist, L, sb.part);
        }
        {
            KernelScope ks("k_rs_scatter", st);
            k_rs_scatter<<<nblk, kRsThreads, 0, st>>>(kin, vin, n, shift, sb.hist, nblk, kout, vout);
        }
        // ping-pong
        uint32_t* tk = kin;
        kin = kout;
        kout = tk;
        vin = vout;
        vout = (vout == sb.va) ? sb.vb : sb.va;
    }
    const uint32_t* vals = vin;
    {
        KernelScope ks("k_cell_start", st);
        k_cell_start<<<grid_for(n + 1, kRsThreads, 4096), kRsThreads, 0, st>>>(kin, n, kmax, sb.start);
    }
    {
        KernelScope ks("k_cell_gather", st);
        const int64_t total = (int64_t)d.W * d.H * nplanes;
        k_cell_gather<<<grid_for(total, kRsThreads, 8192), kRsThreads, 0, st>>>(sb.start, vals, sb.pay, d.W, d.H,
                                                                                 nplanes, out, qdiv, pstride);
    }
    return cudaGetLastError();
}

}  // namespace

SortSizes sort_sizes(int64_t max_events, int R, int B, int nfb, size_t HW)
{
    SortSizes z;
    z.entries = (size_t)max_events * (size_t)(R > B + 1 ? R : B + 1);
    const size_t nblk = (z.entries + kRsTile - 1) / kRsTile;
    z.hist = (size_t)kRadix * (nblk < 1 ? 1 : nblk);
    z.part = (z.hist + kScanChunk - 1) / kScanChunk;
    const size_t planes = (size_t)(2 * R > nfb ? 2 * R : nfb);
    z.start = planes * HW + 1;
    return z;
}

cudaError_t sort_splat(const Win& d, SortBufs& sb, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaMemsetAsync(d.iwe, 0, (size_t)d.R * plane_size_host(d) * sizeof(float4), st);
    const int64_t n = d.n * d.R;
    const uint32_t kmax = (uint32_t)(2 * (size_t)d.R * plane_size_host(d));
    {
        KernelScope ks("k_fill_keys", st);
        k_fill_keys<<<grid_for(n, kRsThreads, 4096), kRsThreads, 0, st>>>(sb.ka, n, kmax);
    }
    EmitSink sink{sb.ka, sb.pay, d.R};
    const int g = grid_for(d.n, kEventThreads, sm_count * 8);
    {
        KernelScope ks("k_splat_emit", st);
        if (d.B <= 1) k_splat_emit<1><<<g, kEventThreads, 0, st>>>(d, sink);
        else if (d.B <= 10) k_splat_emit<10><<<g, kEventThreads, 0, st>>>(d, sink);
        else if (d.B <= 20) k_splat_emit<20><<<g, kEventThreads, 0, st>>>(d, sink);
        else k_splat_emit<32><<<g, kEventThreads, 0, st>>>(d, sink);
    }
    return sort_and_gather(d, sb, n, kmax, 2 * d.R, reinterpret_cast<float*>(d.iwe), 2, 4, st);
}

cudaError_t sort_adjoint(const Win& d, SortBufs& sb, int sm_count, cudaStream_t st)
{
    if (d.n == 0) return cudaMemsetAsync(d.dflow, 0, (size_t)d.nfb * plane_size_host(d) * sizeof(float2), st);
    const int64_t n = d.n * (d.B + 1);
    const uint32_t kmax = (uint32_t)((size_t)d.nfb * plane_size_host(d));
    {
        KernelScope ks("k_fill_keys", st);
        k_fill_keys<<<grid_for(n, kRsThreads, 4096), kRsThreads, 0, st>>>(sb.ka, n, kmax);
    }
    EmitSink sink{sb.ka, sb.pay, d.B + 1};
    const int g = grid_for(d.n, kEventThreads, sm_count * 8);
    {
        KernelScope ks("k_adjoint_emit", st);
        if (d.B <= 1) k_adjoint_emit<1><<<g, kEventThreads, 0, st>>>(d, sink);
        else if (d.B <= 10) k_adjoint_emit<10><<<g, kEventThreads, 0, st>>>(d, sink);
        else if (d.B <= 20) k_adjoint_emit<20><<<g, kEventThreads, 0, st>>>(d, sink);
        else k_adjoint_emit<32><<<g, kEventThreads, 0, st>>>(d, sink);
    }
    return sort_and_gather(d, sb, n, kmax, d.nfb, reinterpret_cast<float*>(d.dflow), 1, 2, st);
}

}  // namespace cmk
