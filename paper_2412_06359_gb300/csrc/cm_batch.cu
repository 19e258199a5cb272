// cm_batch.cu -- the batched path: the loss and gradient of many windows,
// replayed from one CUDA graph.
//
// Work decomposition.  The events of window w form ceil(n_w / 256) chunks and
// its pixel passes form per-window tiles; device prefix tables map a chunk or
// tile to its window (binary search), so windows of very different sizes share
// a launch with no padding.  Every kernel covers a range of windows.
//
// Layout.  A window's images of warped events are polarity planes of (C, S)
// pairs ([R][2][H][W] float2), so the two corners of a splat row that start on
// a 16-byte boundary take one 16-byte reduction (and one gather in the
// adjoint).  The flow is kept as 32-byte quads (the four values a bilinear
// sample reads) and dL/dflow is accumulated per cell in the same layout, then
// folded per pixel by the gradient pass.
//
// Schedule.  A window's images of warped events (R x H x W x 16 bytes, 54 MB at
// 640x480 with 11 references) are zeroed by the prep pass, reduced into by the
// splat, read by the loss pass and gathered by the adjoint.  The schedule
// groups windows (group = windows per kernel) and runs the groups on several
// concurrent chains of the graph, each chain taking its groups one after
// another, so the chains overlap each other's tails and launch gaps and their
// kernels share the SMs; group 0 puts every window in each kernel on one
// chain.  Fewer windows in flight would keep their images in the 129 MB L2
// but leave the GPU idle between a window's phases (measured: the 64-window
// step is fastest with 12-14 windows in flight).  Alternatives behind the same
// interface: a persistent kernel pulling every window's phases from a device
// work queue (persist > 0), and the deterministic mode (CM_SPLAT_SORT: each
// window whole through the sort path, one window at a time per chain).
// cm_batch_autotune times the candidates on the plan's own windows.

// The window table, the prefix tables and the totals live in device memory;
// cm_batch_set_windows rewrites the staging copy and the next cm_batch_run
// uploads it before the replay.  With group 0 the graph stays valid for any
// windows that fit the plan; otherwise it is captured again for the new set.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cm.h"
#include "cm_bands.cuh"
#include "cm_batch_kernels.cuh"
#include "cm_launch.h"
#include "cm_sort.h"


static_assert(cmk::kMaxRefs >= CM_MAX_BINS + 1, "per-reference shared arrays hold every reference");

using cmk::BatchHdr;
using cmk::Win;

namespace {

constexpr int kPhases = 9;
const char* const kPhaseName[kPhases + 1] = {"k_prep_batch",        "k_bin_count_batch", "k_bin_scatter_batch",
                                             "k_splat_batch",       "k_loss_batch",      "k_adjoint_batch",
                                             "k_grad_batch",        "k_splat_tiles_batch",
                                             "k_adjoint_tiles_batch", "k_step_persistent"};
constexpr int kPersistentPhase = kPhases;  // the name of the persistent step's node
constexpr int kMaxPersist = 8;             // largest persist value: a queue staggered by 7 phases
constexpr int kSortChains = 8;             // deterministic mode: concurrent chains (one set of sort buffers each)
// the order of the phases in a window group's chain (the tile phases run with bin 3 only)
constexpr int kPhaseOrder[kPhases] = {0, 1, 2, 3, 7, 4, 5, 8, 6};
constexpr int kSyncInts = 4;  // per window: loss, gradient and binning counters (one spare)
constexpr int kMaxChains = 8;

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// the persistent step's queue head, error word and per-window counters
size_t pq_bytes(int cap) { return (2 + (size_t)cap * cmk::kPCounters) * sizeof(int32_t); }

// dynamic shared memory of the tile kernels: the splat's images of the tile
// for min(R, kTileRefs) references, the adjoint's cell records
size_t tiles_smem(const cm_loss_cfg& cfg, int which)
{
    const int R = cfg.ref_mode == CM_REF_END ? 1 : cfg.nbins + 1;
    const int rt = R < cmk::kTileRefs ? R : cmk::kTileRefs;
    constexpr size_t T2 = (size_t)cmk::kSmemTile * cmk::kSmemTile;
    return which == 0 ? (size_t)rt * 2 * T2 * sizeof(float2) : T2 * sizeof(cmk::FQ);
}

int tiles_for(size_t hw, size_t px_per_tile, int cap)
{
    size_t t = (hw + px_per_tile - 1) / px_per_tile;
    if (t < 1) t = 1;
    if (t > (size_t)cap) t = cap;
    return (int)t;
}

// Tiles of a window's pixel passes (a tile is one block's share, 256 threads):
// 2048 pixels of every reference for the loss pass and the gradient pass (8
// pixels per thread), 512 pixels for the prep pass (2 per thread: halving the
// prep tiles' pixels made prep faster on GB300 at 640x480).
int loss_tiles_for(size_t hw) { return tiles_for(hw, 2048, 2048); }
int pix_tiles_for(size_t hw) { return tiles_for(hw, 512, 4096); }

int refs_of(const cm_loss_cfg& c) { return c.ref_mode == CM_REF_END ? 1 : c.nbins + 1; }

// device bytes of the per-window slabs for a list of windows
struct Need {
    size_t iwe, flow, dflow, quad, part, stat, dego, bins, warp;
    cmk::SortSizes sort;  // the deterministic mode's sort buffers, sized for the largest window (else zero)
};

bool window_ok(const cm_window& w)
{
    const cm_camera& c = w.cam;
    if (c.width < 2 || c.height < 2 || c.width > 32767 || c.height > 32767) return false;
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !std::isfinite(c.fx) || !std::isfinite(c.fy)) return false;
    if (!std::isfinite(c.cx) || !std::isfinite(c.cy)) return false;
    const cm_events& e = w.ev;
    if (e.n < 0 || (e.n > 0 && (!e.x || !e.y || !e.t || !e.p))) return false;
    if (!std::isfinite(e.t0) || !std::isfinite(e.t1) || !(e.t1 - e.t0 > 0.0f)) return false;
    if (!w.dloss || !w.loss_out) return false;
    if (!w.flow && (!w.inv_depth || !w.ego6 || !std::isfinite(w.dt_window))) return false;
    if (w.flow && (w.dinv_depth || w.dego6)) return false;
    if (reinterpret_cast<uintptr_t>(w.scratch) % 256) return false;
    return true;
}

bool cfg_ok(const cm_loss_cfg* cfg)
{
    if (!cfg || cfg->nbins < 1 || cfg->nbins > CM_MAX_BINS) return false;
    if (cfg->ref_mode != CM_REF_END && cfg->ref_mode != CM_REF_ALL_EDGES) return false;
    if (cfg->splat != CM_SPLAT_AUTO && cfg->splat != CM_SPLAT_ATOMIC && cfg->splat != CM_SPLAT_TILES &&
        cfg->splat != CM_SPLAT_SORT)
        return false;
    return (cfg->store_warps == 0 || cfg->store_warps == 1) && std::isfinite(cfg->eps);
}

size_t bin_bytes(int W, int H, int64_t n);

Need need_of(const cm_window* wins, int32_t nwin, const cm_loss_cfg& cfg)
{
    Need n{};
    const int R = refs_of(cfg);
    for (int i = 0; i < nwin; ++i) {
        // the grouped copy of the events is the plan's, also for a window with its own scratch
        n.bins += bin_bytes(wins[i].cam.width, wins[i].cam.height, wins[i].ev.n);
        if (wins[i].scratch) continue;  // the window brings its other buffers
        const size_t HW = (size_t)wins[i].cam.width * wins[i].cam.height;
        n.iwe += up256((size_t)R * HW * sizeof(float4));
        if (!wins[i].dflow && wins[i].flow) n.dflow += HW * sizeof(float2);
        n.quad += 2 * HW * sizeof(cmk::FQ);
        n.part += (size_t)R * loss_tiles_for(HW) * sizeof(float2);
        n.stat += (size_t)R;
        n.dego += (size_t)loss_tiles_for(HW) * 6 * sizeof(float);
        if (cfg.store_warps) n.warp += up256((size_t)(cfg.nbins + 1) * wins[i].ev.n * sizeof(float2));
    }
    if (cfg.splat == CM_SPLAT_SORT) {
        // the deterministic mode runs one window at a time on each of at most
        // kSortChains chains: the windows of a chain share one image slab and
        // one quad slab (the largest window's size), and no events are grouped
        int64_t mn = 0;
        size_t mhw = 0;
        for (int i = 0; i < nwin; ++i) {
            mn = std::max(mn, wins[i].ev.n);
            mhw = std::max(mhw, (size_t)wins[i].cam.width * wins[i].cam.height);
        }
        const size_t slots = (size_t)std::min(nwin, kSortChains);
        n.iwe = slots * up256((size_t)R * mhw * sizeof(float4));
        n.quad = slots * 2 * mhw * sizeof(cmk::FQ);
        n.bins = 0;
        n.sort = cmk::sort_sizes(mn, R, cfg.nbins, 1, mhw);
    }
    return n;
}

// device bytes of the spatial grouping of a window: the count table (tile
// starts and cursors, or the band x super-chunk offsets, whichever is larger)
// and the grouped events
size_t bin_bytes(int W, int H, int64_t n)
{
    // the smaller tiles of bin 3 are the most (their table also holds the work items)
    const size_t nt = (size_t)((W + cmk::kSmemTile - 1) / cmk::kSmemTile) * ((H + cmk::kSmemTile - 1) / cmk::kSmemTile);
    const size_t nband = (size_t)((H + cmk::kBandRows - 1) / cmk::kBandRows) *
                         (size_t)((n + cmk::kSuperChunk - 1) / cmk::kSuperChunk);
    const size_t table = 3 * nt + 2 > nband ? 3 * nt + 2 : nband;
    return up256(table * sizeof(int32_t)) + 2 * up256(2 * (size_t)n) + up256(4 * (size_t)n) + up256((size_t)n);
}

// a window's own scratch: the per-window buffers, one after another
struct WinScratch {
    size_t iwe, flow, dflow, fq, dq, part, norm, lr, nnz, dego, sync, total;
};

WinScratch win_scratch(size_t HW, int R)
{
    WinScratch s;
    size_t o = 0;
    s.iwe = o;
    o = up256(o + (size_t)R * HW * sizeof(float4));
    s.dflow = o;
    o = up256(o + HW * sizeof(float2));
    s.fq = o;
    o = up256(o + HW * sizeof(cmk::FQ));
    s.dq = o;
    o = up256(o + HW * sizeof(cmk::FQ));
    s.part = o;
    o = up256(o + (size_t)R * loss_tiles_for(HW) * sizeof(float2));
    s.norm = o;
    o = up256(o + (size_t)R * sizeof(float));
    s.lr = o;
    o = up256(o + (size_t)R * sizeof(float));
    s.nnz = o;
    o = up256(o + (size_t)R * sizeof(int32_t));
    s.dego = o;
    o = up256(o + (size_t)loss_tiles_for(HW) * 6 * sizeof(float));
    s.sync = o;
    o = up256(o + kSyncInts * sizeof(int32_t));
    s.total = o;
    return s;
}

struct Layout {
    size_t hdr, tab, cstart, sstart, lstart, pstart, pseg, table_end;  // the uploaded region [0, table_end)
    size_t pq;  // persistent step: queue head, error word, [windows][kPCounters] counters (zeroed per run)
    size_t iwe, flow, dflow, quad, part, norm, lr, nnz, dego, sync, bins, warp;
    size_t ska, skb, sva, svb, spay, shist, spart, sstart_keys;  // deterministic mode: chain 0's sort buffers
    size_t sort_stride;                                         // bytes from one chain's set to the next
    size_t total;
};

Layout layout_of(int cap, const Need& n)
{
    Layout L;
    size_t o = 0;
    L.hdr = o;
    o = up256(o + sizeof(BatchHdr));
    L.tab = o;
    o += (size_t)cap * sizeof(Win);
    L.cstart = o = (o + 15) / 16 * 16;
    o += (size_t)(cap + 1) * sizeof(long long);
    L.sstart = o;
    o += (size_t)(cap + 1) * sizeof(long long);
    L.lstart = o;
    o += (size_t)(cap + 1) * sizeof(int);
    L.pstart = o;
    o += (size_t)(cap + 1) * sizeof(int);
    L.pseg = o = (o + 15) / 16 * 16;
    o += (size_t)cap * 7 * sizeof(cmk::PSeg);
    L.table_end = o = up256(o);
    L.pq = o;
    o = up256(o + pq_bytes(cap));
    L.iwe = o;
    o = up256(o + n.iwe);
    L.dflow = o;
    o = up256(o + n.dflow);
    L.quad = o;
    o = up256(o + n.quad);
    L.part = o;
    o = up256(o + n.part);
    L.norm = o;
    o = up256(o + n.stat * sizeof(float));
    L.lr = o;
    o = up256(o + n.stat * sizeof(float));
    L.nnz = o;
    o = up256(o + n.stat * sizeof(int32_t));
    L.dego = o;
    o = up256(o + n.dego);
    L.sync = o;
    o = up256(o + (size_t)cap * kSyncInts * sizeof(int32_t));
    L.bins = o;
    o = up256(o + n.bins);
    L.warp = o;
    o = up256(o + n.warp);
    // the deterministic mode: one set of sort buffers per chain (kSortChains sets)
    const cmk::SortSizes& z = n.sort;
    const size_t sort_begin = o;
    L.ska = o;
    o = up256(o + z.entries * 4);
    L.skb = o;
    o = up256(o + z.entries * 4);
    L.sva = o;
    o = up256(o + z.entries * 4);
    L.svb = o;
    o = up256(o + z.entries * 4);
    L.spay = o;
    o = up256(o + z.entries * 16);
    L.shist = o;
    o = up256(o + z.hist * 4);
    L.spart = o;
    o = up256(o + z.part * 4);
    L.sstart_keys = o;
    o = up256(o + z.start * 4);
    L.sort_stride = o - sort_begin;
    o += (kSortChains - 1) * L.sort_stride;
    L.total = o;
    return L;
}

// one kernel node of the graph and the event-record nodes around it
struct ProfNode {
    int phase;
    cudaEvent_t ea, eb;           // the plan's own events (recorded when timing is off)
    cudaGraphNode_t na, nb;
};

struct Group {
    int w0, w1, chain;
    long long chunks;
    int ltiles, ptiles;
};

}  // namespace

struct cm_batch {
    char* base = nullptr;
    size_t bytes = 0;
    cm_loss_cfg cfg{};
    int cap = 0;
    Need capn{};
    Layout L{};
    unsigned char* staging = nullptr;  // pinned host copy of [0, table_end)
    bool dirty = false;
    cudaEvent_t staged = nullptr;      // recorded after the last upload of the staging copy
    int nwin = 0;
    std::vector<long long> chunks;     // per window, host copy
    std::vector<int> ltiles, ptiles;   // per window, host copy
    std::vector<const float*> stat_lr; // per window: device L_r and N_nz of the last run
    std::vector<const int32_t*> stat_nnz;
    std::vector<cm_window> last;       // the windows of the last staging (re-staged when grouping changes)
    int grid_events = 0, grid_tiles = 0, grid_tiles_smem = 0, grid_persist = 0;
    int grid_splat = 0;  // the splat: eight blocks per SM in waves (its reductions need no reply)
    cm_batch_schedule sched{2, 1, 0};
    int stall_window = -1;             // test hook: the persistent queue leaves out this window's prep pass
    long long graph_kernels = 0;       // kernel nodes of the captured graph
    bool stale = true;                 // the graph must be (re)captured before the next replay
    cudaStream_t streams[kMaxChains] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxChains] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<ProfNode> prof;
    bool swapped = false;
};

namespace {

// fill the staging copy of the table for these windows; checks the capacities
std::vector<Group> make_groups(const cm_batch* b);

// The persistent step's queue: for every window its phases in order (prep,
// the band count and scatter when its events are grouped by band, splat,
// loss, adjoint, gradient), each a segment of work items; the segments of all
// windows sorted by (window x stagger + phase rank, window), so window w + 1's
// first phase comes `stagger` phases after window w's (stagger 0: phase by
// phase over all windows) and a window's phases keep their order (every
// dependency is queued before its dependants).
void build_queue(int stagger, const Win* tab, int nwin, int stall_window, cmk::PSeg* seg, BatchHdr* h)
{
    struct Key {
        long long key;
        int w, phase, count;
    };
    std::vector<Key> keys;
    for (int w = 0; w < nwin; ++w) {
        const Win& d = tab[w];
        const bool grouped = d.tile_cnt && d.band_rows;
        const int chunks = (int)((d.n + cmk::kEventThreads - 1) / cmk::kEventThreads);
        const int nsc = (int)((d.n + cmk::kSuperChunk - 1) / cmk::kSuperChunk);
        const int order[7] = {cmk::kPPrep, cmk::kPBandCount, cmk::kPBandScatter, cmk::kPSplat,
                              cmk::kPLoss, cmk::kPAdjoint,   cmk::kPGrad};
        int rank = 0;
        for (int ph : order) {
            if (!grouped && (ph == cmk::kPBandCount || ph == cmk::kPBandScatter)) continue;
            // a stalled window (test hook) has no prep items: its later phases wait until their bound
            if (w == stall_window && ph == cmk::kPPrep) {
                ++rank;
                continue;
            }
            int count = 0;
            switch (ph) {
            case cmk::kPPrep: count = d.pix_tiles; break;
            case cmk::kPBandCount:
            case cmk::kPBandScatter: count = nsc; break;
            case cmk::kPSplat:
            case cmk::kPAdjoint: count = chunks; break;
            default: count = d.loss_tiles; break;
            }
            if (count > 0) keys.push_back({(long long)w * stagger + rank, w, ph, count});
            ++rank;
        }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
        return a.key != b.key ? a.key < b.key : a.w < b.w;
    });
    int start = 0;
    for (size_t i = 0; i < keys.size(); ++i) {
        seg[i] = cmk::PSeg{keys[i].w, keys[i].phase, start, keys[i].count};
        start += keys[i].count;
    }
    h->p_nseg = (int)keys.size();
    h->p_total = start;
}

// Image and quad slabs shared along a chain: the groups of one chain run one
// after another, so the windows at the same position of its groups can use
// one slab (the next group's prep pass zeroes it after the previous group's
// gradient pass has read it).  Fewer slabs in flight keep the images in L2
// between the passes, and no window's images need to reach DRAM once another
// reuses them.  With group 0 every window is in flight: no sharing.
// slot[i]: the slab of window i; slab offsets of the images and quads.
struct Slabs {
    std::vector<int> slot;
    std::vector<size_t> iwe_off, quad_off;
};

Slabs share_slabs(const cm_batch* b, const cm_window* wins, int32_t nwin, int R)
{
    Slabs sl;
    sl.slot.assign(nwin, -1);
    std::vector<size_t> iwe_sz, quad_sz;
    if (b->sched.group > 0) {
        std::vector<std::vector<int>> chain_slots(kMaxChains);
        for (const Group& g : make_groups(b)) {
            std::vector<int>& cs = chain_slots[g.chain];
            for (int i = g.w0; i < g.w1; ++i) {
                if (wins[i].scratch) continue;
                const int p = i - g.w0;
                while ((int)cs.size() <= p) {
                    cs.push_back((int)iwe_sz.size());
                    iwe_sz.push_back(0);
                    quad_sz.push_back(0);
                }
                const int k = cs[p];
                const size_t HW = (size_t)wins[i].cam.width * wins[i].cam.height;
                iwe_sz[k] = std::max(iwe_sz[k], up256((size_t)R * HW * sizeof(float4)));
                quad_sz[k] = std::max(quad_sz[k], 2 * HW * sizeof(cmk::FQ));
                sl.slot[i] = k;
            }
        }
    } else {
        for (int i = 0; i < nwin; ++i) {
            if (wins[i].scratch) continue;
            const size_t HW = (size_t)wins[i].cam.width * wins[i].cam.height;
            sl.slot[i] = (int)iwe_sz.size();
            iwe_sz.push_back(up256((size_t)R * HW * sizeof(float4)));
            quad_sz.push_back(2 * HW * sizeof(cmk::FQ));
        }
    }
    size_t oi = 0, oq = 0;
    for (size_t k = 0; k < iwe_sz.size(); ++k) {
        sl.iwe_off.push_back(oi);
        sl.quad_off.push_back(oq);
        oi += iwe_sz[k];
        oq += quad_sz[k];
    }
    return sl;
}

int stage_windows(cm_batch* b, const cm_window* wins, int32_t nwin)
{
    if (nwin < 1 || nwin > b->cap) return CM_EINVAL;
    for (int i = 0; i < nwin; ++i)
        if (!window_ok(wins[i])) return CM_EINVAL;
    const Need n = need_of(wins, nwin, b->cfg);
    const Need& c = b->capn;
    if (n.iwe > c.iwe || n.dflow > c.dflow || n.quad > c.quad || n.part > c.part ||
        n.stat > c.stat || n.dego > c.dego || n.warp > c.warp)
        return CM_ENOMEM;
    const bool sorted = b->cfg.splat == CM_SPLAT_SORT;
    if (sorted) {
        // the deterministic mode: the plan's own buffers only, sort buffers for its largest window
        for (int i = 0; i < nwin; ++i)
            if (wins[i].scratch) return CM_EINVAL;
        if (n.sort.entries > c.sort.entries || n.sort.hist > c.sort.hist || n.sort.part > c.sort.part ||
            n.sort.start > c.sort.start)
            return CM_ENOMEM;
    }
    // the previous upload must have left the staging buffer before it is rewritten
    if (cudaEventSynchronize(b->staged) != cudaSuccess) return CM_ECUDA;
    unsigned char* s = b->staging;
    std::memset(s, 0, b->L.table_end);
    BatchHdr* h = reinterpret_cast<BatchHdr*>(s + b->L.hdr);
    Win* tab = reinterpret_cast<Win*>(s + b->L.tab);
    long long* cs = reinterpret_cast<long long*>(s + b->L.cstart);
    long long* ss = reinterpret_cast<long long*>(s + b->L.sstart);
    long long supers = 0;
    int* ls = reinterpret_cast<int*>(s + b->L.lstart);
    int* ps = reinterpret_cast<int*>(s + b->L.pstart);

    const int R = refs_of(b->cfg);
    const float eps = b->cfg.eps > 0.0f ? b->cfg.eps : 1e-9f;
    size_t o_warp = 0, o_dflow = 0, o_part = 0, o_stat = 0, o_dego = 0, o_bins = 0;
    long long chunks = 0;
    int lt_total = 0, pt_total = 0;
    char* base = b->base;
    // the per-window work counts first: the groups (and so the shared slabs) depend on them
    b->nwin = nwin;
    b->chunks.assign(nwin, 0);
    b->ltiles.assign(nwin, 0);
    b->ptiles.assign(nwin, 0);
    for (int i = 0; i < nwin; ++i) {
        const size_t HW = (size_t)wins[i].cam.width * wins[i].cam.height;
        b->chunks[i] = (wins[i].ev.n + cmk::kEventThreads - 1) / cmk::kEventThreads;
        b->ltiles[i] = loss_tiles_for(HW);
        b->ptiles[i] = pix_tiles_for(HW);
    }
    const Slabs slabs = share_slabs(b, wins, nwin, R);
    b->chunks.assign(nwin, 0);
    b->ltiles.assign(nwin, 0);
    b->ptiles.assign(nwin, 0);
    b->stat_lr.assign(nwin, nullptr);
    b->stat_nnz.assign(nwin, nullptr);
    for (int i = 0; i < nwin; ++i) {
        const cm_window& w = wins[i];
        const size_t HW = (size_t)w.cam.width * w.cam.height;
        Win& d = tab[i];
        d.x = w.ev.x;
        d.y = w.ev.y;
        d.t = w.ev.t;
        d.p = w.ev.p;
        d.n = w.ev.n;
        d.W = w.cam.width;
        d.H = w.cam.height;
        d.B = b->cfg.nbins;
        d.R = R;
        d.ref_mode = b->cfg.ref_mode;
        d.nfb = 1;
        d.t0 = w.ev.t0;
        d.span = w.ev.t1 - w.ev.t0;
        d.eps = eps;
        d.iwe_split = 1;  // polarity planes: row pairs of corners take one 16-byte reduction / gather
        d.dt = w.dt_window;
        d.fx = w.cam.fx;
        d.fy = w.cam.fy;
        d.cx = w.cam.cx;
        d.cy = w.cam.cy;
        d.loss_tiles = loss_tiles_for(HW);
        d.pix_tiles = pix_tiles_for(HW);
        if (w.scratch) {
            // every per-window buffer in the window's own scratch
            char* sc = static_cast<char*>(w.scratch);
            const WinScratch ws = win_scratch(HW, R);
            d.iwe = reinterpret_cast<float4*>(sc + ws.iwe);
            d.flow = reinterpret_cast<const float2*>(w.flow);  // nullptr for depth input (the quads hold its flow)
            // dL/dflow of a depth window is stored only where the caller asks for it
            d.dflow = w.dflow ? reinterpret_cast<float2*>(w.dflow)
                              : (w.flow ? reinterpret_cast<float2*>(sc + ws.dflow) : nullptr);
            d.fq = reinterpret_cast<const cmk::FQ*>(sc + ws.fq);
            d.dq = reinterpret_cast<cmk::FQ*>(sc + ws.dq);
            d.loss_part = reinterpret_cast<float2*>(sc + ws.part);
            d.norm = reinterpret_cast<float*>(sc + ws.norm);
            d.loss_r = reinterpret_cast<float*>(sc + ws.lr);
            d.nnz_r = reinterpret_cast<int32_t*>(sc + ws.nnz);
            d.dego_part = reinterpret_cast<float*>(sc + ws.dego);
            d.sync = reinterpret_cast<int32_t*>(sc + ws.sync);
        } else {
            d.iwe = reinterpret_cast<float4*>(base + b->L.iwe + slabs.iwe_off[slabs.slot[i]]);
            d.flow = reinterpret_cast<const float2*>(w.flow);  // nullptr for depth input (the quads hold its flow)
            if (w.dflow) {
                d.dflow = reinterpret_cast<float2*>(w.dflow);
            } else if (w.flow) {
                d.dflow = reinterpret_cast<float2*>(base + b->L.dflow + o_dflow);
                o_dflow += HW * sizeof(float2);
            } else {
                d.dflow = nullptr;  // dL/dflow of a depth window is stored only where the caller asks for it
            }
            if (b->cfg.store_warps && d.n > 0) {
                d.warp = reinterpret_cast<float2*>(base + b->L.warp + o_warp);
                o_warp += up256((size_t)(d.B + 1) * d.n * sizeof(float2));
            }
            d.fq = reinterpret_cast<const cmk::FQ*>(base + b->L.quad + slabs.quad_off[slabs.slot[i]]);
            d.dq = reinterpret_cast<cmk::FQ*>(base + b->L.quad + slabs.quad_off[slabs.slot[i]] + HW * sizeof(cmk::FQ));
            d.loss_part = reinterpret_cast<float2*>(base + b->L.part + o_part);
            o_part += (size_t)R * d.loss_tiles * sizeof(float2);
            d.norm = reinterpret_cast<float*>(base + b->L.norm) + o_stat;
            d.loss_r = reinterpret_cast<float*>(base + b->L.lr) + o_stat;
            d.nnz_r = reinterpret_cast<int32_t*>(base + b->L.nnz) + o_stat;
            o_stat += R;
            d.dego_part = reinterpret_cast<float*>(base + b->L.dego + o_dego);
            o_dego += (size_t)d.loss_tiles * 6 * sizeof(float);
            d.sync = reinterpret_cast<int32_t*>(base + b->L.sync) + kSyncInts * i;
        }
        // the grouping's counter is the plan's (zeroed at creation) also for a window with its own scratch
        d.gsync = reinterpret_cast<int32_t*>(base + b->L.sync) + kSyncInts * i + 2;
        // events grouped by 32x32 tile (bin 1) or by 32-row band in their given
        // order (bin 2), while the plan's grouping memory lasts
        const size_t bb = bin_bytes(d.W, d.H, d.n);
        const bool bands = b->sched.bin == 2;
        const int tp = b->sched.bin == 3 ? cmk::kSmemTile : cmk::kBinTile;
        const int tx = bands ? 1 : (d.W + tp - 1) / tp;
        const int ty = bands ? (d.H + cmk::kBandRows - 1) / cmk::kBandRows : (d.H + tp - 1) / tp;
        const bool fits = bands ? ty <= cmk::kMaxBands : tx * ty <= cmk::kMaxBinTiles;
        if (b->sched.bin && d.n > 0 && fits && o_bins + bb <= b->capn.bins) {
            char* q = base + b->L.bins + o_bins;
            o_bins += bb;
            d.ntx = tx;
            d.nty = ty;
            d.band_rows = bands ? cmk::kBandRows : 0;
            d.smem_tiles = b->sched.bin == 3 ? 1 : 0;
            d.tile_px = tp;
            const size_t nt = (size_t)d.ntx * d.nty;
            d.tile_cnt = reinterpret_cast<int32_t*>(q);
            d.tile_cur = bands ? nullptr : d.tile_cnt + nt + 1;
            const size_t nband = (size_t)ty * ((d.n + cmk::kSuperChunk - 1) / cmk::kSuperChunk);
            const size_t table = 3 * nt + 2 > nband ? 3 * nt + 2 : nband;
            d.item_start = bands ? nullptr : d.tile_cnt + 2 * nt + 1;
            q += up256(table * sizeof(int32_t));
            d.rx = reinterpret_cast<int16_t*>(q);
            q += up256(2 * (size_t)d.n);
            d.ry = reinterpret_cast<int16_t*>(q);
            q += up256(2 * (size_t)d.n);
            d.rt = reinterpret_cast<float*>(q);
            q += up256(4 * (size_t)d.n);
            d.rp = reinterpret_cast<int8_t*>(q);
        }
        if (!w.flow) {
            d.rho = w.inv_depth;
            d.ego = w.ego6;
            d.drho = w.dinv_depth;
            d.dego = w.dego6;
        }
        if (sorted) {
            // the single-window layout for the sort path: [R][H][W] float4 images in the
            // image slab; for depth input the flow in the quad slab's first half and
            // dL/dflow (unless the caller takes it) in its second half
            float2* qa = reinterpret_cast<float2*>(const_cast<cmk::FQ*>(d.fq));
            float2* qb = reinterpret_cast<float2*>(d.dq);
            d.iwe_split = 0;
            d.fq = nullptr;
            d.dq = nullptr;
            d.tile_cnt = nullptr;
            if (!w.flow) {
                d.flow = qa;
                if (!d.dflow) d.dflow = qb;
            }
            d.pix_tiles = d.loss_tiles;  // the gradient pass's partials use the loss tiles' slab
        }
        b->stat_lr[i] = d.loss_r;
        b->stat_nnz[i] = d.nnz_r;
        d.loss = w.loss_out;
        d.dloss = w.dloss;
        cs[i] = chunks;
        ss[i] = supers;
        supers += (w.ev.n + cmk::kSuperChunk - 1) / cmk::kSuperChunk;
        ls[i] = lt_total;
        ps[i] = pt_total;

        b->chunks[i] = (w.ev.n + cmk::kEventThreads - 1) / cmk::kEventThreads;
        b->ltiles[i] = d.loss_tiles;
        b->ptiles[i] = d.pix_tiles;
        chunks += b->chunks[i];
        lt_total += b->ltiles[i];
        pt_total += b->ptiles[i];
    }
    cs[nwin] = chunks;
    ss[nwin] = supers;
    ls[nwin] = lt_total;
    ps[nwin] = pt_total;

    h->nwin = nwin;
    h->total_chunks = chunks;
    h->total_ltiles = lt_total;
    h->total_ptiles = pt_total;
    if (b->sched.persist > 0)
        build_queue(b->sched.persist - 1, tab, nwin, b->stall_window, reinterpret_cast<cmk::PSeg*>(s + b->L.pseg), h);
    b->nwin = nwin;
    if (b->last.data() != wins) b->last.assign(wins, wins + nwin);
    b->dirty = true;
    if (b->sched.group > 0) b->stale = true;  // the graph's window groups depend on the windows
    // (the persistent step reads its queue's size from the uploaded header: its graph stays valid)
    return CM_OK;
}

// Window groups and their chains.  group <= 0: one group over every slot of the
// table on one chain (the kernels clamp to the windows in use, so the graph
// stays valid when the windows change).  Otherwise consecutive groups of
// `group` windows, each assigned to the chain with the least work so far.
std::vector<Group> make_groups(const cm_batch* b)
{
    std::vector<Group> g;
    if (b->sched.group <= 0) {
        long long c = 0;
        int lt = 0, pt = 0;
        for (int i = 0; i < b->nwin; ++i) {
            c += b->chunks[i];
            lt += b->ltiles[i];
            pt += b->ptiles[i];
        }
        g.push_back({0, b->cap, 0, c, lt, pt});
        return g;
    }
    const int chains = b->sched.chains < 1 ? 1 : (b->sched.chains > kMaxChains ? kMaxChains : b->sched.chains);
    std::vector<double> load(chains, 0.0);
    for (int w = 0; w < b->nwin; w += b->sched.group) {
        Group x{w, w + b->sched.group < b->nwin ? w + b->sched.group : b->nwin, 0, 0, 0, 0};
        double work = 0.0;
        for (int i = x.w0; i < x.w1; ++i) {
            x.chunks += b->chunks[i];
            x.ltiles += b->ltiles[i];
            x.ptiles += b->ptiles[i];
            work += (double)b->chunks[i] + 0.5 * refs_of(b->cfg) * b->ltiles[i];
        }
        int best = 0;
        for (int c = 1; c < chains; ++c)
            if (load[c] < load[best]) best = c;
        x.chain = best;
        load[best] += work;
        g.push_back(x);
    }
    return g;
}

template <int MAXB>
void enqueue_event_kernel(cm_batch* b, cudaStream_t s, int which, int grid, int w0, int w1)
{
    const BatchHdr* h = reinterpret_cast<const BatchHdr*>(b->base + b->L.hdr);
    const Win* tab = reinterpret_cast<const Win*>(b->base + b->L.tab);
    const long long* cs = reinterpret_cast<const long long*>(b->base + b->L.cstart);
    if (which == 0)
        cmk::k_splat_batch<MAXB><<<grid, cmk::kEventThreads, 0, s>>>(h, tab, cs, w0, w1);
    else
        cmk::k_adjoint_batch<MAXB><<<grid, cmk::kEventThreads, 0, s>>>(h, tab, cs, w0, w1);
}

template <int MAXB>
void enqueue_tiles_kernel(cm_batch* b, cudaStream_t s, int which, int grid, int w0, int w1)
{
    const BatchHdr* h = reinterpret_cast<const BatchHdr*>(b->base + b->L.hdr);
    const Win* tab = reinterpret_cast<const Win*>(b->base + b->L.tab);
    if (which == 0)
        cmk::k_splat_tiles_batch<MAXB><<<grid, cmk::kTileThreads, tiles_smem(b->cfg, 0), s>>>(h, tab, w0, w1);
    else
        cmk::k_adjoint_tiles_batch<MAXB><<<grid, cmk::kTileThreads, tiles_smem(b->cfg, 1), s>>>(h, tab, w0, w1);
}

void enqueue_tiles(cm_batch* b, cudaStream_t s, int which, int grid, int w0, int w1)
{
    const int B = b->cfg.nbins;
    if (B <= 1) enqueue_tiles_kernel<1>(b, s, which, grid, w0, w1);
    else if (B <= 10) enqueue_tiles_kernel<10>(b, s, which, grid, w0, w1);
    else if (B <= 20) enqueue_tiles_kernel<20>(b, s, which, grid, w0, w1);
    else enqueue_tiles_kernel<32>(b, s, which, grid, w0, w1);
}

template <int MAXB>
void enqueue_persistent_kernel(cm_batch* b, cudaStream_t s)
{
    const BatchHdr* h = reinterpret_cast<const BatchHdr*>(b->base + b->L.hdr);
    const Win* tab = reinterpret_cast<const Win*>(b->base + b->L.tab);
    const cmk::PSeg* seg = reinterpret_cast<const cmk::PSeg*>(b->base + b->L.pseg);
    int* q = reinterpret_cast<int*>(b->base + b->L.pq);
    cmk::k_step_persistent<MAXB><<<b->grid_persist, cmk::kEventThreads, 0, s>>>(h, tab, seg, q, q + 2);
}

void enqueue_persistent(cm_batch* b, cudaStream_t s)
{
    const int B = b->cfg.nbins;
    if (B <= 1) enqueue_persistent_kernel<1>(b, s);
    else if (B <= 10) enqueue_persistent_kernel<10>(b, s);
    else if (B <= 20) enqueue_persistent_kernel<20>(b, s);
    else enqueue_persistent_kernel<32>(b, s);
}

void enqueue_event(cm_batch* b, cudaStream_t s, int which, int grid, int w0, int w1)
{
    const int B = b->cfg.nbins;
    if (B <= 1) enqueue_event_kernel<1>(b, s, which, grid, w0, w1);
    else if (B <= 10) enqueue_event_kernel<10>(b, s, which, grid, w0, w1);
    else if (B <= 20) enqueue_event_kernel<20>(b, s, which, grid, w0, w1);
    else enqueue_event_kernel<32>(b, s, which, grid, w0, w1);
}

void release_graph(cm_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    for (ProfNode& p : b->prof) {
        cudaEventDestroy(p.ea);
        cudaEventDestroy(p.eb);
    }
    b->prof.clear();
    b->swapped = false;
}

int clampi(long long v, int lo, int hi) { return (int)(v < lo ? lo : (v > hi ? hi : v)); }

// Capture the five phases of every group on its chain's stream, each kernel
// bracketed by event-record nodes (used for per-kernel timing).
int capture(cm_batch* b)
{
    release_graph(b);
    const std::vector<Group> groups = make_groups(b);
    int chains = 1;
    for (const Group& g : groups) chains = g.chain + 1 > chains ? g.chain + 1 : chains;
    for (int c = 0; c < chains; ++c)
        if (!b->streams[c] && cudaStreamCreateWithFlags(&b->streams[c], cudaStreamNonBlocking) != cudaSuccess)
            return CM_ECUDA;
    if (!b->fork && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return CM_ECUDA;
    for (int c = 0; c < chains; ++c)
        if (!b->join[c] && cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming) != cudaSuccess)
            return CM_ECUDA;
    const BatchHdr* h = reinterpret_cast<const BatchHdr*>(b->base + b->L.hdr);
    const Win* tab = reinterpret_cast<const Win*>(b->base + b->L.tab);
    const int* ls = reinterpret_cast<const int*>(b->base + b->L.lstart);
    const int* ps = reinterpret_cast<const int*>(b->base + b->L.pstart);
    const long long* ss = reinterpret_cast<const long long*>(b->base + b->L.sstart);
    cudaStream_t s0 = b->streams[0];
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CM_ECUDA;
    bool ok = true;
    if (chains > 1) {
        ok = ok && cudaEventRecord(b->fork, s0) == cudaSuccess;
        for (int c = 1; c < chains; ++c) ok = ok && cudaStreamWaitEvent(b->streams[c], b->fork, 0) == cudaSuccess;
    }
    const bool wide = b->sched.group <= 0;
    if (b->sched.persist > 0) {
        // the persistent step: zero the queue and the counters, then one kernel
        ProfNode p{kPersistentPhase, nullptr, nullptr, nullptr, nullptr};
        ok = cudaEventCreate(&p.ea) == cudaSuccess && cudaEventCreate(&p.eb) == cudaSuccess;
        if (ok) {
            b->prof.push_back(p);
            ok = cudaMemsetAsync(b->base + b->L.pq, 0, pq_bytes(b->cap), s0) == cudaSuccess;
            cudaEventRecordWithFlags(p.ea, s0, cudaEventRecordExternal);
            enqueue_persistent(b, s0);
            cudaEventRecordWithFlags(p.eb, s0, cudaEventRecordExternal);
        }
    }
    const bool sorted = b->cfg.splat == CM_SPLAT_SORT;
    if (sorted) {
        // the deterministic mode: the windows one after another through the
        // single-window sort path (every sum in a fixed order), on one stream
        const Win* ht = reinterpret_cast<const Win*>(b->staging + b->L.tab);
        const int sms = cmk::sm_count_current();
        for (const Group& g : groups) {  // one window per group, the groups spread over the chains
            if (!ok) break;
            cudaStream_t s = b->streams[g.chain];
            char* o = b->base + (size_t)g.chain * b->L.sort_stride;
            cmk::SortBufs sb{reinterpret_cast<uint32_t*>(o + b->L.ska), reinterpret_cast<uint32_t*>(o + b->L.skb),
                             reinterpret_cast<uint32_t*>(o + b->L.sva), reinterpret_cast<uint32_t*>(o + b->L.svb),
                             reinterpret_cast<float4*>(o + b->L.spay), reinterpret_cast<uint32_t*>(o + b->L.shist),
                             reinterpret_cast<uint32_t*>(o + b->L.spart),
                             reinterpret_cast<uint32_t*>(o + b->L.sstart_keys)};
            for (int i = g.w0; i < g.w1 && ok; ++i) {
                const Win& d = ht[i];
                if (d.rho) ok = cmk::launch_flow(d, s) == cudaSuccess;
                ok = ok && cmk::sort_splat(d, sb, sms, s) == cudaSuccess;
                ok = ok && cmk::launch_loss(d, s) == cudaSuccess;
                ok = ok && cmk::sort_adjoint(d, sb, sms, s) == cudaSuccess;
                if (d.rho && (d.drho || d.dego)) ok = ok && cmk::launch_depth_ego(d, s) == cudaSuccess;
            }
        }
    }
    for (const Group& g : groups) {
        if (b->sched.persist > 0 || sorted) break;
        cudaStream_t s = b->streams[g.chain];
        for (int pi = 0; pi < kPhases && ok; ++pi) {
            const int ph = kPhaseOrder[pi];
            if (!b->sched.bin && (ph == 1 || ph == 2)) continue;  // no grouping kernels
            if (b->sched.bin == 2 && ph == 1) continue;             // the band count runs inside the prep pass
            if (b->sched.bin != 3 && (ph == 7 || ph == 8)) continue;  // shared-memory tiles with bin 3 only
            ProfNode p{ph, nullptr, nullptr, nullptr, nullptr};
            ok = cudaEventCreate(&p.ea) == cudaSuccess && cudaEventCreate(&p.eb) == cudaSuccess;
            if (!ok) break;
            b->prof.push_back(p);
            cudaEventRecordWithFlags(p.ea, s, cudaEventRecordExternal);
            const int gt = wide ? b->grid_tiles : clampi(g.ptiles, 1, b->grid_tiles);
            const int gl = wide ? b->grid_tiles : clampi(g.ltiles, 1, b->grid_tiles);
            const int ge = wide ? b->grid_events : clampi(g.chunks, 1, b->grid_events);
            // super-chunks of the group: at most chunks / 16 rounded up per window
            const int gs = wide ? b->grid_events
                                : clampi(g.chunks / (cmk::kSuperChunk / cmk::kEventThreads) + (g.w1 - g.w0), 1,
                                         b->grid_events);
            switch (ph) {
            case 0: cmk::k_prep_batch<<<gt, cmk::kEventThreads, 0, s>>>(h, tab, ps, ss, b->sched.bin == 2, g.w0, g.w1); break;
            case 1: cmk::k_bin_count_batch<<<gs, cmk::kEventThreads, 0, s>>>(h, tab, ss, g.w0, g.w1); break;
            case 2: cmk::k_bin_scatter_batch<<<gs, cmk::kEventThreads, 0, s>>>(h, tab, ss, g.w0, g.w1); break;
            case 3: enqueue_event(b, s, 0, wide ? b->grid_splat : clampi(g.chunks, 1, b->grid_splat), g.w0, g.w1); break;
            case 4: cmk::k_loss_batch<<<gl, 256, 0, s>>>(h, tab, ls, g.w0, g.w1); break;
            case 5: enqueue_event(b, s, 1, ge, g.w0, g.w1); break;
            case 6: cmk::k_grad_batch<<<gl, 256, 0, s>>>(h, tab, ls, g.w0, g.w1); break;
            case 7: enqueue_tiles(b, s, 0, b->grid_tiles_smem, g.w0, g.w1); break;
            case 8: enqueue_tiles(b, s, 1, b->grid_tiles_smem, g.w0, g.w1); break;
            }
            cudaEventRecordWithFlags(p.eb, s, cudaEventRecordExternal);
        }
    }
    for (int c = 1; c < chains && ok; ++c) {
        ok = cudaEventRecord(b->join[c], b->streams[c]) == cudaSuccess;
        ok = ok && cudaStreamWaitEvent(s0, b->join[c], 0) == cudaSuccess;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s0, &g);
    if (!ok || e != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        return CM_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return CM_ECUDA;
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        cudaGraphEventRecordNodeGetEvent(n, &ev);
        for (ProfNode& p : b->prof) {
            if (ev == p.ea) p.na = n;
            if (ev == p.eb) p.nb = n;
        }
    }
    for (const ProfNode& p : b->prof)
        if (!p.na || !p.nb) return CM_ECUDA;
    b->graph_kernels = 0;
    for (cudaGraphNode_t n : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++b->graph_kernels;
    }
    b->stale = false;
    return CM_OK;
}

void destroy_batch(cm_batch* b)
{
    if (!b) return;
    release_graph(b);
    for (int c = 0; c < kMaxChains; ++c) {
        if (b->streams[c]) cudaStreamDestroy(b->streams[c]);
        if (b->join[c]) cudaEventDestroy(b->join[c]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->staged) {
        cudaEventSynchronize(b->staged);
        cudaEventDestroy(b->staged);
    }
    if (b->staging) cudaFreeHost(b->staging);
    delete b;
}

// the tile kernels take more than the default 48 KB of dynamic shared memory
template <int MAXB>
bool allow_tiles_smem(const cm_loss_cfg& cfg)
{
    return cudaFuncSetAttribute(cmk::k_splat_tiles_batch<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tiles_smem(cfg, 0)) == cudaSuccess &&
           cudaFuncSetAttribute(cmk::k_adjoint_tiles_batch<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)tiles_smem(cfg, 1)) == cudaSuccess;
}

template <int MAXB>
int occupancy_persistent()
{
    int a = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cmk::k_step_persistent<MAXB>, cmk::kEventThreads, 0);
    return a < 1 ? 1 : a;
}

template <int MAXB>
int occupancy_blocks()
{
    int a = 0, c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cmk::k_splat_batch<MAXB>, cmk::kEventThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, cmk::k_adjoint_batch<MAXB>, cmk::kEventThreads, 0);
    const int m = a < c ? a : c;
    return m < 1 ? 1 : m;
}

int run_plan(cm_batch* b, cudaStream_t s)
{
    if (b->dirty) {
        if (cudaMemcpyAsync(b->base, b->staging, b->L.table_end, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return CM_ECUDA;
        if (cudaEventRecord(b->staged, s) != cudaSuccess) return CM_ECUDA;
        b->dirty = false;
    }
    if (b->stale || !b->exec) {
        const int st = capture(b);
        if (st) return st;
    }
    // per-kernel timing: point the event-record nodes at fresh events from the
    // profiler's pool for this replay; otherwise back at the plan's own events
    const bool prof = cmk::profiling_on();
    std::vector<cudaEvent_t> ev;
    if (prof) {
        ev.resize(2 * b->prof.size());
        for (size_t i = 0; i < b->prof.size(); ++i) {
            ev[2 * i] = cmk::profile_take_event();
            ev[2 * i + 1] = cmk::profile_take_event();
            if (!ev[2 * i] || !ev[2 * i + 1] ||
                cudaGraphExecEventRecordNodeSetEvent(b->exec, b->prof[i].na, ev[2 * i]) != cudaSuccess ||
                cudaGraphExecEventRecordNodeSetEvent(b->exec, b->prof[i].nb, ev[2 * i + 1]) != cudaSuccess)
                return CM_ECUDA;
        }
        b->swapped = true;
    } else if (b->swapped) {
        for (const ProfNode& p : b->prof)
            if (cudaGraphExecEventRecordNodeSetEvent(b->exec, p.na, p.ea) != cudaSuccess ||
                cudaGraphExecEventRecordNodeSetEvent(b->exec, p.nb, p.eb) != cudaSuccess)
                return CM_ECUDA;
        b->swapped = false;
    }
    if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return CM_ECUDA;
    cmk::count_launches(b->graph_kernels);
    if (prof)
        for (size_t i = 0; i < b->prof.size(); ++i)
            cmk::profile_push(kPhaseName[b->prof[i].phase], ev[2 * i], ev[2 * i + 1]);
    return CM_OK;
}

// autotuner cache: (window count, first window's size, references, events
// bucket) -> schedule, for the life of the process
struct TuneKey {
    int nwin, W, H, R, ebucket, sorted;
};
std::vector<std::pair<TuneKey, cm_batch_schedule>> g_tuned;

TuneKey key_of(const cm_batch* b)
{
    long long c = 0;
    for (long long v : b->chunks) c += v;
    int e = 0;
    while ((1LL << e) < c + 1) ++e;
    const Win* tab = reinterpret_cast<const Win*>(b->staging + b->L.tab);
    return {b->nwin, tab[0].W, tab[0].H, refs_of(b->cfg), e, b->cfg.splat == CM_SPLAT_SORT ? 1 : 0};
}

}  // namespace

extern "C" {

int cm_window_scratch_query(const cm_camera* cam, const cm_loss_cfg* cfg, size_t* bytes)
{
    if (!cam || !bytes || !cfg_ok(cfg) || cam->width < 2 || cam->height < 2 || cam->width > 32767 ||
        cam->height > 32767)
        return CM_EINVAL;
    *bytes = win_scratch((size_t)cam->width * cam->height, refs_of(*cfg)).total;
    return CM_OK;
}

int cm_batch_query(const cm_window* wins, int32_t nwin, const cm_loss_cfg* cfg, size_t* bytes)
{
    if (!wins || nwin < 1 || !bytes || !cfg_ok(cfg)) return CM_EINVAL;
    for (int i = 0; i < nwin; ++i)
        if (!window_ok(wins[i])) return CM_EINVAL;
    *bytes = layout_of(nwin, need_of(wins, nwin, *cfg)).total;
    return CM_OK;
}

int cm_batch_create(void* dev_mem, size_t bytes, const cm_window* wins, int32_t nwin, const cm_loss_cfg* cfg,
                    cm_batch** out)
{
    if (!dev_mem || !wins || nwin < 1 || !out || !cfg_ok(cfg)) return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(dev_mem) % 256) return CM_EINVAL;
    for (int i = 0; i < nwin; ++i)
        if (!window_ok(wins[i])) return CM_EINVAL;
    const Need n = need_of(wins, nwin, *cfg);
    const Layout L = layout_of(nwin, n);
    if (bytes < L.total) return CM_ENOMEM;
    cm_batch* b = new (std::nothrow) cm_batch;
    if (!b) return CM_ENOMEM;
    b->base = static_cast<char*>(dev_mem);
    b->bytes = bytes;
    b->cfg = *cfg;
    b->cap = nwin;
    b->capn = n;
    b->L = L;
    b->sched = nwin > 1 ? cm_batch_schedule{2, 1, 0} : cm_batch_schedule{1, 0, 0};
    if (cfg->splat == CM_SPLAT_TILES) b->sched.bin = 3;  // the shared-memory tile strategy
    if (cfg->splat == CM_SPLAT_SORT)  // deterministic: one window at a time on each chain
        b->sched = cm_batch_schedule{nwin < kSortChains ? nwin : kSortChains, 1, 0, 0};
    int st = CM_OK;
    if (cudaMallocHost(reinterpret_cast<void**>(&b->staging), L.table_end) != cudaSuccess) st = CM_ENOMEM;
    if (!st && cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming) != cudaSuccess) st = CM_ECUDA;
    if (!st) {
        const int sms = cmk::sm_count_current();
        int occ = 1;
        const int B = cfg->nbins;
        if (B <= 1) occ = occupancy_blocks<1>();
        else if (B <= 10) occ = occupancy_blocks<10>();
        else if (B <= 20) occ = occupancy_blocks<20>();
        else occ = occupancy_blocks<32>();
        b->grid_events = sms * occ;
        b->grid_splat = sms * 8;
        b->grid_tiles = sms * 4;
        b->grid_tiles_smem = sms;  // one tile block (512 threads, up to 192 KB) per SM
        int occp = 1;
        if (B <= 1) occp = occupancy_persistent<1>();
        else if (B <= 10) occp = occupancy_persistent<10>();
        else if (B <= 20) occp = occupancy_persistent<20>();
        else occp = occupancy_persistent<32>();
        b->grid_persist = sms * occp;
        bool tiles_ok = false;
        if (B <= 1) tiles_ok = allow_tiles_smem<1>(*cfg);
        else if (B <= 10) tiles_ok = allow_tiles_smem<10>(*cfg);
        else if (B <= 20) tiles_ok = allow_tiles_smem<20>(*cfg);
        else tiles_ok = allow_tiles_smem<32>(*cfg);
        if (!tiles_ok) st = CM_ECUDA;
        if (!st) st = stage_windows(b, wins, nwin);
    }
    // the completion counters start at zero (the prep kernel also resets them)
    if (!st && cudaMemset(b->base + L.sync, 0, (size_t)nwin * kSyncInts * sizeof(int32_t)) != cudaSuccess)
        st = CM_ECUDA;
    if (!st && cudaMemset(b->base + L.pq, 0, pq_bytes(nwin)) != cudaSuccess) st = CM_ECUDA;
    if (st) {
        destroy_batch(b);
        return st;
    }
    *out = b;
    return CM_OK;
}

int cm_batch_set_windows(cm_batch* b, const cm_window* wins, int32_t nwin)
{
    if (!b || !wins) return CM_EINVAL;
    return stage_windows(b, wins, nwin);
}

namespace {
// take schedule `s` and re-stage the current windows: the binning buffers and
// the slabs shared along a chain are assigned per window when the table is filled
int apply_schedule(cm_batch* b, const cm_batch_schedule& s)
{
    b->sched = s;
    b->stale = true;
    if (b->nwin > 0) {
        const std::vector<cm_window> w = b->last;
        return stage_windows(b, w.data(), (int32_t)w.size());
    }
    return CM_OK;
}
}  // namespace

int cm_batch_set_schedule(cm_batch* b, const cm_batch_schedule* s)
{
    if (!b || !s || s->chains < 1 || s->chains > kMaxChains || s->group < 0) return CM_EINVAL;
    if (s->group == 0 && s->chains != 1) return CM_EINVAL;
    if (s->bin < 0 || s->bin > 3) return CM_EINVAL;
    if (s->persist < 0 || s->persist > kMaxPersist) return CM_EINVAL;
    // the persistent step: one kernel over every window, events in their order or grouped by band
    if (s->persist > 0 && (s->chains != 1 || s->group != 0 || (s->bin != 0 && s->bin != 2))) return CM_EINVAL;
    // the deterministic mode runs one window at a time on each of up to kSortChains chains
    if (b->cfg.splat == CM_SPLAT_SORT && (s->chains > kSortChains || s->group != 1 || s->bin != 0 || s->persist != 0))
        return CM_EINVAL;
    return apply_schedule(b, *s);
}

int cm_batch_get_schedule(const cm_batch* b, cm_batch_schedule* s)
{
    if (!b || !s) return CM_EINVAL;
    *s = b->sched;
    return CM_OK;
}

int cm_batch_run(cm_batch* b, void* stream)
{
    if (!b) return CM_EINVAL;
    return run_plan(b, reinterpret_cast<cudaStream_t>(stream));
}

int cm_batch_autotune(cm_batch* b, void* stream, cm_batch_schedule* chosen)
{
    if (!b) return CM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const TuneKey k = key_of(b);
    for (const auto& e : g_tuned) {
        const TuneKey& q = e.first;
        if (q.nwin == k.nwin && q.W == k.W && q.H == k.H && q.R == k.R && q.ebucket == k.ebucket &&
            q.sorted == k.sorted) {
            const int st = apply_schedule(b, e.second);
            if (chosen) *chosen = b->sched;
            return st;
        }
    }
    std::vector<cm_batch_schedule> cand;
    if (k.sorted) {  // the deterministic mode: 1..kSortChains chains of one window at a time
        for (int c = 1; c <= kSortChains && c <= b->nwin; ++c) cand.push_back(cm_batch_schedule{c, 1, 0, 0});
    } else {
        for (int bin = 0; bin < 4; ++bin)
            for (const auto& cg : {std::pair<int, int>{1, 0}, {1, 1}, {2, 1}, {3, 1}, {4, 1}, {2, 2}, {4, 2}, {6, 1},
                                   {6, 2}, {7, 2}, {8, 1}, {8, 2}})
                cand.push_back(cm_batch_schedule{cg.first, cg.second, bin, 0});
        if (b->nwin == 1) cand = {{1, 0, 0, 0}, {1, 0, 1, 0}, {1, 0, 2, 0}, {1, 0, 3, 0}};
        for (int bin : {0, 2})  // the persistent step, its queue staggered by 0, 1, 2 or 7 phases
            for (int p : {1, 2, 3, 8}) cand.push_back(cm_batch_schedule{1, 0, bin, p});
    }
    cudaEvent_t a = nullptr, z = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&z) != cudaSuccess) return CM_ECUDA;
    float best = 1e30f;
    cm_batch_schedule pick = b->sched;
    int st = CM_OK;
    for (const cm_batch_schedule& c : cand) {
        if ((st = apply_schedule(b, c))) break;
        if ((st = run_plan(b, s))) break;  // capture + warm-up
        cudaEventRecord(a, s);
        for (int r = 0; r < 5 && !st; ++r) st = run_plan(b, s);
        cudaEventRecord(z, s);
        if (st || cudaEventSynchronize(z) != cudaSuccess) {
            st = st ? st : CM_ECUDA;
            break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, z);
        if (ms < best) {
            best = ms;
            pick = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    if (st) return st;
    if ((st = apply_schedule(b, pick))) return st;
    g_tuned.push_back({k, pick});
    if (chosen) *chosen = pick;
    return CM_OK;
}

int cm_batch_status(const cm_batch* b, void* stream)
{
    if (!b) return CM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (b->sched.persist <= 0) return cudaStreamSynchronize(s) == cudaSuccess ? CM_OK : CM_ECUDA;
    int32_t err = 0;  // the error word, behind the queue head
    if (cudaMemcpyAsync(&err, b->base + b->L.pq + sizeof(int32_t), sizeof(err), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CM_ECUDA;
    return err ? CM_ETIMEOUT : CM_OK;
}

int cm_batch_inject_stall(cm_batch* b, int32_t window)
{
    if (!b || window < -1 || window >= b->cap) return CM_EINVAL;
    b->stall_window = window;
    return apply_schedule(b, b->sched);
}

int cm_batch_stats(const cm_batch* b, int32_t window, const float** loss_r, const int32_t** nnz_r)
{
    if (!b || window < 0 || window >= b->nwin) return CM_EINVAL;
    if (loss_r) *loss_r = b->stat_lr[window];
    if (nnz_r) *nnz_r = b->stat_nnz[window];
    return CM_OK;
}

int cm_batch_destroy(cm_batch* b)
{
    destroy_batch(b);
    return CM_OK;
}

}  // extern "C"
