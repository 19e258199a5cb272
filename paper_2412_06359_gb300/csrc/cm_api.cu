// cm_api.cu -- the C ABI of libcm.so (include/cm.h): argument validation,
// workspace layout over caller-owned device memory, and the launch sequence
// of each entry point.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "../../include/cm.h"
#include "cm_bands.cuh"
#include "cm_launch.h"
#include "cm_sort.h"

using cmk::Win;

struct cm_workspace {
    char* base;
    size_t bytes;
    cm_camera cam;
    cm_loss_cfg cfg;
    int64_t max_events;
    int32_t nfb;
    int32_t R;
    int32_t loss_tiles, pix_tiles;
    float4* iwe;
    float2* flow;
    float2* dflow;
    float2* loss_part;
    float* norm;
    float* loss_r;
    int32_t* nnz_r;
    float* dego_part;
    float2* warp;            // [B+1][max_events] stored trajectory points (store_warps), else nullptr
    cmk::FQ* fq;             // [H][W] flow quads and
    cmk::FQ* dq;             // [H][W] quad accumulators of dL/dflow: the plane layout (below), else nullptr
    int32_t bands;           // > 0: events grouped by band of rows on the plane layout (below)
    int32_t* band_tab;       // [bands][super-chunks of max_events]
    int32_t* sync;           // [4] completion counters (zeroed by the first forward)
    int16_t* gx;             // [max_events] the events grouped by band
    int16_t* gy;
    float* gt;
    int8_t* gp;
    bool sync_zeroed;
    float* scal;             // [4] device scalars of cm_rsat
    bool has_sort;           // buffers of the deterministic sort path are laid out
    cmk::SortBufs sb;
    // state of the last forward on this workspace
    int fwd_mode;            // 0 none, 1 flow input, 2 depth input
    const void* fwd_events;  // event x pointer of the last forward
    int64_t fwd_n;
    bool fwd_warp;           // the last forward stored its trajectory points in `warp`
    bool fwd_planes;         // the last forward used the plane layout
    bool fwd_grouped;        // the last forward grouped its events by band
    bool dq_dirty;           // the quad accumulators hold a backward's sums (else zero, as the prep pass left them)
};

namespace cmk {

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

int check_camera(const cm_camera* cam)
{
    if (!cam) return CM_EINVAL;
    if (cam->width < 2 || cam->height < 2 || cam->width > 32767 || cam->height > 32767) return CM_EINVAL;
    if (!finite_pos(cam->fx) || !finite_pos(cam->fy) || !std::isfinite(cam->cx) || !std::isfinite(cam->cy))
        return CM_EINVAL;
    return CM_OK;
}

int check_cfg(const cm_loss_cfg* cfg)
{
    if (!cfg) return CM_EINVAL;
    if (cfg->nbins < 1 || cfg->nbins > CM_MAX_BINS) return CM_EINVAL;
    if (cfg->ref_mode != CM_REF_END && cfg->ref_mode != CM_REF_ALL_EDGES) return CM_EINVAL;
    if (cfg->splat != CM_SPLAT_AUTO && cfg->splat != CM_SPLAT_ATOMIC && cfg->splat != CM_SPLAT_SORT) return CM_EINVAL;
    if (cfg->store_warps != 0 && cfg->store_warps != 1) return CM_EINVAL;
    if (!std::isfinite(cfg->eps)) return CM_EINVAL;
    return CM_OK;
}

int check_events(const cm_events* ev)
{
    if (!ev || ev->n < 0) return CM_EINVAL;
    if (ev->n > 0 && (!ev->x || !ev->y || !ev->t || !ev->p)) return CM_EINVAL;
    if (!std::isfinite(ev->t0) || !std::isfinite(ev->t1) || !(ev->t1 > ev->t0)) return CM_EINVAL;
    const float span = ev->t1 - ev->t0;
    if (!(span > 0.0f) || !std::isfinite(span)) return CM_EINVAL;
    return CM_OK;
}

}  // namespace cmk

namespace {

using cmk::check_camera;
using cmk::check_cfg;
using cmk::check_events;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int n_refs(const cm_loss_cfg& c) { return c.ref_mode == CM_REF_END ? 1 : c.nbins + 1; }

int tiles_for(size_t hw, size_t px, int cap)
{
    size_t t = (hw + px - 1) / px;
    if (t < 1) t = 1;
    if (t > (size_t)cap) t = cap;
    return (int)t;
}

struct Layout {
    size_t iwe, flow, dflow, loss_part, norm, loss_r, nnz_r, dego_part, warp, scal, fq, dq, total;
    size_t band_tab, sync, gx, gy, gt, gp;
    int bands;
    size_t ka, kb, va, vb, pay, hist, part, start;  // sort path (CM_SPLAT_SORT only)
    int R, loss_tiles, pix_tiles;
    bool sort, planes;
};

// The atomic path of a window with one flow field keeps the batched plan's
// layout: the images as polarity planes of (C, S) pairs (a splat row's two
// corners in one 16-byte reduction, the adjoint's gathers in 16-byte loads),
// the flow as 32-byte quads (one load per bilinear sample) and dL/dflow in
// per-cell quad accumulators.  cm_warp_splat, the sort path and per-bin flows
// keep the [R][H][W] float4 images and the flow as given.
bool plane_layout(const cm_loss_cfg& cfg, int32_t nfb) { return cfg.splat != CM_SPLAT_SORT && nfb == 1; }

// On the plane layout, windows whose images exceed about 3/4 of the 129 MB L2
// group their events by band of 32 rows first (their time order kept within a
// band): the events in flight then touch one strip of the images.  Returns the
// number of bands, or 0.
int band_count_for(const cm_camera& cam, int R)
{
    const size_t img = (size_t)R * cam.width * cam.height * sizeof(float4);
    const int nb = (cam.height + cmk::kBandRows - 1) / cmk::kBandRows;
    return img > ((size_t)96 << 20) && nb <= cmk::kMaxBands ? nb : 0;
}

float eps_of(const cm_loss_cfg& c) { return c.eps > 0.0f ? c.eps : 1e-9f; }

Layout layout(const cm_camera& cam, const cm_loss_cfg& cfg, int32_t nfb, int64_t max_events)
{
    Layout L{};
    const size_t HW = (size_t)cam.width * cam.height;
    L.R = n_refs(cfg);
    // pixel passes of one window: tiles of 512 pixels (up to 1024 tiles), so
    // that even a 346x260 window's passes spread over every SM
    L.loss_tiles = tiles_for(HW, 512, 1024);
    L.pix_tiles = tiles_for(HW, 512, 1024);
    size_t off = 0;
    L.iwe = off;
    off = align_up(off + (size_t)L.R * HW * sizeof(float4));
    L.flow = off;
    off = align_up(off + HW * sizeof(float2));
    L.dflow = off;
    off = align_up(off + (size_t)nfb * HW * sizeof(float2));
    L.loss_part = off;
    off = align_up(off + (size_t)L.R * L.loss_tiles * sizeof(float2));
    L.norm = off;
    off = align_up(off + (size_t)L.R * sizeof(float));
    L.loss_r = off;
    off = align_up(off + (size_t)L.R * sizeof(float));
    L.nnz_r = off;
    off = align_up(off + (size_t)L.R * sizeof(int32_t));
    L.dego_part = off;
    off = align_up(off + (size_t)L.pix_tiles * 6 * sizeof(float));
    L.warp = off;
    if (cfg.store_warps) off = align_up(off + (size_t)(cfg.nbins + 1) * max_events * sizeof(float2));
    L.scal = off;
    off = align_up(off + 4 * sizeof(float));
    L.planes = plane_layout(cfg, nfb);
    L.bands = 0;
    if (L.planes) {
        L.fq = off;
        off = align_up(off + HW * sizeof(cmk::FQ));
        L.dq = off;
        off = align_up(off + HW * sizeof(cmk::FQ));
        // completion counters: the fused loss and gradient reductions, the grouping
        L.sync = off;
        off = align_up(off + 4 * sizeof(int32_t));
        L.bands = max_events > 0 ? band_count_for(cam, L.R) : 0;
        if (L.bands) {
            const size_t nsc = (size_t)((max_events + cmk::kSuperChunk - 1) / cmk::kSuperChunk);
            L.band_tab = off;
            off = align_up(off + (size_t)L.bands * nsc * sizeof(int32_t));
            L.gx = off;
            off = align_up(off + (size_t)max_events * sizeof(int16_t));
            L.gy = off;
            off = align_up(off + (size_t)max_events * sizeof(int16_t));
            L.gt = off;
            off = align_up(off + (size_t)max_events * sizeof(float));
            L.gp = off;
            off = align_up(off + (size_t)max_events);
        }
    }
    L.sort = cfg.splat == CM_SPLAT_SORT;
    if (L.sort) {
        const cmk::SortSizes z = cmk::sort_sizes(max_events, L.R, cfg.nbins, nfb, HW);
        L.ka = off;
        off = align_up(off + z.entries * 4);
        L.kb = off;
        off = align_up(off + z.entries * 4);
        L.va = off;
        off = align_up(off + z.entries * 4);
        L.vb = off;
        off = align_up(off + z.entries * 4);
        L.pay = off;
        off = align_up(off + z.entries * 16);
        L.hist = off;
        off = align_up(off + z.hist * 4);
        L.part = off;
        off = align_up(off + z.part * 4);
        L.start = off;
        off = align_up(off + z.start * 4);
    }
    L.total = off;
    return L;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? CM_OK : CM_ECUDA; }

// RSAT from the two losses (0 when the zero-flow loss is 0: no event in the image)
__global__ void k_ratio(const float* ab, float* out) { out[0] = ab[1] > 0.0f ? ab[0] / ab[1] : 0.0f; }

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// descriptor of one window over the workspace buffers
Win make_win(const cm_camera& cam, const cm_events* ev, const cm_loss_cfg& cfg, int32_t nfb)
{
    Win d;
    std::memset(&d, 0, sizeof(d));
    if (ev) {
        d.x = ev->x;
        d.y = ev->y;
        d.t = ev->t;
        d.p = ev->p;
        d.n = ev->n;
        d.t0 = ev->t0;
        d.span = ev->t1 - ev->t0;
    }
    d.W = cam.width;
    d.H = cam.height;
    d.B = cfg.nbins;
    d.R = n_refs(cfg);
    d.ref_mode = cfg.ref_mode;
    d.nfb = nfb;
    d.eps = eps_of(cfg);
    d.fx = cam.fx;
    d.fy = cam.fy;
    d.cx = cam.cx;
    d.cy = cam.cy;
    return d;
}

void attach_ws(Win& d, cm_workspace* ws)
{
    d.iwe = ws->iwe;
    d.loss_part = ws->loss_part;
    d.loss_tiles = ws->loss_tiles;
    d.pix_tiles = ws->pix_tiles;
    d.norm = ws->norm;
    d.loss_r = ws->loss_r;
    d.nnz_r = ws->nnz_r;
    d.dego_part = ws->dego_part;
}

bool same_shape(const cm_workspace* ws, const cm_camera& cam, const cm_loss_cfg& cfg, int32_t nfb)
{
    return ws->cam.width == cam.width && ws->cam.height == cam.height && ws->cfg.nbins == cfg.nbins &&
           ws->cfg.ref_mode == cfg.ref_mode && nfb <= ws->nfb && (!cfg.store_warps || ws->warp);
}

// stored warps: [B+1][n] points of this call's events in the workspace
float2* warp_of(const cm_workspace* ws, const cm_loss_cfg& cfg) { return cfg.store_warps ? ws->warp : nullptr; }

}  // namespace

namespace cmk {
int sm_count_current()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    if (dev < 64) cache[dev] = n;
    return n;
}
}  // namespace cmk

extern "C" {

const char* cm_status_string(int s)
{
    switch (s) {
    case CM_OK: return "ok";
    case CM_EINVAL: return "invalid argument";
    case CM_ENOMEM: return "out of memory (workspace or server budget too small)";
    case CM_EBUSY: return "busy: no slot or memory free for the request";
    case CM_ETIMEOUT: return "a bounded wait gave up";
    case CM_ECUDA: return "CUDA runtime error";
    case CM_ENOTFOUND: return "unknown ticket";
    case CM_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

int cm_abi_version(void) { return 1; }

int cm_workspace_query(const cm_camera* cam, const cm_loss_cfg* cfg, int64_t max_events, int32_t n_flow_bins,
                       size_t* bytes)
{
    int st;
    if ((st = check_camera(cam)) || (st = check_cfg(cfg))) return st;
    if (!bytes || max_events < 0 || (n_flow_bins != 1 && n_flow_bins != cfg->nbins)) return CM_EINVAL;
    *bytes = layout(*cam, *cfg, n_flow_bins, max_events).total;
    return CM_OK;
}

int cm_workspace_create(void* dev_mem, size_t bytes, const cm_camera* cam, const cm_loss_cfg* cfg,
                        int64_t max_events, int32_t n_flow_bins, cm_workspace** out)
{
    int st;
    if ((st = check_camera(cam)) || (st = check_cfg(cfg))) return st;
    if (!out || !dev_mem || max_events < 0 || (n_flow_bins != 1 && n_flow_bins != cfg->nbins)) return CM_EINVAL;
    if (reinterpret_cast<uintptr_t>(dev_mem) % kAlign) return CM_EINVAL;
    const Layout L = layout(*cam, *cfg, n_flow_bins, max_events);
    if (bytes < L.total) return CM_ENOMEM;
    cm_workspace* ws = new (std::nothrow) cm_workspace{};
    if (!ws) return CM_ENOMEM;
    std::memset(ws, 0, sizeof(*ws));
    char* b = static_cast<char*>(dev_mem);
    ws->base = b;
    ws->bytes = bytes;
    ws->cam = *cam;
    ws->cfg = *cfg;
    ws->max_events = max_events;
    ws->nfb = n_flow_bins;
    ws->R = L.R;
    ws->loss_tiles = L.loss_tiles;
    ws->pix_tiles = L.pix_tiles;
    ws->iwe = reinterpret_cast<float4*>(b + L.iwe);
    ws->flow = reinterpret_cast<float2*>(b + L.flow);
    ws->dflow = reinterpret_cast<float2*>(b + L.dflow);
    ws->loss_part = reinterpret_cast<float2*>(b + L.loss_part);
    ws->norm = reinterpret_cast<float*>(b + L.norm);
    ws->loss_r = reinterpret_cast<float*>(b + L.loss_r);
    ws->nnz_r = reinterpret_cast<int32_t*>(b + L.nnz_r);
    ws->dego_part = reinterpret_cast<float*>(b + L.dego_part);
    ws->warp = cfg->store_warps ? reinterpret_cast<float2*>(b + L.warp) : nullptr;
    ws->scal = reinterpret_cast<float*>(b + L.scal);
    ws->fq = L.planes ? reinterpret_cast<cmk::FQ*>(b + L.fq) : nullptr;
    ws->dq = L.planes ? reinterpret_cast<cmk::FQ*>(b + L.dq) : nullptr;
    ws->bands = L.bands;
    ws->sync = L.planes ? reinterpret_cast<int32_t*>(b + L.sync) : nullptr;
    ws->sync_zeroed = false;
    if (L.bands) {
        ws->band_tab = reinterpret_cast<int32_t*>(b + L.band_tab);
        ws->gx = reinterpret_cast<int16_t*>(b + L.gx);
        ws->gy = reinterpret_cast<int16_t*>(b + L.gy);
        ws->gt = reinterpret_cast<float*>(b + L.gt);
        ws->gp = reinterpret_cast<int8_t*>(b + L.gp);
    }
    ws->has_sort = L.sort;
    if (L.sort) {
        ws->sb.ka = reinterpret_cast<uint32_t*>(b + L.ka);
        ws->sb.kb = reinterpret_cast<uint32_t*>(b + L.kb);
        ws->sb.va = reinterpret_cast<uint32_t*>(b + L.va);
        ws->sb.vb = reinterpret_cast<uint32_t*>(b + L.vb);
        ws->sb.pay = reinterpret_cast<float4*>(b + L.pay);
        ws->sb.hist = reinterpret_cast<uint32_t*>(b + L.hist);
        ws->sb.part = reinterpret_cast<uint32_t*>(b + L.part);
        ws->sb.start = reinterpret_cast<uint32_t*>(b + L.start);
    }
    *out = ws;
    return CM_OK;
}

int cm_workspace_destroy(cm_workspace* ws)
{
    delete ws;
    return CM_OK;
}

int cm_workspace_stats(const cm_workspace* ws, const float** loss_r, const int32_t** nnz_r)
{
    if (!ws) return CM_EINVAL;
    if (loss_r) *loss_r = ws->loss_r;
    if (nnz_r) *nnz_r = ws->nnz_r;
    return CM_OK;
}

int cm_flow_from_depth(const cm_camera* cam, const float* inv_depth, const float* ego6, float dt_window,
                       float* flow_out, void* stream)
{
    int st;
    if ((st = check_camera(cam))) return st;
    if (!inv_depth || !ego6 || !flow_out || !std::isfinite(dt_window)) return CM_EINVAL;
    cm_loss_cfg c{1, CM_REF_END, CM_SPLAT_AUTO, 0, 0.0f};
    Win d = make_win(*cam, nullptr, c, 1);
    d.rho = inv_depth;
    d.ego = ego6;
    d.dt = dt_window;
    d.flow = reinterpret_cast<const float2*>(flow_out);
    return cuda_status(cmk::launch_flow(d, as_stream(stream)));
}

int cm_warp_splat(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                  const cm_loss_cfg* cfg, cm_workspace* ws, float* iwe_out, void* stream)
{
    int st;
    if ((st = check_camera(cam)) || (st = check_cfg(cfg)) || (st = check_events(ev))) return st;
    if (!flow || (n_flow_bins != 1 && n_flow_bins != cfg->nbins)) return CM_EINVAL;
    if (!iwe_out && !ws) return CM_EINVAL;
    if (ws && !iwe_out && !same_shape(ws, *cam, *cfg, n_flow_bins)) return CM_EINVAL;
    Win d = make_win(*cam, ev, *cfg, n_flow_bins);
    d.flow = reinterpret_cast<const float2*>(flow);
    d.iwe = iwe_out ? reinterpret_cast<float4*>(iwe_out) : ws->iwe;
    cudaStream_t s = as_stream(stream);
    if (cfg->splat == CM_SPLAT_SORT) {
        // the sort path needs a workspace laid out for it and for this shape
        if (!ws || !ws->has_sort || !same_shape(ws, *cam, *cfg, n_flow_bins)) return CM_EINVAL;
        if (ev->n > ws->max_events) return CM_ENOMEM;
        return cuda_status(cmk::sort_splat(d, ws->sb, cmk::sm_count_current(), s));
    }
    const size_t bytes = (size_t)d.R * d.W * d.H * sizeof(float4);
    if ((st = cuda_status(cudaMemsetAsync(d.iwe, 0, bytes, s)))) return st;
    return cuda_status(cmk::launch_splat(d, cmk::sm_count_current(), s));
}

int cm_loss_forward(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                    const float* inv_depth, const float* ego6, float dt_window, const cm_loss_cfg* cfg,
                    cm_workspace* ws, float* loss_out, void* stream)
{
    int st;
    if ((st = check_camera(cam)) || (st = check_cfg(cfg)) || (st = check_events(ev))) return st;
    if (!ws || !loss_out) return CM_EINVAL;
    if (n_flow_bins != 1 && n_flow_bins != cfg->nbins) return CM_EINVAL;
    const bool depth = flow == nullptr;
    if (depth && (!inv_depth || !ego6 || n_flow_bins != 1 || !std::isfinite(dt_window))) return CM_EINVAL;
    if (!same_shape(ws, *cam, *cfg, n_flow_bins)) return CM_EINVAL;
    if (ev->n > ws->max_events) return CM_ENOMEM;
    cudaStream_t s = as_stream(stream);
    Win d = make_win(*cam, ev, *cfg, n_flow_bins);
    attach_ws(d, ws);
    d.loss = loss_out;
    d.warp = warp_of(ws, *cfg);
    if (ws->fq && plane_layout(*cfg, n_flow_bins)) {
        // the plane layout: quads built (from the flow or the motion field) by the prep pass
        d.iwe_split = 1;
        d.fq = ws->fq;
        d.dq = ws->dq;
        if (depth) {
            d.rho = inv_depth;
            d.ego = ego6;
            d.dt = dt_window;
        } else {
            d.flow = reinterpret_cast<const float2*>(flow);
        }
        const int sms = cmk::sm_count_current();
        const bool grouped = ws->bands > 0 && ev->n >= cmk::kSuperChunk;
        // the completion counters of the fused reductions (and of the grouping)
        // start at zero once; every use returns them to zero
        if (!ws->sync_zeroed) {
            if ((st = cuda_status(cudaMemsetAsync(ws->sync, 0, 4 * sizeof(int32_t), s)))) return st;
            ws->sync_zeroed = true;
        }
        d.sync = ws->sync;
        if (grouped) {
            Win g = d;
            g.tile_cnt = ws->band_tab;
            g.sync = ws->sync;
            g.gsync = ws->sync + 2;
            g.rx = ws->gx;
            g.ry = ws->gy;
            g.rt = ws->gt;
            g.rp = ws->gp;
            g.ntx = 1;
            g.nty = ws->bands;
            g.band_rows = cmk::kBandRows;
            if ((st = cuda_status(cmk::launch_bands(g, sms, s)))) return st;
            d.x = ws->gx;
            d.y = ws->gy;
            d.t = ws->gt;
            d.p = ws->gp;
        }
        if ((st = cuda_status(cmk::launch_prep(d, sms, s)))) return st;
        if ((st = cuda_status(cmk::launch_splat(d, sms, s)))) return st;
        if ((st = cuda_status(cmk::launch_loss_planes(d, s)))) return st;
        ws->fwd_mode = depth ? 2 : 1;
        ws->fwd_events = ev->x;
        ws->fwd_n = ev->n;
        ws->fwd_warp = d.warp != nullptr;
        ws->fwd_planes = true;
        ws->fwd_grouped = grouped;
        ws->dq_dirty = false;
        return CM_OK;
    }
    if (depth) {
        d.rho = inv_depth;
        d.ego = ego6;
        d.dt = dt_window;
        d.flow = ws->flow;
        if ((st = cuda_status(cmk::launch_flow(d, s)))) return st;
    } else {
        d.flow = reinterpret_cast<const float2*>(flow);
    }
    if (cfg->splat == CM_SPLAT_SORT) {
        if (!ws->has_sort) return CM_EINVAL;
        if ((st = cuda_status(cmk::sort_splat(d, ws->sb, cmk::sm_count_current(), s)))) return st;
    } else {
        const size_t bytes = (size_t)d.R * d.W * d.H * sizeof(float4);
        if ((st = cuda_status(cudaMemsetAsync(d.iwe, 0, bytes, s)))) return st;
        if ((st = cuda_status(cmk::launch_splat(d, cmk::sm_count_current(), s)))) return st;
    }
    if ((st = cuda_status(cmk::launch_loss(d, s)))) return st;
    ws->fwd_mode = depth ? 2 : 1;
    ws->fwd_events = ev->x;
    ws->fwd_n = ev->n;
    ws->fwd_warp = d.warp != nullptr;
    ws->fwd_planes = false;
    return CM_OK;
}

int cm_loss_backward(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                     const float* inv_depth, const float* ego6, float dt_window, const cm_loss_cfg* cfg,
                     cm_workspace* ws, const float* dloss, float* dflow, float* dinv_depth, float* dego6,
                     void* stream)
{
    int st;
    if ((st = check_camera(cam)) || (st = check_cfg(cfg)) || (st = check_events(ev))) return st;
    if (!ws || !dloss) return CM_EINVAL;
    if (n_flow_bins != 1 && n_flow_bins != cfg->nbins) return CM_EINVAL;
    const bool depth = flow == nullptr;
    if (depth && (!inv_depth || !ego6 || n_flow_bins != 1 || !std::isfinite(dt_window))) return CM_EINVAL;
    if (!same_shape(ws, *cam, *cfg, n_flow_bins)) return CM_EINVAL;
    if (ws->fwd_mode != (depth ? 2 : 1) || ws->fwd_events != ev->x || ws->fwd_n != ev->n) return CM_ESTATE;
    if (!depth && (dinv_depth || dego6)) return CM_EINVAL;
    cudaStream_t s = as_stream(stream);
    Win d = make_win(*cam, ev, *cfg, n_flow_bins);
    attach_ws(d, ws);
    d.dloss = dloss;
    d.warp = ws->fwd_warp ? ws->warp : nullptr;  // read back whenever the forward stored them
    if (ws->fwd_planes) {
        // the plane layout: pushes into the quad accumulators (zeroed by the
        // forward's prep pass), then folded per pixel
        d.iwe_split = 1;
        d.fq = ws->fq;
        d.dq = ws->dq;
        d.flow = depth ? nullptr : reinterpret_cast<const float2*>(flow);
        d.dflow = dflow ? reinterpret_cast<float2*>(dflow) : nullptr;
        if (ws->fwd_grouped) {  // the forward's grouped copy of the events, in the same order
            d.x = ws->gx;
            d.y = ws->gy;
            d.t = ws->gt;
            d.p = ws->gp;
        }
        if (!depth && !dflow) return CM_OK;
        if (ws->dq_dirty &&
            (st = cuda_status(cudaMemsetAsync(ws->dq, 0, (size_t)cam->width * cam->height * sizeof(cmk::FQ), s))))
            return st;
        if ((st = cuda_status(cmk::launch_adjoint(d, cmk::sm_count_current(), s)))) return st;
        ws->dq_dirty = true;
        if (depth) {
            if (!dinv_depth && !dego6) {
                if (d.dflow) return cuda_status(cmk::launch_fold(d, s));
                return CM_OK;
            }
            d.rho = inv_depth;
            d.ego = ego6;
            d.dt = dt_window;
            d.drho = dinv_depth;
            d.dego = dego6;
            d.sync = ws->sync;  // zeroed by the forward
            return cuda_status(cmk::launch_depth_ego_planes(d, s));  // folds the accumulators (and stores dL/dflow)
        }
        return cuda_status(cmk::launch_fold(d, s));
    }
    d.flow = depth ? ws->flow : reinterpret_cast<const float2*>(flow);
    d.dflow = dflow ? reinterpret_cast<float2*>(dflow) : ws->dflow;
    if (!depth && !dflow) return CM_OK;
    if (cfg->splat == CM_SPLAT_SORT) {
        if (!ws->has_sort) return CM_EINVAL;
        if ((st = cuda_status(cmk::sort_adjoint(d, ws->sb, cmk::sm_count_current(), s)))) return st;
    } else {
        const size_t gbytes = (size_t)n_flow_bins * d.W * d.H * sizeof(float2);
        if ((st = cuda_status(cudaMemsetAsync(d.dflow, 0, gbytes, s)))) return st;
        if ((st = cuda_status(cmk::launch_adjoint(d, cmk::sm_count_current(), s)))) return st;
    }
    if (depth && (dinv_depth || dego6)) {
        d.rho = inv_depth;
        d.ego = ego6;
        d.dt = dt_window;
        d.drho = dinv_depth;
        d.dego = dego6;
        if ((st = cuda_status(cmk::launch_depth_ego(d, s)))) return st;
    }
    return CM_OK;
}

int cm_rsat(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
            const cm_loss_cfg* cfg, cm_workspace* ws, float* rsat_out, void* stream)
{
    if (!ws || !rsat_out || !flow) return CM_EINVAL;
    cudaStream_t s = as_stream(stream);
    int st = cm_loss_forward(cam, ev, flow, n_flow_bins, nullptr, nullptr, 0.0f, cfg, ws, ws->scal + 0, stream);
    if (st) return st;
    // the unwarped events: zero flow in the workspace's own flow buffer
    if ((st = cuda_status(cudaMemsetAsync(ws->flow, 0, (size_t)cam->width * cam->height * sizeof(float2), s))))
        return st;
    st = cm_loss_forward(cam, ev, reinterpret_cast<const float*>(ws->flow), 1, nullptr, nullptr, 0.0f, cfg, ws,
                         ws->scal + 1, stream);
    ws->fwd_mode = 0;  // neither forward is left for a backward
    if (st) return st;
    cmk::KernelScope ks("k_ratio", s);
    k_ratio<<<1, 1, 0, s>>>(ws->scal, rsat_out);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
