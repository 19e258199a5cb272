/*
 * cm.h -- C ABI of the GB300 contrast-maximisation (CM) library, libcm.so.
 *
 * The library computes the self-supervised loss of arXiv 2412.06359 ("On-Device
 * Self-Supervised Learning of Low-Latency Monocular Depth from Only Events")
 * and its gradient on one GPU, every step in hand-written sm_103a kernels:
 *
 *   flow from inverse depth and ego-motion   (Sec. 3.2, Eq. 2; rigid motion field)
 *   iterative warp of every event to the bin edges, bilinearly re-sampling
 *     the flow at the current position        (Sec. 3.1; Sec. 3.3)
 *   masking of events that leave the image at any point   (Sec. 3.1)
 *   bilinear splat into polarity-split images of warped events (IWEs) of
 *     counts and timestamp sums               (Sec. 3.1, kernel kappa in Eq. 1)
 *   the average-timestamp focus loss, scaled by the number of non-empty
 *     pixels and averaged over the reference times   (Eq. 1)
 *   the analytic backward to flow, inverse depth and ego-motion (Sec. 3.3)
 *
 * Definitions used throughout (the paper leaves these open; the design notes
 * of the repository list each reading with its reason):
 *   tau = (t - t0) / (t1 - t0) is time normalised to the window [t0, t1];
 *   B bins of equal length, edges tau_j = j / B; an event at tau lies in bin
 *   b = min(floor(tau B), B - 1).
 *   Reference times: CM_REF_END -> only the window end (R = 1);
 *   CM_REF_ALL_EDGES -> all B + 1 bin edges (R = B + 1).
 *   Average timestamp of an event at reference tau_r: 1 - |tau_r - tau|.
 *   IWE of reference r, pixel x, polarity p: C_p(x) = sum of bilinear weights,
 *   S_p(x) = sum of weight * average timestamp; T_p = S_p / (C_p + eps);
 *   L_r = sum_x (T_+^2 + T_-^2) / (N_nz(r) + eps), N_nz(r) = number of pixels
 *   with C_+ + C_- > 0;  loss L = (1/R) sum_r L_r.
 *   Pixel centres lie at integer coordinates; the image is the closed box
 *   [0, W-1] x [0, H-1]; an event any of whose computed trajectory points lies
 *   outside it contributes to no IWE.
 *   Flow is in pixels per window (per unit tau).
 *
 * Conventions for every entry point:
 *   - Pointers named dev_* or documented as "device" are CUDA device memory the
 *     caller owns (for example torch tensors' data_ptr()).  Host structs
 *     (cm_camera, cm_events, cm_loss_cfg) are read during the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every call is asynchronous and stream-ordered: it enqueues work
 *     and returns; results are valid once the stream reaches that point.
 *   - The return value is a status code (CM_OK = 0).  Arguments are validated
 *     on the host before anything is enqueued; nothing is enqueued on error.
 *     No exception crosses the ABI.
 *   - Events are structure-of-arrays in device memory: x, y int16 pixel column
 *     and row, t float32 (ascending order is expected for performance, not for
 *     correctness), p int8 polarity (> 0 positive, otherwise negative).  An
 *     event whose (x, y) lies outside the sensor is treated as masked.
 */
#ifndef CM_H
#define CM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CM_OK 0
#define CM_EINVAL 1     /* invalid argument (sizes, null pointers, nbins, t1 <= t0, ...) */
#define CM_ENOMEM 2     /* workspace or server memory too small / allocation failed */
#define CM_EBUSY 3      /* server: no slot or memory free for the request right now */
#define CM_ETIMEOUT 4   /* a bounded wait gave up */
#define CM_ECUDA 5      /* a CUDA runtime call failed (launch error, ...) */
#define CM_ENOTFOUND 6  /* server: unknown ticket */
#define CM_ESTATE 7     /* call out of order (backward without a forward, ...) */

/* ---- reference-time modes ---- */
#define CM_REF_END 0        /* one reference at the window end (the linear-warp variant, Sec. 4.2) */
#define CM_REF_ALL_EDGES 1  /* every bin edge (supp. "Training": warp all events to all bin edges) */

/* ---- splat strategies ---- */
#define CM_SPLAT_AUTO 0     /* pick by the autotuner's cached choice (atomic until tuned) */
#define CM_SPLAT_ATOMIC 1   /* FP32 vector atomics into the IWE (order of additions not fixed) */
#define CM_SPLAT_SORT 2     /* deterministic: sort contributions by pixel, segmented sums.  In a batched
                               plan each window runs whole through this path, one window at a time on
                               each of 1..8 chains (schedule {chains, 1, 0, 0}, default 8 chains; other
                               schedules are refused with CM_EINVAL; the autotuner picks the chains),
                               windows with their own scratch are refused, and the outputs are the same
                               bits on every run whatever the number of chains */
#define CM_SPLAT_TILES 3    /* batched plans only: accumulate each 32x32 tile in shared memory, flush once
                               (warp-aggregated shared-memory atomics; schedule bin 3).  The single-window
                               entry points refuse it (CM_EINVAL) */

#define CM_MAX_BINS 32      /* largest supported number of bins B */

/* Pinhole intrinsics of an undistorted, rectified sensor of width x height pixels. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
} cm_camera;

/* One window of events (device SoA arrays of n entries) and its time span. */
typedef struct {
    const int16_t* x;
    const int16_t* y;
    const float* t;
    const int8_t* p;
    int64_t n;
    float t0, t1;
} cm_events;

/* Loss configuration. */
typedef struct {
    int32_t nbins;        /* B, 1..CM_MAX_BINS */
    int32_t ref_mode;     /* CM_REF_END or CM_REF_ALL_EDGES */
    int32_t splat;        /* CM_SPLAT_* */
    int32_t store_warps;  /* 0: the backward recomputes the trajectories (default); 1: the forward
                             stores every computed trajectory point ((B+1) x 8 bytes per event, in
                             the workspace or the batch plan) and the backward reads them back, the
                             choice of the paper's own backward (Sec. 3.3).  Same results either way
                             (the points are the same FP32 values).  Windows that bring their own
                             scratch (cm_window.scratch) always recompute. */
    float eps;            /* regulariser of both ratios; 1e-9 when <= 0 */
} cm_loss_cfg;

/* Opaque handle: the layout of a caller-provided device buffer (IWE, flow,
 * reduction partials, statistics) plus the state the backward needs. */
typedef struct cm_workspace cm_workspace;

/* Human-readable name of a status code (static string). */
const char* cm_status_string(int status);

/* Library ABI version (incremented on incompatible changes). */
int cm_abi_version(void);

/*
 * Device bytes a workspace needs for windows of this camera and configuration
 * with up to max_events events and n_flow_bins flow fields (1 or nbins).
 * Writes the size to *bytes.  Errors: CM_EINVAL.
 */
int cm_workspace_query(const cm_camera* cam, const cm_loss_cfg* cfg, int64_t max_events,
                       int32_t n_flow_bins, size_t* bytes);

/*
 * Lay a workspace over caller-owned device memory dev_mem of `bytes` bytes
 * (256-byte aligned, at least cm_workspace_query's size).  The library never
 * allocates device memory for a workspace and never frees dev_mem; *ws is a
 * small host object released by cm_workspace_destroy.  A workspace serves one
 * stream at a time.  Errors: CM_EINVAL, CM_ENOMEM (buffer too small).
 */
int cm_workspace_create(void* dev_mem, size_t bytes, const cm_camera* cam, const cm_loss_cfg* cfg,
                        int64_t max_events, int32_t n_flow_bins, cm_workspace** ws);
int cm_workspace_destroy(cm_workspace* ws);

/*
 * S1 (Sec. 3.2, Eq. 2 in its instantaneous form): per-pixel flow of a static
 * scene for a camera moving with linear velocity v and angular velocity w,
 *   xn = (u - cx)/fx, yn = (v - cy)/fy, rho = inverse depth,
 *   flow_x = dt fx [rho(-vx + xn vz) + xn yn wx - (1 + xn^2) wy + yn wz]
 *   flow_y = dt fy [rho(-vy + yn vz) + (1 + yn^2) wx - xn yn wy - xn wz]
 * inv_depth: device float [H][W]; ego6: device float (vx, vy, vz, wx, wy, wz);
 * flow_out: device float [H][W][2].  dt_window: window length in the units of
 * the velocities.  Errors: CM_EINVAL, CM_ECUDA.
 */
int cm_flow_from_depth(const cm_camera* cam, const float* inv_depth, const float* ego6, float dt_window,
                       float* flow_out, void* stream);

/*
 * S2-S4 (Sec. 3.1, 3.3): warp every event along its trajectory and splat it
 * into the IWEs.  flow: device float [n_flow_bins][H][W][2] (n_flow_bins 1 or
 * cfg->nbins).  iwe_out: device float [R][H][W][4] holding (C+, S+, C-, S-) per
 * pixel; it is zeroed and filled by the call.  If iwe_out is NULL the IWE is
 * built in the workspace.  ws may be NULL when iwe_out is given.
 * Errors: CM_EINVAL, CM_ECUDA.
 */
int cm_warp_splat(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                  const cm_loss_cfg* cfg, cm_workspace* ws, float* iwe_out, void* stream);

/*
 * S1-S5: the CM loss of one window, written to the device float *loss_out.
 * Give either flow (device [n_flow_bins][H][W][2]) or, with flow NULL,
 * inv_depth (device [H][W]) + ego6 (device [6]) + dt_window, from which the
 * flow is computed into the workspace (n_flow_bins must then be 1).
 * The workspace keeps what the backward needs; the per-reference losses and
 * non-empty counts can be read with cm_workspace_stats.  With one flow field
 * and the atomic splat the workspace holds the images as polarity planes of
 * (C, S) pairs and the flow as 32-byte cell quads (the batched plan's layout:
 * 16-byte splat reductions and gathers, one load per bilinear sample); with
 * per-bin flows or the sort splat, [R][H][W] float4 images and the flow as
 * given.  The results are the same either way (within the parity tolerances).
 * Errors: CM_EINVAL, CM_ENOMEM (workspace too small for n), CM_ECUDA.
 */
int cm_loss_forward(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                    const float* inv_depth, const float* ego6, float dt_window, const cm_loss_cfg* cfg,
                    cm_workspace* ws, float* loss_out, void* stream);

/*
 * S6-S7 (Sec. 3.3 backward pass): gradient of dloss * L, where dloss is a device
 * float scalar (the upstream gradient).  Must follow cm_loss_forward on the
 * same workspace and stream with the same arguments.  Trajectories are
 * recomputed, not stored.  Outputs (each may be NULL):
 *   dflow       device float [n_flow_bins][H][W][2]   dL/dflow
 *   dinv_depth  device float [H][W]                    dL/d(inverse depth)  (depth input only)
 *   dego6       device float [6]                       dL/d(ego-motion)     (depth input only)
 * Outputs are overwritten, not accumulated; the backward may be called again
 * after the same forward.  Errors: CM_EINVAL, CM_ESTATE, CM_ECUDA.
 */
int cm_loss_backward(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                     const float* inv_depth, const float* ego6, float dt_window, const cm_loss_cfg* cfg,
                     cm_workspace* ws, const float* dloss, float* dflow, float* dinv_depth, float* dego6,
                     void* stream);

/*
 * Device pointers to the per-reference statistics of the last forward on ws:
 * loss_r -> float [R] (L_r), nnz_r -> int32 [R] (N_nz(r)).  Either may be NULL.
 */
int cm_workspace_stats(const cm_workspace* ws, const float** loss_r, const int32_t** nnz_r);

/* ---- network input and evaluation metric ----
 * The network's input frame (supp. Table 4, a (2, H, W) input): the events of
 * a window counted per pixel and polarity, channel 0 positive, channel 1
 * negative, as float; events outside the sensor are skipped.  frame_out is
 * device memory [2][H][W], overwritten.  Counts are exact integers, so the
 * result is the same on every run.  Errors: CM_EINVAL, CM_ECUDA. */
int cm_event_frame(const cm_camera* cam, const cm_events* ev, float* frame_out, void* stream);
/* RSAT, the ratio of squared average timestamps (the deblurring metric the
 * paper reports beside depth error, Sec. 4.3, Fig. 4): the CM loss of the
 * events warped by `flow` over the CM loss of the unwarped events (zero flow),
 * same configuration and references; 0 when the zero-flow loss is 0.  Runs two
 * forwards on `ws` (whose own flow buffer holds the zero flow), so a
 * following cm_loss_backward on `ws` returns CM_ESTATE until the next
 * cm_loss_forward.  rsat_out: device scalar.  Errors as cm_loss_forward. */
int cm_rsat(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
            const cm_loss_cfg* cfg, cm_workspace* ws, float* rsat_out, void* stream);

/* ---- discrete flow: Eq. 2 with one pose per bin ----
 * The flow of bin i (of nb) by the reprojection of Eq. 2 (Sec. 3.2): pixel
 * (u, v) with inverse depth rho is back-projected to X = (xn, yn, 1) / rho
 * (xn = (u - cx)/fx, yn = (v - cy)/fy), moved as P = R X + t for a camera that
 * moves with velocity v_i and angular velocity w_i (ego6[6i .. 6i+5] =
 * (vx, vy, vz, wx, wy, wz), m/s and rad/s, camera frame) for dt_bin seconds
 * (R = Rodrigues(-w_i dt_bin), t = -v_i dt_bin), and re-projected; the flow is
 * `scale` times the displacement (fx (P0/P2 - xn), fy (P1/P2 - yn)), px.
 * With nb = B bins splitting a window evenly, dt_bin = window / B and
 * scale = B give px per window, the unit cm_loss_forward takes with
 * n_flow_bins = B.  All pointers are device memory; stream-ordered.
 *   flow_out [nb][H][W][2].  Errors: CM_EINVAL (bad camera, nb outside
 *   1..CM_MAX_BINS, non-finite dt_bin / scale, NULL pointers), CM_ECUDA. */
int cm_flow_eq2(const cm_camera* cam, const float* inv_depth, const float* ego6, int32_t nb, float dt_bin,
                float scale, float* flow_out, void* stream);
/* Device bytes of the scratch cm_flow_eq2_backward needs (per-tile partial sums). */
int cm_flow_eq2_scratch_query(const cm_camera* cam, int32_t nb, size_t* bytes);
/* Adjoint of cm_flow_eq2: from dflow [nb][H][W][2] = dL/dflow, writes
 * dinv_depth [H][W] = dL/d(inverse depth) summed over the bins and
 * dego6 [nb][6] = dL/d(v_i, w_i), through the projection, the rigid transform
 * and the derivative of Rodrigues' formula (fixed-order reductions:
 * deterministic).  scratch: device memory, 16-byte aligned, at least
 * cm_flow_eq2_scratch_query bytes (CM_ENOMEM otherwise). */
int cm_flow_eq2_backward(const cm_camera* cam, const float* inv_depth, const float* ego6, int32_t nb, float dt_bin,
                         float scale, const float* dflow, float* dinv_depth, float* dego6, void* scratch,
                         size_t scratch_bytes, void* stream);

/* ---- geometry-consistency loss (Eq. 3) ----
 * Between the depth of view 0 (inv_depth0) moved by the camera motion from
 * view 0 to view 1 (ego6 = (v, w) over dt seconds, the rigid transform of
 * cm_flow_eq2: P = R X + t) and the depth of view 1 (inv_depth1): for every
 * pixel x of view 0 the forward-projected depth a = P2 and the depth b of
 * view 1 bilinearly interpolated at the projection x' (corner indices
 * clamped); valid pixels V have P2 > 0 and x' inside the closed image box;
 *   L_geo = (1/|V|) sum_V |a - b| / (a + b)   (0 when V is empty).
 * The total loss of Eq. 4 is L_CM + lambda L_geo (lambda = 0.05 in the paper),
 * composed by the caller.  The projection follows the FP32 sequence of
 * cm_flow_eq2 (x' = u + displacement), so the valid set is a fixed function
 * of the inputs; fixed-order reductions.  All pointers are device memory.
 * scratch: 16-byte aligned, cm_geo_scratch_query bytes; the backward reads the
 * valid count the forward left there, so it follows a forward on the same
 * inputs and scratch.  dinv_depth1 is overwritten (its pixels receive the
 * bilinear adjoint, in no fixed order).  Errors: CM_EINVAL, CM_ENOMEM
 * (scratch too small), CM_ECUDA. */
int cm_geo_scratch_query(const cm_camera* cam, size_t* bytes);
int cm_geo_forward(const cm_camera* cam, const float* inv_depth0, const float* inv_depth1, const float* ego6,
                   float dt, void* scratch, size_t scratch_bytes, float* loss_out, void* stream);
int cm_geo_backward(const cm_camera* cam, const float* inv_depth0, const float* inv_depth1, const float* ego6,
                    float dt, const float* dloss, float* dinv_depth0, float* dinv_depth1, float* dego6, void* scratch,
                    size_t scratch_bytes, void* stream);

/* ---- batched evaluation ----
 * Loss and gradient of many windows at once (the batched training step of the
 * paper, supp. "Training": batches of 4-8 event windows on one GPU), with
 * windows of different sizes and event counts in one launch per phase:
 * events are split into chunks of 256 and handed out in window order, pixel
 * passes into per-window tiles, with device-side prefix tables mapping a chunk
 * or tile to its window, so no window is padded.  The phases (zero, flow from
 * depth, warp + splat, loss pass 1 and 2, adjoint, depth / ego gradient and its
 * reduction) run as one CUDA graph, captured at the first cm_batch_run and
 * replayed afterwards.
 *
 * One window of a batch (all pointers are device memory; nbins, reference mode
 * and eps come from the batch's cm_loss_cfg and are shared by all windows). */
typedef struct {
    cm_camera cam;
    cm_events ev;
    const float* flow;      /* [H][W][2] flow input, or NULL: flow from inv_depth + ego6 */
    const float* inv_depth; /* [H][W] (depth input) */
    const float* ego6;      /* [6]    (depth input) */
    float dt_window;        /* window length for the motion field (depth input) */
    const float* dloss;     /* scalar: upstream gradient of this window's loss (required) */
    float* loss_out;        /* scalar: this window's loss (required) */
    float* dflow;           /* [H][W][2] dL/dflow, or NULL (then kept in the plan's memory) */
    float* dinv_depth;      /* [H][W] dL/d(inverse depth), or NULL (depth input only) */
    float* dego6;           /* [6] dL/d(ego-motion), or NULL (depth input only) */
    void* scratch;          /* NULL, or 256-byte-aligned device memory of cm_window_scratch_query bytes
                               holding this window's images of warped events, flow quads, gradient
                               accumulators, reduction buffers and counters (instead of the plan's
                               memory), e.g. kept resident per client stream by a server */
} cm_window;

/* Bytes of a window's own scratch (cm_window.scratch) for this camera and configuration. */
int cm_window_scratch_query(const cm_camera* cam, const cm_loss_cfg* cfg, size_t* bytes);

typedef struct cm_batch cm_batch;

/* Device bytes of a batch plan for these windows (they also fix its
 * capacities: the number of windows and the image sizes it can hold). */
int cm_batch_query(const cm_window* wins, int32_t nwin, const cm_loss_cfg* cfg, size_t* bytes);
/* Lay a plan over caller-owned device memory (256-byte aligned, at least
 * cm_batch_query's size) and point it at `wins`.  The plan owns a small pinned
 * host staging buffer, a capture stream and a few events (host-side); it never
 * allocates device memory.  cfg->splat must be AUTO or ATOMIC.
 * Errors: CM_EINVAL, CM_ENOMEM, CM_ECUDA. */
int cm_batch_create(void* dev_mem, size_t bytes, const cm_window* wins, int32_t nwin, const cm_loss_cfg* cfg,
                    cm_batch** plan);
/* Point the plan at another set of windows.  They must fit its capacities
 * (window count and the per-window image memory, summed); CM_ENOMEM otherwise.
 * Takes effect at the next cm_batch_run, which uploads the new table first. */
int cm_batch_set_windows(cm_batch* plan, const cm_window* wins, int32_t nwin);
/* Forward and backward of every window of the plan, stream-ordered on
 * `stream`: writes each loss_out and the requested gradients. */
int cm_batch_run(cm_batch* plan, void* stream);
/* Synchronises `stream`, then reports how the last run's device-side waits
 * ended: CM_ETIMEOUT when a wait of the persistent step (schedule persist > 0)
 * gave up after its bound (about 4 s; that run's outputs are invalid, the
 * context stays usable), else CM_OK.  CM_ECUDA when the stream reports an error. */
int cm_batch_status(const cm_batch* plan, void* stream);
/* Test hook for the failure path above: window >= 0 makes the persistent
 * step's queue leave out that window's prep pass from the next run on, so its
 * later phases wait until their bound runs out; -1 restores the full queue.
 * Restages the plan's windows; CM_EINVAL outside [-1, capacity). */
int cm_batch_inject_stall(cm_batch* plan, int32_t window);

/* Schedule of a plan: windows are taken `group` at a time (each kernel of the
 * graph covers one group) and the groups run on `chains` concurrent chains of
 * the graph, each chain one group after another; group 0 (with chains 1) puts
 * every window in each kernel.  Few windows in flight keep their images of
 * warped events in L2; several chains overlap each other's tails.  With `bin`
 * the events of each window are first regrouped into a copy in the plan's
 * memory (bin 1: two extra kernels; bin 2: a count inside the prep pass and one
 * extra kernel): bin 1 by 32x32-pixel tile (unordered within a
 * tile), bin 2 by band of 32 image rows with a counting sort that keeps the
 * order of 4096-event super-chunks within a band (with time-ordered input the
 * events of a warp then share their bin).  Either way the events in flight touch a
 * compact region of the flow and of the images.  Windows that do not fit the
 * plan's grouping memory (sized for the windows it was created with), and
 * sensors taller than 4096 rows in bin 2, stay ungrouped.  bin 3 groups by tile
 * as bin 1 and runs the splat and the adjoint one block per tile: the block
 * accumulates the (C, S) pairs of the points landing in its tile (the first 12
 * references; 16 KB of shared memory each) and its pushes into the tile's cell
 * records of dL/dflow, with warp-aggregated shared-memory atomics, and flushes
 * each tile once with 16-byte reductions; points and pushes outside the tile go
 * straight to the images and records.  Every schedule gives the same results
 * up to the order of the floating-point reductions.
 * persist > 0 replaces the graph's kernels by one persistent kernel: its blocks
 * take work items (a pixel tile, a super-chunk, a chunk of 256 events or a
 * loss tile of one phase of one window) from a device queue in which window
 * w + 1's first phase comes persist - 1 phases after window w's, and before an
 * item a block waits (bounded) on the window's per-phase completion counters
 * for the phases it depends on; the graph holds a memset of the queue and the
 * kernel.  There is no launch or graph edge between a window's phases; the
 * stagger sets how many windows are in flight at once.
 * A plan whose cfg->splat is CM_SPLAT_SORT (the deterministic mode) takes
 * only {chains 1..8, group 1, bin 0, persist 0}: each window runs whole
 * through the sort path, one window at a time on each chain.
 * Default: chains 2, group 1, bin 0, persist 0 (bin 3 when the plan's
 * cfg->splat is CM_SPLAT_TILES; min(windows, 8) chains for CM_SPLAT_SORT). */
typedef struct {
    int32_t chains;  /* 1..8 */
    int32_t group;   /* windows per kernel; 0 = all */
    int32_t bin;     /* 0: events in their given order; 1: grouped by tile; 2: by row band, stable;
                        3: grouped by tile, splat and adjoint pushes accumulated per tile in shared memory */
    int32_t persist; /* 0: the graph of per-phase kernels above; 1..8: one persistent kernel (chains 1,
                        group 0, bin 0 or 2) whose device work queue staggers the windows by persist - 1
                        phases (1: each phase over all windows before the next phase) */
} cm_batch_schedule;
int cm_batch_set_schedule(cm_batch* plan, const cm_batch_schedule* schedule);
int cm_batch_get_schedule(const cm_batch* plan, cm_batch_schedule* schedule);
/* Autotuner: times each candidate schedule on the plan's own windows (five
 * replays each, CUDA events on `stream`), keeps the fastest and remembers it
 * for plans of the same shape (window count, first window size, references,
 * event count to a power of two, deterministic or not) for the life of the
 * process.  In the deterministic mode (CM_SPLAT_SORT) the candidates are 1..8
 * chains of one window at a time.  Runs the plan
 * several times (outputs are overwritten); synchronises `stream`. */
int cm_batch_autotune(cm_batch* plan, void* stream, cm_batch_schedule* chosen);
/* Device pointers to window `window`'s per-reference losses (float [R]) and
 * non-empty counts (int32 [R]) of the last run. */
int cm_batch_stats(const cm_batch* plan, int32_t window, const float** loss_r, const int32_t** nnz_r);
int cm_batch_destroy(cm_batch* plan);

/* ---- serving: continuous batching of requests from many event streams ----
 * The paper learns on board from a live event stream (Sec. 3.5, Sec. 4.2);
 * a server evaluates loss + gradient requests from many such streams on one
 * GPU.  It reserves its whole HBM budget at creation (the only device
 * allocation, released by cm_server_destroy) and keeps, inside it, a resident
 * state per client stream (images of warped events, reduction buffers, inverse
 * depth and gradients, an event buffer that grows to the largest request) and
 * one batch plan per lane.  A scheduler thread admits queued requests into
 * batches while a lane is free and their stream's state fits the budget
 * (evicting idle streams' state, least recently used first); batches on
 * different lanes overlap on the device.  Requests of one stream run in
 * submission order, one at a time.  Results are bit-for-bit those of the same
 * request evaluated alone up to the order of FP32 additions of the atomic
 * splat (within the parity tolerances). */
typedef struct {
    size_t hbm_budget;  /* device bytes the server reserves (>= 1 MiB) */
    int32_t max_batch;  /* requests per batch */
    int32_t lanes;      /* batches in flight at once, each on its own CUDA stream (1..16) */
    int32_t max_queue;  /* queued requests before cm_batch_submit returns CM_EBUSY */
    int32_t nbins;      /* B for every request */
    int32_t ref_mode;   /* CM_REF_END or CM_REF_ALL_EDGES */
    float eps;          /* <= 0: 1e-9 */
    int32_t device;     /* CUDA device ordinal */
    int64_t group_events; /* events per batch that a lane regroups by 32-row band before the splat
                             (0: none, the events in their given order).  Each lane reserves about
                             9 bytes per event for the grouped copy; the windows of a batch are
                             grouped in order while that lasts, the rest run ungrouped. */
} cm_server_cfg;

/* One request: a depth + ego-motion window of stream `stream_id`.  All
 * pointers are HOST memory (pinned memory avoids staging copies) that must stay
 * valid until the request is done; outputs are written when it completes. */
typedef struct {
    int32_t stream_id;
    cm_camera cam;
    const int16_t* x;
    const int16_t* y;
    const float* t;
    const int8_t* p;
    int64_t n;
    float t0, t1;
    const float* inv_depth;  /* [H][W] */
    const float* ego6;       /* [6] */
    float dt_window;
    float* loss_out;         /* scalar */
    float* dinv_depth_out;   /* [H][W] or NULL */
    float* dego6_out;        /* [6] or NULL */
} cm_request;

typedef struct {
    int32_t status;      /* CM_OK, or the error that ended the request */
    int32_t batch_size;  /* requests in the batch it ran in */
    double t_submit, t_start, t_done;  /* seconds on a monotonic clock */
} cm_result;

typedef struct {
    int64_t submitted, completed, batches, batched_requests, evictions, memory_waits, queued;
    size_t pool_bytes, pool_used, pool_peak;
} cm_server_stats;

typedef struct cm_server cm_server;

/* Errors: CM_EINVAL, CM_ENOMEM (budget not allocatable), CM_ECUDA. */
int cm_server_create(const cm_server_cfg* cfg, cm_server** server);
/* Non-blocking: queue a request, get its ticket.  CM_EBUSY when the queue is
 * full; CM_ENOMEM when the request could never fit the budget; CM_EINVAL. */
int cm_batch_submit(cm_server* server, const cm_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 and *result filled once the request completed (the
 * ticket is then consumed); CM_ENOTFOUND for an unknown ticket. */
int cm_batch_poll(cm_server* server, uint64_t ticket, cm_result* result, int32_t* done);
/* Wait at most timeout_s seconds for a request; CM_ETIMEOUT when it is not done
 * by then (the ticket stays valid). */
int cm_batch_wait(cm_server* server, uint64_t ticket, double timeout_s, cm_result* result);
int cm_server_get_stats(cm_server* server, cm_server_stats* stats);
/* Stops the scheduler, waits for the batches in flight, frees the budget. */
int cm_server_destroy(cm_server* server);

/* ---- loss and flow gradient without any allocation ----
 * The paper has no counterpart of this entry point; it exists for callers that
 * cannot allocate device memory where they evaluate the loss: a real-time
 * control or on-board learning loop that must not pay an allocator's latency or
 * risk an out-of-memory failure mid-cycle, a plug-in inside a framework that
 * owns all device memory through its own pool, code whose memory was budgeted
 * up front.  It computes what cm_loss_forward followed by cm_loss_backward
 * compute for a flow input, but keeps every intermediate buffer in one fixed
 * device array inside the library instead of a caller workspace.
 *
 *   flow       device float [n_flow_bins][H][W][2] (input)
 *   dloss      device float scalar, the upstream gradient (input)
 *   loss_out   device float scalar (output)
 *   dflow_out  device float [n_flow_bins][H][W][2], overwritten with dL/dflow scaled by dloss (output)
 *
 * Limits and behaviour:
 *   - The fixed array holds CM_STATIC_SCRATCH_BYTES; a window whose images of
 *     warped events and reduction buffers need more (about R x W x H x 16 bytes,
 *     e.g. 346x260 with 11 references fits, 640x480 with 11 does not) is rejected
 *     with CM_ENOMEM before anything is enqueued.
 *   - The call makes no cudaMalloc, cudaFree or other allocating call.  The
 *     first call on each device looks up the array's device address (once, with
 *     that device current), and that first lookup is where the device reserves
 *     the array (the library's module is loaded lazily, on first use): it fails
 *     with CM_ENOMEM when the device has no room for it.  The device then keeps
 *     the array until the process exits.  Make a first call at set-up time, on
 *     every device used (a window of n = 0 events does), before any stream
 *     capture and before the loop that must not fail.
 *   - All calls share the array and it keeps the last call's contents; each
 *     call clears what must start at zero.  Calls whose work overlaps on the
 *     GPU race on the array: order them on one stream or synchronise between them.
 *   - cfg->splat must be CM_SPLAT_AUTO or CM_SPLAT_ATOMIC.
 * Errors: CM_EINVAL (the checks of cm_loss_forward, plus store_warps = 1 or the
 * sort splat), CM_ENOMEM (window too large for the array, or no room for the
 * array on the first call on a device), CM_ECUDA. */
#define CM_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
int cm_loss_grad_static(const cm_camera* cam, const cm_events* ev, const float* flow, int32_t n_flow_bins,
                        const cm_loss_cfg* cfg, const float* dloss, float* loss_out, float* dflow_out,
                        void* stream);

/* ---- tracing ----
 * Per-kernel timing with CUDA events recorded on each kernel's own launch
 * stream (no counterpart in the paper, which reports phase runtimes in its
 * Fig. 2).  While enabled, every library kernel launch is bracketed by two
 * events; cm_profile_collect waits for the recorded events and returns, per
 * kernel name, the number of launches and the summed elapsed milliseconds since
 * the last cm_profile_reset.  Launches captured into a CUDA graph are not timed. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} cm_kernel_stat;

int cm_profile_enable(int on);
/* Fills out[0 .. min(cap, *count) - 1]; *count receives the number of kernel names. */
int cm_profile_collect(cm_kernel_stat* out, int32_t cap, int32_t* count);
int cm_profile_reset(void);
/* Number of kernels the library has enqueued since it was loaded (graph replays
 * count each kernel node). */
int64_t cm_launch_count(void);

/* Measured ceiling of the request-bound kernels (the splat and the adjoint
 * scatter and gather at data-dependent addresses, so the L2's rate of random
 * requests bounds them, not bytes; no counterpart in the paper).  Times random
 * 8-byte vector reductions and random 8-byte loads over `buf` (device memory,
 * 256-byte aligned, at least 16 MiB, about the size of one window's images to
 * stay in L2; overwritten) with CUDA events on `stream`, and returns the best
 * of three timed launches of each, in requests per second.  Synchronises
 * `stream`.  Errors: CM_EINVAL, CM_ECUDA. */
int cm_measure_l2_rates(void* buf, size_t bytes, void* stream, double* red_per_s, double* load_per_s);

#ifdef __cplusplus
}
#endif
#endif /* CM_H */
