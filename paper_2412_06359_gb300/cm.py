"""Torch-facing helpers over the C ABI: device buffers, streams and a
torch.autograd.Function.

PyTorch supplies device memory, the current stream and autograd plumbing;
every step of the loss and its gradient runs in libcm.so's kernels.  The only
work done here is allocating outputs with torch.empty and passing pointers.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _capi as C

REF_END = C.CM_REF_END
REF_ALL = C.CM_REF_ALL_EDGES
SPLAT_AUTO, SPLAT_ATOMIC, SPLAT_SORT, SPLAT_TILES = (C.CM_SPLAT_AUTO, C.CM_SPLAT_ATOMIC, C.CM_SPLAT_SORT,
                                                   C.CM_SPLAT_TILES)


def _require_cuda(t: torch.Tensor, name: str, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def camera(cam) -> C.cm_camera:
    """cm_camera from anything with width, height, fx, fy, cx, cy."""
    return C.cm_camera(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy))


def loss_cfg(nbins: int, ref_mode: int, splat: int = SPLAT_AUTO, eps: float = 1e-9,
             store_warps: bool = False) -> C.cm_loss_cfg:
    """store_warps: the forward keeps every trajectory point for the backward
    ((B+1) x 8 bytes per event) instead of the backward recomputing them."""
    return C.cm_loss_cfg(int(nbins), int(ref_mode), int(splat), int(bool(store_warps)), float(eps))


def n_refs(cfg: C.cm_loss_cfg) -> int:
    return 1 if cfg.ref_mode == REF_END else cfg.nbins + 1


def stream_handle(device=None) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclasses.dataclass
class DeviceEvents:
    """One window of events resident on the GPU (structure of arrays)."""
    x: torch.Tensor  # int16
    y: torch.Tensor  # int16
    t: torch.Tensor  # float32
    p: torch.Tensor  # int8
    t0: float
    t1: float

    @property
    def n(self) -> int:
        return int(self.x.numel())

    @staticmethod
    def from_host(ev, device="cuda", pin: bool = False) -> "DeviceEvents":
        def mv(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            if pin:
                t = t.pin_memory()
            return t.to(device, non_blocking=pin)
        return DeviceEvents(mv(ev.x, np.int16), mv(ev.y, np.int16), mv(ev.t, np.float32), mv(ev.p, np.int8),
                            float(ev.t0), float(ev.t1))

    def c(self) -> C.cm_events:
        if self.n:
            ptrs = (_require_cuda(self.x, "x", torch.int16), _require_cuda(self.y, "y", torch.int16),
                    _require_cuda(self.t, "t", torch.float32), _require_cuda(self.p, "p", torch.int8))
        else:
            ptrs = (None, None, None, None)
        return C.cm_events(*ptrs, self.n, float(self.t0), float(self.t1))


class Workspace:
    """Device memory for one window shape, allocated through torch and laid out
    by cm_workspace_create."""

    def __init__(self, cam, cfg: C.cm_loss_cfg, max_events: int, n_flow_bins: int = 1, device="cuda"):
        self.cam = camera(cam)
        self.cfg = cfg
        self.n_flow_bins = n_flow_bins
        self.nbytes = C.cm_workspace_query(self.cam, cfg, int(max_events), n_flow_bins)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        base = self.buf.data_ptr()
        self.ptr = (base + 255) // 256 * 256
        self.handle = C.cm_workspace_create(self.ptr, self.nbytes, self.cam, cfg, int(max_events), n_flow_bins)

    def stats(self):
        """(loss_r [R] float32, nnz_r [R] int32) of the last forward, copied to host."""
        R = n_refs(self.cfg)
        lr, nz = C.cm_workspace_stats(self.handle)
        off_l, off_n = lr - self.buf.data_ptr(), nz - self.buf.data_ptr()
        loss_r = self.buf[off_l:off_l + 4 * R].view(torch.float32).cpu().numpy()
        nnz_r = self.buf[off_n:off_n + 4 * R].view(torch.int32).cpu().numpy()
        return loss_r, nnz_r

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                C.cm_workspace_destroy(h)
            except Exception:
                pass
            self.handle = None


def flow_from_depth(cam, inv_depth: torch.Tensor, ego: torch.Tensor, dt: float) -> torch.Tensor:
    c = camera(cam)
    out = torch.empty((c.height, c.width, 2), dtype=torch.float32, device=inv_depth.device)
    C.cm_flow_from_depth(c, _require_cuda(inv_depth, "inv_depth", torch.float32), _require_cuda(ego, "ego",
                         torch.float32), float(dt), out.data_ptr(), stream_handle(inv_depth.device))
    return out


def flow_eq2(cam, inv_depth: torch.Tensor, ego: torch.Tensor, dt_bin: float, scale: float) -> torch.Tensor:
    """Per-bin flows [nb, H, W, 2] by the reprojection of Eq. 2: ego [nb, 6]
    holds each bin's (v, w) over dt_bin seconds; the displacement is scaled by
    `scale` (nb for px per window when the bins split the window evenly)."""
    c = camera(cam)
    nb = ego.numel() // 6
    out = torch.empty((nb, c.height, c.width, 2), dtype=torch.float32, device=inv_depth.device)
    C.cm_flow_eq2(c, _require_cuda(inv_depth, "inv_depth", torch.float32), _require_cuda(ego, "ego", torch.float32),
                  nb, float(dt_bin), float(scale), out.data_ptr(), stream_handle(inv_depth.device))
    return out


def flow_eq2_backward(cam, inv_depth: torch.Tensor, ego: torch.Tensor, dt_bin: float, scale: float,
                      dflow: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """Adjoint of flow_eq2: (dL/d inv_depth [H, W], dL/d ego [nb, 6])."""
    c = camera(cam)
    nb = ego.numel() // 6
    dev = inv_depth.device
    scratch = torch.empty(C.cm_flow_eq2_scratch_query(c, nb), dtype=torch.uint8, device=dev)
    drho = torch.empty_like(inv_depth)
    dego = torch.empty((nb, 6), dtype=torch.float32, device=dev)
    C.cm_flow_eq2_backward(c, _require_cuda(inv_depth, "inv_depth", torch.float32),
                           _require_cuda(ego, "ego", torch.float32), nb, float(dt_bin),
                           float(scale), _require_cuda(dflow, "dflow", torch.float32), drho.data_ptr(),
                           dego.data_ptr(), scratch.data_ptr(), scratch.numel(), stream_handle(dev))
    return drho, dego


def event_frame(cam, ev: DeviceEvents) -> torch.Tensor:
    """The network's input frame [2, H, W]: events per pixel, positive then negative."""
    c = camera(cam)
    out = torch.empty((2, c.height, c.width), dtype=torch.float32, device=ev.x.device)
    C.cm_event_frame(c, ev.c(), out.data_ptr(), stream_handle(ev.x.device))
    return out


def rsat(ws: "Workspace", ev: DeviceEvents, flow: torch.Tensor) -> torch.Tensor:
    """RSAT of one window (device tensor [1]): CM loss with `flow` over the CM
    loss of the unwarped events."""
    out = torch.empty(1, dtype=torch.float32, device=flow.device)
    nfb = 1 if flow.dim() == 3 else flow.shape[0]
    C.cm_rsat(ws.cam, ev.c(), _require_cuda(flow, "flow", torch.float32), nfb, ws.cfg, ws.handle, out.data_ptr(),
              stream_handle(flow.device))
    return out


def warp_splat(cam, ev: DeviceEvents, flow: torch.Tensor, cfg: C.cm_loss_cfg,
               ws: "Workspace | None" = None) -> torch.Tensor:
    """IWEs [R, H, W, 4] = (C+, S+, C-, S-) of one window (the sort path needs
    a workspace created with the same configuration)."""
    c = camera(cam)
    nfb = 1 if flow.dim() == 3 else flow.shape[0]
    out = torch.empty((n_refs(cfg), c.height, c.width, 4), dtype=torch.float32, device=flow.device)
    C.cm_warp_splat(c, ev.c(), _require_cuda(flow, "flow", torch.float32), nfb, cfg,
                    None if ws is None else ws.handle, out.data_ptr(), stream_handle(flow.device))
    return out


def loss_forward(ws: Workspace, ev: DeviceEvents, *, flow=None, inv_depth=None, ego=None, dt: float = 0.01,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """CM loss of one window as a device float32 tensor of shape [1]."""
    dev = (flow if flow is not None else inv_depth).device
    loss = out if out is not None else torch.empty(1, dtype=torch.float32, device=dev)
    nfb = 1 if flow is None or flow.dim() == 3 else flow.shape[0]
    C.cm_loss_forward(ws.cam, ev.c(), None if flow is None else _require_cuda(flow, "flow", torch.float32), nfb,
                      None if inv_depth is None else _require_cuda(inv_depth, "inv_depth", torch.float32),
                      None if ego is None else _require_cuda(ego, "ego", torch.float32), float(dt), ws.cfg,
                      ws.handle, loss.data_ptr(), stream_handle(dev))
    return loss


def loss_backward(ws: Workspace, ev: DeviceEvents, dloss: torch.Tensor, *, flow=None, inv_depth=None, ego=None,
                  dt: float = 0.01, want_dflow: bool = True, out: dict | None = None) -> dict:
    """Gradients of dloss * L: {"dflow"} for flow input, {"dinv_depth", "dego"}
    (and "dflow" when want_dflow) for depth input."""
    dev = dloss.device
    res = {} if out is None else out
    if flow is not None:
        nfb = 1 if flow.dim() == 3 else flow.shape[0]
        if "dflow" not in res:
            res["dflow"] = torch.empty_like(flow)
        C.cm_loss_backward(ws.cam, ev.c(), _require_cuda(flow, "flow", torch.float32), nfb, None, None, float(dt),
                           ws.cfg, ws.handle, _require_cuda(dloss, "dloss", torch.float32), res["dflow"].data_ptr(),
                           None, None, stream_handle(dev))
        return res
    H, W = inv_depth.shape
    if want_dflow and "dflow" not in res:
        res["dflow"] = torch.empty((H, W, 2), dtype=torch.float32, device=dev)
    if "dinv_depth" not in res:
        res["dinv_depth"] = torch.empty_like(inv_depth)
    if "dego" not in res:
        res["dego"] = torch.empty(6, dtype=torch.float32, device=dev)
    C.cm_loss_backward(ws.cam, ev.c(), None, 1, _require_cuda(inv_depth, "inv_depth", torch.float32),
                       _require_cuda(ego, "ego", torch.float32), float(dt), ws.cfg, ws.handle,
                       _require_cuda(dloss, "dloss", torch.float32),
                       res["dflow"].data_ptr() if want_dflow else None, res["dinv_depth"].data_ptr(),
                       res["dego"].data_ptr(), stream_handle(dev))
    return res


class CMLossDepth(torch.autograd.Function):
    """L_CM(inv_depth, ego) of one window with the hand-written adjoint as its
    backward (Sec. 3.3); trajectories are recomputed in the backward."""

    @staticmethod
    def forward(ctx, inv_depth, ego, ev: DeviceEvents, ws: Workspace, dt: float):
        inv_depth = inv_depth.contiguous()
        ego = ego.contiguous()
        loss = loss_forward(ws, ev, inv_depth=inv_depth, ego=ego, dt=dt)
        ctx.save_for_backward(inv_depth, ego)
        ctx.ev, ctx.ws, ctx.dt = ev, ws, dt
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        inv_depth, ego = ctx.saved_tensors
        dloss = grad.reshape(1).to(torch.float32).contiguous()
        g = loss_backward(ctx.ws, ctx.ev, dloss, inv_depth=inv_depth, ego=ego, dt=ctx.dt, want_dflow=False)
        return g["dinv_depth"], g["dego"], None, None, None


class CMLossFlow(torch.autograd.Function):
    """L_CM(flow) of one window; backward gives dL/dflow."""

    @staticmethod
    def forward(ctx, flow, ev: DeviceEvents, ws: Workspace):
        flow = flow.contiguous()
        loss = loss_forward(ws, ev, flow=flow)
        ctx.save_for_backward(flow)
        ctx.ev, ctx.ws = ev, ws
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        (flow,) = ctx.saved_tensors
        dloss = grad.reshape(1).to(torch.float32).contiguous()
        g = loss_backward(ctx.ws, ctx.ev, dloss, flow=flow)
        return g["dflow"], None, None


class CMLossEq2(torch.autograd.Function):
    """L_CM of one window whose per-bin flows come from inverse depth and one
    pose per bin through Eq. 2 (ego [nb, 6], nb = 1 or the window's bins);
    backward: the CM adjoint to dL/dflow of every bin, then the Eq. 2 adjoint to
    dL/d inverse depth and dL/d ego."""

    @staticmethod
    def forward(ctx, inv_depth, ego, ev: DeviceEvents, ws: Workspace, dt_bin: float, scale: float):
        inv_depth = inv_depth.contiguous()
        ego = ego.contiguous()
        flow = flow_eq2(ws.cam, inv_depth, ego, dt_bin, scale)
        if flow.shape[0] == 1:
            flow = flow[0]
        loss = loss_forward(ws, ev, flow=flow)
        ctx.save_for_backward(inv_depth, ego, flow)
        ctx.ev, ctx.ws, ctx.dt, ctx.scale = ev, ws, dt_bin, scale
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        inv_depth, ego, flow = ctx.saved_tensors
        dloss = grad.reshape(1).to(torch.float32).contiguous()
        g = loss_backward(ctx.ws, ctx.ev, dloss, flow=flow)
        drho, dego = flow_eq2_backward(ctx.ws.cam, inv_depth, ego, ctx.dt, ctx.scale, g["dflow"])
        return drho, dego.reshape(ego.shape), None, None, None, None


LAMBDA_GEO = 0.05  # weight of the geometry-consistency term in the total loss (Eq. 4; supp. "Training")


class GeoLoss(torch.autograd.Function):
    """Geometry-consistency loss (Eq. 3) between two views' inverse depths
    under the camera motion ego [6] over dt; backward to both inverse depths
    and the motion."""

    @staticmethod
    def forward(ctx, inv_depth0, inv_depth1, ego, cam, dt: float):
        c = camera(cam)
        r0, r1, e = inv_depth0.contiguous(), inv_depth1.contiguous(), ego.contiguous()
        dev = r0.device
        scratch = torch.empty(C.cm_geo_scratch_query(c), dtype=torch.uint8, device=dev)
        loss = torch.empty(1, dtype=torch.float32, device=dev)
        C.cm_geo_forward(c, _require_cuda(r0, "inv_depth0", torch.float32), _require_cuda(r1, "inv_depth1",
                         torch.float32), _require_cuda(e, "ego", torch.float32), float(dt), scratch.data_ptr(),
                         scratch.numel(), loss.data_ptr(), stream_handle(dev))
        ctx.save_for_backward(r0, r1, e, scratch)
        ctx.cam, ctx.dt = c, dt
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        r0, r1, e, scratch = ctx.saved_tensors
        dloss = grad.reshape(1).to(torch.float32).contiguous()
        d0, d1 = torch.empty_like(r0), torch.empty_like(r1)
        de = torch.empty(6, dtype=torch.float32, device=r0.device)
        C.cm_geo_backward(ctx.cam, r0.data_ptr(), r1.data_ptr(), e.data_ptr(), float(ctx.dt), dloss.data_ptr(),
                          d0.data_ptr(), d1.data_ptr(), de.data_ptr(), scratch.data_ptr(), scratch.numel(),
                          stream_handle(r0.device))
        return d0, d1, de, None, None


def geo_loss(cam, inv_depth0, inv_depth1, ego, dt: float):
    """Differentiable geometry-consistency loss (Eq. 3)."""
    return GeoLoss.apply(inv_depth0, inv_depth1, ego, cam, dt)


def cm_loss(ev: DeviceEvents, ws: Workspace, *, flow=None, inv_depth=None, ego=None, dt: float = 0.01):
    """Differentiable CM loss: pass flow, or inv_depth and ego."""
    if flow is not None:
        return CMLossFlow.apply(flow, ev, ws)
    return CMLossDepth.apply(inv_depth, ego, ev, ws, dt)


class BatchPlan:
    """A batch of windows evaluated by cm_batch_run (one persistent launch per
    phase, replayed from a CUDA graph).  Each entry of `windows` is a dict with
    cam, ev (DeviceEvents) and either flow or inv_depth + ego (+ dt).  Outputs
    are allocated here: loss [nwin] and, per window, dflow (flow input) or
    dinv_depth and dego (depth input)."""

    def __init__(self, windows: list, cfg: C.cm_loss_cfg, device="cuda", dloss: torch.Tensor | None = None,
                 want_dflow: bool = False):
        self.cfg = cfg
        self.device = device
        self.loss = torch.empty(len(windows), dtype=torch.float32, device=device)
        self.dloss = dloss if dloss is not None else torch.ones(len(windows), dtype=torch.float32, device=device)
        self.want_dflow = want_dflow
        self.keep = []
        self.structs = self._structs(windows)
        self.nbytes = C.cm_batch_query(self.structs, cfg)
        self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        self.ptr = (self.buf.data_ptr() + 255) // 256 * 256
        self.handle = C.cm_batch_create(self.ptr, self.nbytes, self.structs, cfg)

    def _structs(self, windows):
        # every output lives in one float32 arena (self.output_arena), in window
        # order, so that a caller can fetch all of them with one copy
        sizes = []
        for w in windows:
            cam = camera(w["cam"])
            hw = cam.width * cam.height
            if w.get("flow") is not None:
                sizes.append([("dflow", (cam.height, cam.width, 2))])
            else:
                e = [("dinv_depth", (cam.height, cam.width)), ("dego", (6,))]
                if self.want_dflow:
                    e.append(("dflow", (cam.height, cam.width, 2)))
                sizes.append(e)
        total = sum(((int(np.prod(shape)) + 63) // 64) * 64 for e in sizes for _, shape in e)
        self.output_arena = torch.empty(max(total, 1), dtype=torch.float32, device=self.device)
        out = []
        self.outputs = []
        self.keep = [windows]
        off = 0
        for i, (w, e) in enumerate(zip(windows, sizes)):
            cam = camera(w["cam"])
            s = C.cm_window()
            s.cam = cam
            s.ev = w["ev"].c()
            s.dloss = self.dloss.data_ptr() + 4 * i
            s.loss_out = self.loss.data_ptr() + 4 * i
            o = {}
            for name, shape in e:
                n = int(np.prod(shape))
                o[name] = self.output_arena[off:off + n].view(shape)
                off += (n + 63) // 64 * 64
            if w.get("flow") is not None:
                s.flow = _require_cuda(w["flow"], "flow", torch.float32)
                s.dflow = o["dflow"].data_ptr()
            else:
                s.inv_depth = _require_cuda(w["inv_depth"], "inv_depth", torch.float32)
                s.ego6 = _require_cuda(w["ego"], "ego", torch.float32)
                s.dt_window = float(w.get("dt", 0.01))
                s.dinv_depth = o["dinv_depth"].data_ptr()
                s.dego6 = o["dego"].data_ptr()
                if self.want_dflow:
                    s.dflow = o["dflow"].data_ptr()
            self.outputs.append(o)
            out.append(s)
        return out

    def set_windows(self, windows: list):
        if len(windows) > self.loss.numel():
            raise ValueError("more windows than the plan holds")
        self.structs = self._structs(windows)
        C.cm_batch_set_windows(self.handle, self.structs)

    def run(self):
        C.cm_batch_run(self.handle, stream_handle(self.buf.device))

    def status(self) -> int:
        """Waits for the plan's stream; CM_OK, or CM_ETIMEOUT when a bounded
        device wait of the last run (persistent step) gave up."""
        return C.cm_batch_status(self.handle, stream_handle(self.buf.device))

    def inject_stall(self, window: int):
        """Test hook: the persistent step's queue leaves out `window`'s prep
        pass from the next run on (-1 restores it)."""
        C.cm_batch_inject_stall(self.handle, window)

    def set_schedule(self, chains: int, group: int, bin: int = 0, persist: int = 0):
        """chains: concurrent kernel chains; group: windows per kernel (0: one
        kernel over every window); bin: 1 to group each window's events by
        32x32 pixel tile before the splat, 2 by band of 32 rows keeping the
        order of 4096-event super-chunks within a band, 3 by tile with the
        splat and the adjoint's pushes accumulated per tile in shared memory;
        persist > 0: one persistent kernel with a device work queue that
        staggers the windows by persist - 1 phases (chains 1, group 0, bin 0
        or 2; persist 1 runs each phase over all windows before the next)."""
        C.cm_batch_set_schedule(self.handle, chains, group, bin, persist)

    def schedule(self) -> tuple[int, int, int, int]:
        return C.cm_batch_get_schedule(self.handle)

    def autotune(self) -> tuple[int, int, int, int]:
        """Pick the fastest schedule for these windows (runs the plan several times)."""
        return C.cm_batch_autotune(self.handle, stream_handle(self.buf.device))

    def stats(self, i: int):
        R = n_refs(self.cfg)
        lr, nz = C.cm_batch_stats(self.handle, i)
        base = self.buf.data_ptr()
        loss_r = self.buf[lr - base:lr - base + 4 * R].view(torch.float32).cpu().numpy()
        nnz_r = self.buf[nz - base:nz - base + 4 * R].view(torch.int32).cpu().numpy()
        return loss_r, nnz_r

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                C.cm_batch_destroy(h)
            except Exception:
                pass
            self.handle = None
