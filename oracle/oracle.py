"""ctypes front end of the plain FP64 CPU oracle in cm_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline / reference legs of bench.py.  The CUDA product path never
imports this module.

Each function cites the part of the paper it follows; the C file states the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cm_oracle.c")
LIB = os.path.join(HERE, "libcm_oracle.so")
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]

REF_END = 0
REF_ALL = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Args(ctypes.Structure):
    _fields_ = [
        ("W", ctypes.c_int32), ("H", ctypes.c_int32), ("nbins", ctypes.c_int32),
        ("ref_mode", ctypes.c_int32), ("n_flow_bins", ctypes.c_int32), ("pos_f32", ctypes.c_int32),
        ("branch_mode", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t", ctypes.c_void_p), ("p", ctypes.c_void_p),
        ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("eps", ctypes.c_double), ("dloss", ctypes.c_double),
        ("flow", ctypes.c_void_p), ("flow32", ctypes.c_void_p),
        ("br_cell", ctypes.c_void_p), ("br_supp", ctypes.c_void_p), ("br_valid", ctypes.c_void_p),
        ("br_bin", ctypes.c_void_p),
        ("loss", ctypes.c_void_p), ("loss_r", ctypes.c_void_p), ("nnz_r", ctypes.c_void_p),
        ("iwe", ctypes.c_void_p), ("dflow", ctypes.c_void_p), ("valid", ctypes.c_void_p), ("pos", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            d, i, f, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p
            l.orc_flow_from_depth.argtypes = [i, i, d, d, d, d, vp, vp, d, vp]
            l.orc_flow_from_depth_f32.argtypes = [i, i, f, f, f, f, vp, vp, f, vp]
            l.orc_depth_ego_grad.argtypes = [i, i, d, d, d, d, vp, vp, d, vp, vp, vp]
            l.orc_flow_eq2.argtypes = [i, i, d, d, d, d, vp, vp, d, vp]
            l.orc_flow_eq2_bins.argtypes = [i, i, d, d, d, d, vp, vp, i, d, d, vp]
            l.orc_flow_eq2_bins_f32.argtypes = [i, i, f, f, f, f, vp, vp, i, f, f, vp]
            l.orc_flow_eq2_grad.argtypes = [i, i, d, d, d, d, vp, vp, i, d, d, vp, vp, vp]
            l.orc_event_frame.argtypes = [i, i, ctypes.c_int64, vp, vp, vp, vp]
            l.orc_geo_proj_f32.argtypes = [i, i, f, f, f, f, vp, vp, vp, f, vp, vp, vp]
            l.orc_geo.argtypes = [i, i, d, d, d, d, vp, vp, vp, d, vp, vp, vp, d, vp, vp, vp, vp]
            l.orc_geo.restype = d
            l.orc_cm.argtypes = [ctypes.POINTER(_Args)]
            l.orc_cm.restype = ctypes.c_int
            _lib = l
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
# S1 / S7: geometry (Sec. 3.2, Eq. 2)


def flow_from_depth(cam, inv_depth, ego, dt):
    """Rigid motion field with intrinsics, FP64 (Sec. 3.2, Eq. 2 in its
    instantaneous form).  Returns [H, W, 2] float64, px per window."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64)
    out = np.empty((cam.height, cam.width, 2), np.float64)
    lib().orc_flow_from_depth(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), float(dt), _p(out))
    return out


def flow_from_depth_f32(cam, inv_depth, ego, dt):
    """The same motion field in FP32 with the kernels' operation order; it
    feeds the FP32 trajectory that takes the floor/mask/support decisions."""
    rho = _c(inv_depth, np.float32)
    e = _c(ego, np.float32)
    out = np.empty((cam.height, cam.width, 2), np.float32)
    lib().orc_flow_from_depth_f32(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e),
                                  float(np.float32(dt)), _p(out))
    return out


def flow_eq2(cam, inv_depth, ego, dt):
    """Eq. 2 literally: reprojection through [R | t] with R = Rodrigues(-w dt),
    t = -v dt and depth 1/rho.  Returns the pixel displacement, FP64."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64)
    out = np.empty((cam.height, cam.width, 2), np.float64)
    lib().orc_flow_eq2(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), float(dt), _p(out))
    return out


def flow_eq2_bins(cam, inv_depth, ego, dt_bin, scale):
    """Eq. 2 with one pose per bin: ego [nb, 6] = (v, w) of each bin over
    dt_bin seconds; flow [nb, H, W, 2] = scale x the pixel displacement, FP64."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64).reshape(-1, 6)
    nb = e.shape[0]
    out = np.empty((nb, cam.height, cam.width, 2), np.float64)
    lib().orc_flow_eq2_bins(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), nb,
                            float(dt_bin), float(scale), _p(out))
    return out


def flow_eq2_bins_f32(cam, inv_depth, ego, dt_bin, scale):
    """The same in FP32 with the kernels' operation sequence (the values that
    decide the FP32 trajectory when these flows drive it)."""
    rho = _c(inv_depth, np.float32)
    e = _c(ego, np.float32).reshape(-1, 6)
    nb = e.shape[0]
    out = np.empty((nb, cam.height, cam.width, 2), np.float32)
    lib().orc_flow_eq2_bins_f32(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), nb,
                                float(dt_bin), float(scale), _p(out))
    return out


def flow_eq2_grad(cam, inv_depth, ego, dt_bin, scale, dflow):
    """Adjoint of flow_eq2_bins: dL/dflow [nb, H, W, 2] -> (dL/d inv_depth [H, W], dL/d ego [nb, 6])."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64).reshape(-1, 6)
    nb = e.shape[0]
    g = _c(dflow, np.float64).reshape(nb, cam.height, cam.width, 2)
    drho = np.empty((cam.height, cam.width), np.float64)
    dego = np.empty((nb, 6), np.float64)
    lib().orc_flow_eq2_grad(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), nb,
                            float(dt_bin), float(scale), _p(g), _p(drho), _p(dego))
    return drho, dego


def geo_proj_f32(cam, inv_depth0, inv_depth1, ego, dt):
    """The decisions of the geometry-consistency loss in the kernels' FP32
    sequence: the projection of every pixel of view 0 into view 1 [H, W, 2],
    the valid flags [H, W] and the sign of a - b [H, W]."""
    r0, r1 = _c(inv_depth0, np.float32), _c(inv_depth1, np.float32)
    e = _c(ego, np.float32)
    proj = np.empty((cam.height, cam.width, 2), np.float32)
    ok = np.empty((cam.height, cam.width), np.uint8)
    sgn = np.empty((cam.height, cam.width), np.int8)
    lib().orc_geo_proj_f32(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(r0), _p(r1), _p(e), float(dt),
                           _p(proj), _p(ok), _p(sgn))
    return proj, ok, sgn


def geo(cam, inv_depth0, inv_depth1, ego, dt, *, decisions=None, grad=False, dloss=1.0):
    """Geometry-consistency loss (Eq. 3) between the depth of view 0 moved by
    the camera motion (v, w) over dt and the depth of view 1, FP64 on the
    FP32 decisions (computed here unless given).  Returns loss, count (valid pixels) and, with grad, dL/d
    inv_depth0 [H, W], dL/d inv_depth1 [H, W], dL/d ego [6] for dloss.
    decisions: (proj, ok, sign) of geo_proj_f32."""
    if decisions is None:
        decisions = geo_proj_f32(cam, inv_depth0, inv_depth1, ego, dt)
    proj, ok, sgn = decisions
    r0, r1 = _c(inv_depth0, np.float64), _c(inv_depth1, np.float64)
    e = _c(ego, np.float64)
    cnt = ctypes.c_int64()
    out = {}
    if grad:
        out["dinv_depth0"] = np.empty((cam.height, cam.width))
        out["dinv_depth1"] = np.empty((cam.height, cam.width))
        out["dego"] = np.empty(6)
        g0, g1, ge = _p(out["dinv_depth0"]), _p(out["dinv_depth1"]), _p(out["dego"])
    else:
        g0 = g1 = ge = None
    out["loss"] = lib().orc_geo(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(r0), _p(r1), _p(e),
                                float(dt), _p(_c(proj, np.float32)), _p(_c(ok, np.uint8)), _p(_c(sgn, np.int8)),
                                float(dloss),
                                ctypes.byref(cnt), g0, g1, ge)
    out["count"] = cnt.value
    return out


def event_frame(events, width, height):
    """Per-pixel event counts [2, H, W] (channel 0 positive, 1 negative), the
    network's input frame."""
    out = np.empty((2, height, width), np.float64)
    x, y, p = _c(events.x, np.int16), _c(events.y, np.int16), _c(events.p, np.int8)
    lib().orc_event_frame(width, height, events.n, _p(x), _p(y), _p(p), _p(out))
    return out


def rsat(events, flow, *, width, height, nbins, ref_mode, eps=1e-9, flow32=None):
    """Ratio of squared average timestamps: the CM loss with `flow` over the CM
    loss with zero flow (the unwarped events), same references; 0 when the
    zero-flow loss is 0 (no event in the image)."""
    fl = np.asarray(flow, np.float64)
    a = cm(events, fl, width=width, height=height, nbins=nbins, ref_mode=ref_mode, eps=eps, flow32=flow32)["loss"]
    b = cm(events, np.zeros((height, width, 2)), width=width, height=height, nbins=nbins, ref_mode=ref_mode,
           eps=eps)["loss"]
    return a / b if b > 0 else 0.0


def depth_ego_grad(cam, inv_depth, ego, dt, dflow):
    """Chain rule from dL/dflow [H, W, 2] to dL/d(inv_depth) [H, W] and dL/d(ego) [6]."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64)
    g = _c(dflow, np.float64).reshape(cam.height, cam.width, 2)
    drho = np.empty((cam.height, cam.width), np.float64)
    dego = np.empty(6, np.float64)
    lib().orc_depth_ego_grad(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), float(dt),
                             _p(g), _p(drho), _p(dego))
    return drho, dego


# ---------------------------------------------------------------------------
# S2-S6: warp, mask, splat, loss, gradient (Sec. 3.1, Eq. 1; Sec. 3.3)


def n_refs(nbins, ref_mode):
    return 1 if ref_mode == REF_END else nbins + 1


def cm(events, flow, *, width, height, nbins, ref_mode, eps=1e-9, positions="f32", flow32=None,
       grad=False, dloss=1.0, want_iwe=False, want_pos=False, record=False, replay=None):
    """Contrast-maximisation loss of one window (and its flow gradient).

    events: synth.Events (x, y int16; t float32; p int8; t0, t1)
    flow:   [nfb, H, W, 2] or [H, W, 2] values (nfb = 1 or nbins), px per window
    positions: "f32" takes the trajectory in the kernels' FP32 arithmetic (the
        floor / mask / support decisions), "f64" is the plain FP64 definition
    flow32: the FP32 flow driving the FP32 trajectory (default: flow cast to FP32)
    record: return the branch (bins, cells, supports, validity) for replay
    replay: a recorded branch; positions are then FP64 with those decisions frozen
    Returns a dict with loss, loss_r [R], nnz_r [R], valid [n] and optionally
    iwe [R, H, W, 4] = (C+, S+, C-, S-), dflow (same shape as flow), pos [n, B+1, 2].
    """
    W, H = int(width), int(height)
    fl = _c(flow, np.float64)
    nfb = 1 if fl.ndim == 3 else fl.shape[0]
    fl = fl.reshape(nfb, H, W, 2)
    R = n_refs(nbins, ref_mode)
    n = events.n
    x = _c(events.x, np.int16)
    y = _c(events.y, np.int16)
    t = _c(events.t, np.float32)
    p = _c(events.p, np.int8)
    f32 = None
    pos_f32 = positions == "f32" and replay is None
    if pos_f32:
        f32 = _c(flow32 if flow32 is not None else fl, np.float32).reshape(nfb, H, W, 2)
    out = {
        "loss": np.zeros(1), "loss_r": np.zeros(R), "nnz_r": np.zeros(R, np.int64),
        "valid": np.zeros(n, np.uint8),
    }
    a = _Args()
    a.W, a.H, a.nbins, a.ref_mode, a.n_flow_bins = W, H, int(nbins), int(ref_mode), nfb
    a.pos_f32 = 1 if pos_f32 else 0
    a.n = n
    a.x, a.y, a.t, a.p = _p(x), _p(y), _p(t), _p(p)
    a.t0, a.t1 = float(np.float32(events.t0)), float(np.float32(events.t1))
    a.eps, a.dloss = float(eps), float(dloss)
    a.flow, a.flow32 = _p(fl), _p(f32)
    br = None
    if record or replay is not None:
        if replay is not None:
            br = replay
            a.branch_mode = 2
        else:
            br = {"cell": np.zeros((n, nbins + 1, 2), np.int32), "supp": np.zeros((n, nbins + 1), np.uint8),
                  "valid": np.zeros(n, np.uint8), "bin": np.zeros(n, np.int32)}
            a.branch_mode = 1
        a.br_cell, a.br_supp, a.br_valid, a.br_bin = _p(br["cell"]), _p(br["supp"]), _p(br["valid"]), _p(br["bin"])
    a.loss, a.loss_r, a.nnz_r, a.valid = _p(out["loss"]), _p(out["loss_r"]), _p(out["nnz_r"]), _p(out["valid"])
    if want_iwe:
        out["iwe"] = np.zeros((R, H, W, 4))
        a.iwe = _p(out["iwe"])
    if grad:
        out["dflow"] = np.zeros((nfb, H, W, 2))
        a.dflow = _p(out["dflow"])
    if want_pos:
        out["pos"] = np.zeros((n, nbins + 1, 2))
        a.pos = _p(out["pos"])
    st = lib().orc_cm(ctypes.byref(a))
    if st != 0:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    out["loss"] = float(out["loss"][0])
    if grad and np.ndim(flow) == 3:
        out["dflow"] = out["dflow"][0]
    if record:
        out["branch"] = br
    return out


def cm_depth(events, cam, inv_depth, ego, dt, *, nbins, ref_mode, eps=1e-9, positions="f32", grad=False,
             dloss=1.0, **kw):
    """Loss of one window whose flow comes from inverse depth and ego-motion
    (Sec. 3.2 then Sec. 3.1); with grad, also dL/d(inv_depth) and dL/d(ego)."""
    f64 = flow_from_depth(cam, inv_depth, ego, dt)
    f32 = flow_from_depth_f32(cam, inv_depth, ego, dt) if positions == "f32" else None
    out = cm(events, f64, width=cam.width, height=cam.height, nbins=nbins, ref_mode=ref_mode, eps=eps,
             positions=positions, flow32=f32, grad=grad, dloss=dloss, **kw)
    out["flow"] = f64
    if grad:
        out["dinv_depth"], out["dego"] = depth_ego_grad(cam, inv_depth, ego, dt, out["dflow"])
    return out


def cm_window(win, **kw):
    """Oracle on a synth.Window (flow input or depth + ego input)."""
    if win.flow is not None:
        return cm(win.events, win.flow, width=win.cam.width, height=win.cam.height, nbins=win.nbins,
                  ref_mode=win.ref_mode, **kw)
    return cm_depth(win.events, win.cam, win.inv_depth, win.ego, win.dt, nbins=win.nbins,
                    ref_mode=win.ref_mode, **kw)
