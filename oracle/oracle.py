"""ctypes front end of the plain FP64 CPU oracle in cm_oracle.c.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline / reference legs of bench.py.  The CUDA product path never
imports this module.

Each function cites the part of the paper it follows; the C file states the
readings taken where the paper is silent.  Every value is computed in FP64.
The *_bounds functions flag the decisions (cells, supports, mask, bins, the
valid set and branch of Eq. 3) that an FP32 evaluation could take the other
way, and give the interval of the loss over those outcomes.
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
SAFETY = 4.0  # margin of a flagged decision: SAFETY x the FP32 error bound of its input

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
        ("ref_mode", ctypes.c_int32), ("n_flow_bins", ctypes.c_int32), ("branch_mode", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t", ctypes.c_void_p), ("p", ctypes.c_void_p),
        ("t0", ctypes.c_double), ("t1", ctypes.c_double), ("eps", ctypes.c_double), ("dloss", ctypes.c_double),
        ("flow", ctypes.c_void_p),
        ("br_cell", ctypes.c_void_p), ("br_supp", ctypes.c_void_p), ("br_valid", ctypes.c_void_p),
        ("br_bin", ctypes.c_void_p),
        ("loss", ctypes.c_void_p), ("loss_r", ctypes.c_void_p), ("nnz_r", ctypes.c_void_p),
        ("iwe", ctypes.c_void_p), ("dflow", ctypes.c_void_p), ("valid", ctypes.c_void_p), ("pos", ctypes.c_void_p),
    ]


class _Bounds(ctypes.Structure):
    _fields_ = [
        ("safety", ctypes.c_double), ("pad_", ctypes.c_int32), ("pad2_", ctypes.c_int32),
        ("eflow", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("err", ctypes.c_void_p),
        ("loss_lo", ctypes.c_void_p), ("loss_hi", ctypes.c_void_p),
        ("loss_r_lo", ctypes.c_void_p), ("loss_r_hi", ctypes.c_void_p),
        ("nnz_lo", ctypes.c_void_p), ("nnz_hi", ctypes.c_void_p),
        ("counts", ctypes.c_int64 * 4),
    ]


class _GeoDec(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("pad_", ctypes.c_int32), ("cell", ctypes.c_void_p),
                ("ok", ctypes.c_void_p), ("sgn", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            d, i, f, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p
            l.orc_flow_from_depth.argtypes = [i, i, d, d, d, d, vp, vp, d, vp]
            l.orc_flow_error_bound.argtypes = [i, i, d, d, d, d, vp, vp, d, vp]
            l.orc_depth_ego_grad.argtypes = [i, i, d, d, d, d, vp, vp, d, vp, vp, vp]
            l.orc_flow_eq2.argtypes = [i, i, d, d, d, d, vp, vp, d, vp]
            l.orc_flow_eq2_bins.argtypes = [i, i, d, d, d, d, vp, vp, i, d, d, vp]
            l.orc_flow_eq2_error_bound.argtypes = [i, i, d, d, d, d, vp, vp, i, d, d, vp]
            l.orc_flow_eq2_grad.argtypes = [i, i, d, d, d, d, vp, vp, i, d, d, vp, vp, vp]
            l.orc_event_frame.argtypes = [i, i, ctypes.c_int64, vp, vp, vp, vp]
            l.orc_geo.argtypes = [i, i, d, d, d, d, vp, vp, vp, d, ctypes.POINTER(_GeoDec), d, vp, vp, vp, vp]
            l.orc_geo.restype = d
            l.orc_geo_bounds.argtypes = [i, i, d, d, d, d, vp, vp, vp, d, d, vp, vp, vp, vp, vp]
            l.orc_geo_bounds.restype = ctypes.c_int64
            l.orc_cm.argtypes = [ctypes.POINTER(_Args)]
            l.orc_cm.restype = ctypes.c_int
            l.orc_cm_bounds.argtypes = [ctypes.POINTER(_Args), ctypes.POINTER(_Bounds)]
            l.orc_cm_bounds.restype = ctypes.c_int
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


def flow_error_bound(cam, inv_depth, ego, dt):
    """Bound on |FP32 flow - flow| per pixel [H, W] for the motion field
    evaluated in single precision (the larger of the two components)."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64)
    out = np.empty((cam.height, cam.width), np.float64)
    lib().orc_flow_error_bound(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), float(dt),
                               _p(out))
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


def flow_eq2_error_bound(cam, inv_depth, ego, dt_bin, scale):
    """Bound on |FP32 flow - flow| per bin and pixel [nb, H, W] for
    flow_eq2_bins evaluated in single precision without cancellation."""
    rho = _c(inv_depth, np.float64)
    e = _c(ego, np.float64).reshape(-1, 6)
    nb = e.shape[0]
    out = np.empty((nb, cam.height, cam.width), np.float64)
    lib().orc_flow_eq2_error_bound(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(rho), _p(e), nb,
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


def geo(cam, inv_depth0, inv_depth1, ego, dt, *, grad=False, dloss=1.0, record=False, replay=None):
    """Geometry-consistency loss (Eq. 3) between the depth of view 0 moved by
    the camera motion (v, w) over dt and the depth of view 1, FP64.  Returns
    loss, count (valid pixels) and, with grad, dL/d inv_depth0 [H, W], dL/d
    inv_depth1 [H, W], dL/d ego [6] for dloss.  record: also return the
    decisions (cells, valid flags, signs of a - b); replay: such decisions,
    frozen (positions FP64), for differences on one branch."""
    r0, r1 = _c(inv_depth0, np.float64), _c(inv_depth1, np.float64)
    e = _c(ego, np.float64)
    HW = cam.width * cam.height
    dec = None
    if record or replay is not None:
        rec = replay if replay is not None else {"cell": np.zeros((HW, 2), np.int32), "ok": np.zeros(HW, np.uint8),
                                                 "sgn": np.zeros(HW, np.int8)}
        dec = _GeoDec(2 if replay is not None else 1, 0, _p(rec["cell"]), _p(rec["ok"]), _p(rec["sgn"]))
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
                                float(dt), ctypes.byref(dec) if dec is not None else None, float(dloss),
                                ctypes.byref(cnt), g0, g1, ge)
    out["count"] = cnt.value
    if record:
        out["decisions"] = rec
    return out


def geo_bounds(cam, inv_depth0, inv_depth1, ego, dt, *, safety=SAFETY):
    """Straddles of the geometry-consistency loss for an FP32 evaluation:
    flags [H, W] (bit 0 sample cell, bit 1 valid set, bit 2 branch of
    |a - b|), and the valid count and loss over every outcome of the bit-1
    decisions (count_lo/hi, loss_lo/hi)."""
    r0, r1 = _c(inv_depth0, np.float64), _c(inv_depth1, np.float64)
    e = _c(ego, np.float64)
    flags = np.zeros((cam.height, cam.width), np.uint8)
    clo, chi = ctypes.c_int64(), ctypes.c_int64()
    llo, lhi = ctypes.c_double(), ctypes.c_double()
    nf = lib().orc_geo_bounds(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, _p(r0), _p(r1), _p(e),
                              float(dt), float(safety), _p(flags), ctypes.byref(clo), ctypes.byref(chi),
                              ctypes.byref(llo), ctypes.byref(lhi))
    return {"flags": flags, "flagged": int(nf), "count_lo": clo.value, "count_hi": chi.value,
            "loss_lo": llo.value, "loss_hi": lhi.value}


def event_frame(events, width, height):
    """Per-pixel event counts [2, H, W] (channel 0 positive, 1 negative), the
    network's input frame."""
    out = np.empty((2, height, width), np.float64)
    x, y, p = _c(events.x, np.int16), _c(events.y, np.int16), _c(events.p, np.int8)
    lib().orc_event_frame(width, height, events.n, _p(x), _p(y), _p(p), _p(out))
    return out


def rsat(events, flow, *, width, height, nbins, ref_mode, eps=1e-9, bounds=False, eflow=None):
    """Ratio of squared average timestamps: the CM loss with `flow` over the CM
    loss with zero flow (the unwarped events), same references; 0 when the
    zero-flow loss is 0 (no event in the image).  With bounds, returns
    (value, lo, hi): the interval over the flagged decisions of the numerator
    (the zero-flow positions are exact integers, so its loss has none)."""
    fl = np.asarray(flow, np.float64)
    kw = dict(width=width, height=height, nbins=nbins, ref_mode=ref_mode, eps=eps)
    a = cm(events, fl, **kw)["loss"]
    b = cm(events, np.zeros((height, width, 2)), **kw)["loss"]
    v = a / b if b > 0 else 0.0
    if not bounds:
        return v
    bo = cm_bounds(events, fl, eflow=eflow, **kw)
    if b <= 0:
        return v, 0.0, 0.0
    return v, bo["loss_lo"] / b, bo["loss_hi"] / b


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


def _args(events, fl, W, H, nbins, ref_mode, eps, dloss):
    a = _Args()
    nfb = fl.shape[0]
    a.W, a.H, a.nbins, a.ref_mode, a.n_flow_bins = W, H, int(nbins), int(ref_mode), nfb
    arrs = (_c(events.x, np.int16), _c(events.y, np.int16), _c(events.t, np.float32), _c(events.p, np.int8))
    a.n = events.n
    a.x, a.y, a.t, a.p = (_p(v) for v in arrs)
    a.t0, a.t1 = float(np.float32(events.t0)), float(np.float32(events.t1))
    a.eps, a.dloss = float(eps), float(dloss)
    a.flow = _p(fl)
    return a, arrs


def cm(events, flow, *, width, height, nbins, ref_mode, eps=1e-9, grad=False, dloss=1.0, want_iwe=False,
       want_pos=False, record=False, replay=None):
    """Contrast-maximisation loss of one window (and its flow gradient), FP64.

    events: synth.Events (x, y int16; t float32; p int8; t0, t1)
    flow:   [nfb, H, W, 2] or [H, W, 2] values (nfb = 1 or nbins), px per window
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
    out = {
        "loss": np.zeros(1), "loss_r": np.zeros(R), "nnz_r": np.zeros(R, np.int64),
        "valid": np.zeros(n, np.uint8),
    }
    a, _keep = _args(events, fl, W, H, nbins, ref_mode, eps, dloss)
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


def cm_bounds(events, flow, *, width, height, nbins, ref_mode, eps=1e-9, eflow=None, safety=SAFETY,
              want_err=False):
    """Straddles of an FP32 evaluation of the window (orc_cm_bounds): flags [n]
    (bit 0 cell / support, bit 1 mask, bit 2 bin), counts of flagged events,
    and the interval of N_nz(r) (nnz_lo/hi), of L_r (loss_r_lo/hi) and of the
    loss (loss_lo/hi) over every outcome of the flagged decisions.  eflow:
    bound on the FP32 error of the flow per pixel ([nfb, H, W]; None: the flow
    values are FP32 numbers both sides use exactly).  want_err: the error bound
    of every trajectory point [n, B+1, 2]."""
    W, H = int(width), int(height)
    fl = _c(flow, np.float64)
    nfb = 1 if fl.ndim == 3 else fl.shape[0]
    fl = fl.reshape(nfb, H, W, 2)
    R = n_refs(nbins, ref_mode)
    n = events.n
    a, _keep = _args(events, fl, W, H, nbins, ref_mode, eps, 1.0)
    ef = None if eflow is None else _c(eflow, np.float64).reshape(nfb, H, W)
    out = {"flags": np.zeros(n, np.uint8), "loss_lo": np.zeros(1), "loss_hi": np.zeros(1),
           "loss_r_lo": np.zeros(R), "loss_r_hi": np.zeros(R), "nnz_lo": np.zeros(R, np.int64),
           "nnz_hi": np.zeros(R, np.int64)}
    b = _Bounds()
    b.safety = float(safety)
    b.eflow = _p(ef)
    b.flags = _p(out["flags"])
    for k in ("loss_lo", "loss_hi", "loss_r_lo", "loss_r_hi", "nnz_lo", "nnz_hi"):
        setattr(b, k, _p(out[k]))
    if want_err:
        out["err"] = np.zeros((n, nbins + 1, 2))
        b.err = _p(out["err"])
    st = lib().orc_cm_bounds(ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise ValueError(f"oracle rejected the arguments (status {st})")
    out["loss_lo"] = float(out["loss_lo"][0])
    out["loss_hi"] = float(out["loss_hi"][0])
    out["counts"] = tuple(int(c) for c in b.counts)
    return out


def cm_depth(events, cam, inv_depth, ego, dt, *, nbins, ref_mode, eps=1e-9, grad=False, dloss=1.0, bounds=False,
             **kw):
    """Loss of one window whose flow comes from inverse depth and ego-motion
    (Sec. 3.2 then Sec. 3.1); with grad, also dL/d(inv_depth) and dL/d(ego);
    with bounds, also the straddle analysis (cm_bounds) under "bounds"."""
    f64 = flow_from_depth(cam, inv_depth, ego, dt)
    out = cm(events, f64, width=cam.width, height=cam.height, nbins=nbins, ref_mode=ref_mode, eps=eps, grad=grad,
             dloss=dloss, **kw)
    out["flow"] = f64
    if grad:
        out["dinv_depth"], out["dego"] = depth_ego_grad(cam, inv_depth, ego, dt, out["dflow"])
    if bounds:
        out["bounds"] = cm_bounds(events, f64, width=cam.width, height=cam.height, nbins=nbins, ref_mode=ref_mode,
                                  eps=eps, eflow=flow_error_bound(cam, inv_depth, ego, dt)[None])
    return out


def cm_window(win, bounds=False, **kw):
    """Oracle on a synth.Window (flow input or depth + ego input); with
    bounds, the straddle analysis under "bounds" (cm_bounds)."""
    if win.flow is not None:
        out = cm(win.events, win.flow, width=win.cam.width, height=win.cam.height, nbins=win.nbins,
                 ref_mode=win.ref_mode, **kw)
        if bounds:
            out["bounds"] = cm_bounds(win.events, win.flow, width=win.cam.width, height=win.cam.height,
                                      nbins=win.nbins, ref_mode=win.ref_mode, eps=kw.get("eps", 1e-9))
        return out
    return cm_depth(win.events, win.cam, win.inv_depth, win.ego, win.dt, nbins=win.nbins, ref_mode=win.ref_mode,
                    bounds=bounds, **kw)
