"""Shared helpers of the GPU parity tests: run windows through the C ABI and
through the FP64 CPU oracle, and compare.

How an FP32 result is judged against the FP64 definition (the oracle computes
everything in FP64 and shares no arithmetic with the kernels):

* full window: the oracle's straddle analysis (oracle.cm_bounds) flags every
  event with a decision (cell / support, mask, bin) within its FP32 error
  margin and gives the interval of N_nz(r), L_r and the loss over every outcome
  of those decisions.  The GPU's N_nz(r) must lie in its interval (integers,
  exactly) and its loss and every L_r within LOSS_RTOL of theirs.
* unflagged window: the same window without its flagged events.  No decision
  of it is in doubt, so N_nz(r) must equal the oracle's exactly, the loss and
  every L_r must match within LOSS_RTOL, and every gradient within
  GRAD_RTOL_L2 relative L2 at eps = GRAD_EPS.  The gradient is compared at an
  eps where it is well-conditioned: at eps = 1e-9 the term of a pixel reached
  by one small weight w is ~ eps / w^2 and T - tbar is below FP32 resolution,
  so the FP32 gradient of such pixels is rounding noise.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses

import numpy as np

from oracle import oracle as O
from paper_2412_06359_gb300 import synth

LOSS_RTOL = 1e-5      # relative error of the loss (FP32 accumulation against FP64)
GRAD_RTOL_L2 = 1e-4   # relative L2 error of every gradient
GRAD_EPS = 1e-2       # eps of the gradient comparisons (well-conditioned)


def gpu_lib():
    import torch

    from paper_2412_06359_gb300 import build
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    build.build()
    from paper_2412_06359_gb300 import cm
    return cm


def run_gpu(win: synth.Window, *, splat=None, grad=True, dloss=1.0, eps=1e-9, want_iwe=False, store_warps=False):
    """Loss (and gradients) of one window through cm_loss_forward / backward."""
    import torch
    cm = gpu_lib()
    if splat is None:
        splat = cm.SPLAT_ATOMIC
    dev = "cuda"
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, splat, eps, store_warps)
    nfb = 1 if win.flow is None else win.flow.shape[0]
    ws = cm.Workspace(win.cam, cfg, max(win.events.n, 1), nfb, dev)
    ev = cm.DeviceEvents.from_host(win.events, dev)
    out = {}
    dl = torch.tensor([dloss], dtype=torch.float32, device=dev)
    if win.flow is not None:
        flow = torch.from_numpy(np.ascontiguousarray(win.flow, np.float32)).to(dev)
        if nfb == 1:
            flow = flow[0].contiguous()
        loss = cm.loss_forward(ws, ev, flow=flow)
        if grad:
            g = cm.loss_backward(ws, ev, dl, flow=flow)
            out["dflow"] = g["dflow"].cpu().numpy().reshape(nfb, win.cam.height, win.cam.width, 2)
        if want_iwe:
            out["iwe"] = cm.warp_splat(win.cam, ev, flow, cfg, ws).cpu().numpy()
    else:
        rho = torch.from_numpy(np.ascontiguousarray(win.inv_depth, np.float32)).to(dev)
        ego = torch.from_numpy(np.ascontiguousarray(win.ego, np.float32)).to(dev)
        loss = cm.loss_forward(ws, ev, inv_depth=rho, ego=ego, dt=win.dt)
        if grad:
            g = cm.loss_backward(ws, ev, dl, inv_depth=rho, ego=ego, dt=win.dt)
            out["dflow"] = g["dflow"].cpu().numpy()
            out["dinv_depth"] = g["dinv_depth"].cpu().numpy()
            out["dego"] = g["dego"].cpu().numpy()
        if want_iwe:
            flow = cm.flow_from_depth(win.cam, rho, ego, win.dt)
            out["flow"] = flow.cpu().numpy()
            out["iwe"] = cm.warp_splat(win.cam, ev, flow, cfg, ws).cpu().numpy()
    torch.cuda.synchronize()
    out["loss"] = float(loss.cpu().numpy()[0])
    out["loss_r"], out["nnz_r"] = ws.stats()
    return out


def plain(**kw):
    """A runner for check_windows: one cm_loss_forward / backward call per window."""
    return lambda wins, eps: [run_gpu(w, eps=eps, **kw) for w in wins]


def run_oracle(win: synth.Window, *, grad=True, dloss=1.0, eps=1e-9, want_iwe=False, bounds=False):
    """The FP64 oracle on one window (with bounds: the straddle analysis too)."""
    return O.cm_window(win, grad=grad, dloss=dloss, eps=eps, want_iwe=want_iwe, bounds=bounds)


def unflagged(win: synth.Window, flags) -> synth.Window:
    """The window without the events whose decisions are in doubt."""
    keep = np.nonzero(np.asarray(flags) == 0)[0]
    return dataclasses.replace(win, events=win.events.take(keep))


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.linalg.norm(a)
    return np.linalg.norm(a - b) / nb


def check_interval(g, o, *, loss_rtol=LOSS_RTOL):
    """GPU result g of a full window against the oracle's interval (o from
    run_oracle(..., bounds=True)): N_nz(r) inside [nnz_lo, nnz_hi] exactly, the
    loss and every L_r within loss_rtol of [lo, hi]."""
    b = o["bounds"]
    nnz = np.asarray(g["nnz_r"], np.int64)
    assert np.all((b["nnz_lo"] <= nnz) & (nnz <= b["nnz_hi"])), (nnz, b["nnz_lo"], b["nnz_hi"])
    tol = loss_rtol * abs(o["loss"])
    assert b["loss_lo"] - tol <= g["loss"] <= b["loss_hi"] + tol, (g["loss"], b["loss_lo"], b["loss_hi"])
    lr = np.asarray(g["loss_r"], np.float64)
    tr = loss_rtol * np.abs(o["loss_r"]) + 1e-30
    assert np.all((b["loss_r_lo"] - tr <= lr) & (lr <= b["loss_r_hi"] + tr)), (lr, b["loss_r_lo"], b["loss_r_hi"])


def check_strict(g, o, *, grad=True, loss_rtol=LOSS_RTOL, grad_rtol=GRAD_RTOL_L2):
    """GPU result g of a window with no flagged decision against the oracle:
    N_nz(r) exact, loss and every L_r within loss_rtol, gradients within
    grad_rtol relative L2."""
    assert np.array_equal(np.asarray(g["nnz_r"], np.int64), np.asarray(o["nnz_r"], np.int64)), \
        (g["nnz_r"], o["nnz_r"])
    if o["loss"] == 0:
        assert g["loss"] == 0
    else:
        assert abs(g["loss"] - o["loss"]) <= loss_rtol * abs(o["loss"]), (g["loss"], o["loss"])
        np.testing.assert_allclose(g["loss_r"], o["loss_r"], rtol=loss_rtol, atol=1e-30)
    if grad:
        for k in ("dflow", "dinv_depth", "dego"):
            if k in o and k in g:
                gk = np.asarray(g[k]).reshape(np.shape(o[k]))
                e = rel_l2(gk, o[k])
                assert e <= grad_rtol, f"{k}: relative L2 error {e:.3g} > {grad_rtol}"


def _oracles(wins, **kw):
    # the oracle releases the GIL: windows in parallel threads
    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(wins)))) as ex:
        return list(ex.map(lambda w: run_oracle(w, **kw) if w.events.n else None, wins))


def check_windows(wins, run, *, eps=1e-9, grad_eps=GRAD_EPS, dloss=1.0, grad=True, full=None):
    """Parity of GPU results against the FP64 oracle for a list of windows.

    run(windows, eps) -> list of GPU result dicts (run_gpu's keys; dloss is the
    runner's).  full: the GPU results of `wins` at eps if already computed.
    Full windows are checked against the oracle's interval, the windows
    without their flagged events strictly (loss and N_nz at eps, and with grad
    the gradients at grad_eps).  Returns the oracle's flagged-event counts."""
    if full is None:
        full = run(wins, eps)
    ofull = _oracles(wins, grad=False, eps=eps, bounds=True)
    flagged = []
    for w, g, o in zip(wins, full, ofull):
        if w.events.n == 0:
            assert g["loss"] == 0.0 and not np.any(g["nnz_r"])
            flagged.append(0)
            continue
        check_interval(g, o)
        flagged.append(o["bounds"]["counts"][3])
    subs = [unflagged(w, o["bounds"]["flags"]) if o is not None else w for w, o in zip(wins, ofull)]
    gs = run(subs, eps)
    os_ = _oracles(subs, grad=False, eps=eps)
    for w, g, o in zip(subs, gs, os_):
        if w.events.n:
            check_strict(g, o, grad=False)
    if grad:
        gg = run(subs, grad_eps)
        og = _oracles(subs, grad=True, eps=grad_eps, dloss=dloss)
        for w, g, o in zip(subs, gg, og):
            if w.events.n:
                check_strict(g, o, grad=True)
            else:
                for k in ("dflow", "dinv_depth", "dego"):
                    if k in g:
                        assert not np.any(g[k])
    return flagged


def check_window(win, run=None, **kw):
    """check_windows for one window (default runner: plain single-window calls)."""
    return check_windows([win], run or plain(), **kw)[0]
