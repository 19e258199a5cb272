"""Shared helpers of the GPU parity tests: run one window through the C ABI
and through the CPU oracle, and compare."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2412_06359_gb300 import synth

LOSS_RTOL = 1e-5      # relative error of the loss (FP32 accumulation against FP64)
GRAD_RTOL_L2 = 1e-4   # relative L2 error of every gradient


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


def run_oracle(win: synth.Window, *, grad=True, dloss=1.0, eps=1e-9, want_iwe=False):
    return O.cm_window(win, grad=grad, dloss=dloss, eps=eps, want_iwe=want_iwe, positions="f32")


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.linalg.norm(a)
    return np.linalg.norm(a - b) / nb


def assert_parity(g, o, *, grad=True, loss_rtol=LOSS_RTOL, grad_rtol=GRAD_RTOL_L2):
    """GPU result g against oracle result o: integer decisions exact, loss and
    gradients within the stated tolerances."""
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
