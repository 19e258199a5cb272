"""Differentiation at scale: the 1280x720 window with 2,000,000 events and 20
bins (21 references).

* The GPU adjoint (trajectories recomputed, no stored warps) against the FP64
  CPU oracle: on the full window N_nz in the oracle's straddle interval and the
  loss within 1e-5 of its interval; on the window without its flagged events
  N_nz exact, the loss within 1e-5, dL/d(inverse depth) and dL/d(ego) within
  1e-4 relative L2 at eps = 1e-2, and 32 sampled pixels one by one.
* Finite differences of the FP64 oracle (step 1e-4, frozen branch) on 32 random
  inverse-depth pixels (one random +-1 combination) and on each of the 6
  ego-motion components, against the oracle's analytic gradient; eps = 1e-2 so
  that the loss is smooth at the step (with eps = 1e-9 the terms of isolated
  tiny bilinear weights change by orders of magnitude within one step).
* Peak device memory of the backward: the workspace holds the images of
  warped events and small buffers only (no stored trajectories), and the
  backward allocates nothing.
"""
import concurrent.futures as cf

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_EPS, check_interval, check_strict, gpu_lib, run_gpu, run_oracle, unflagged

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def hd():
    return synth.hd_window()


def test_hd_gpu_matches_oracle(hd):
    o = run_oracle(hd, grad=False, bounds=True)
    check_interval(run_gpu(hd, grad=False), o)
    assert o["bounds"]["counts"][3] < 0.02 * hd.events.n  # 21 references, 20 pushes: more points near a threshold
    sub = unflagged(hd, o["bounds"]["flags"])
    check_strict(run_gpu(sub, grad=False), run_oracle(sub, grad=False), grad=False)
    g = run_gpu(sub, eps=GRAD_EPS)
    o = run_oracle(sub, eps=GRAD_EPS)
    check_strict(g, o)
    # the 32 sampled pixels and the 6 ego components one by one
    rng = np.random.default_rng(44)
    H, W = hd.inv_depth.shape
    pix = rng.integers(0, H * W, 32)
    gd, od = g["dinv_depth"].ravel()[pix], o["dinv_depth"].ravel()[pix]
    scale = np.abs(o["dinv_depth"]).max()
    np.testing.assert_allclose(gd, od, rtol=1e-3, atol=1e-4 * scale)
    np.testing.assert_allclose(g["dego"], o["dego"], rtol=1e-4, atol=1e-5 * np.abs(o["dego"]).max())


def test_hd_oracle_gradient_matches_finite_differences(hd):
    eps, h = 1e-2, 1e-4
    cam, B = hd.cam, hd.nbins
    rho = hd.inv_depth.astype(np.float64)
    ego = hd.ego.astype(np.float64)
    base = O.cm_depth(hd.events, cam, rho, ego, hd.dt, nbins=B, ref_mode=hd.ref_mode, eps=eps, grad=True,
                      record=True)
    br = base["branch"]

    def loss(r, e):
        fl = O.flow_from_depth(cam, r, e, hd.dt)
        return O.cm(hd.events, fl, width=cam.width, height=cam.height, nbins=B, ref_mode=hd.ref_mode, eps=eps,
                    replay=br)["loss"]

    rng = np.random.default_rng(7)
    H, W = rho.shape
    pix = rng.choice(H * W, 32, replace=False)
    v = np.zeros(H * W)
    v[pix] = rng.choice([-1.0, 1.0], 32)
    v = v.reshape(H, W)
    # central differences at steps h and h/2, combined by Richardson extrapolation
    # (the step-h difference alone carries an O(h^2) truncation error of ~1e-3 here)
    dirs = [(v, None)] + [(None, i) for i in range(6)]
    jobs = []
    for dv, di in dirs:
        for s in (h, h / 2):
            d = np.zeros(6)
            if di is not None:
                d[di] = s
            dr = 0.0 if dv is None else s * dv
            jobs += [(rho + dr, ego + d), (rho - dr, ego - d)]
    with cf.ThreadPoolExecutor(max_workers=7) as ex:  # the oracle releases the GIL
        vals = list(ex.map(lambda a: loss(*a), jobs))
    fd = []
    for k in range(len(dirs)):
        a = (vals[4 * k] - vals[4 * k + 1]) / (2 * h)
        b = (vals[4 * k + 2] - vals[4 * k + 3]) / h
        fd.append((4 * b - a) / 3)
    an_rho = float((base["dinv_depth"] * v).sum())
    assert fd[0] == pytest.approx(an_rho, rel=1e-5)
    for i in range(6):
        assert fd[1 + i] == pytest.approx(base["dego"][i], rel=1e-5, abs=1e-7 * np.abs(base["dego"]).max())


def test_hd_backward_memory():
    import torch
    cm = gpu_lib()
    hd = synth.hd_window()
    cfg = cm.loss_cfg(hd.nbins, hd.ref_mode, cm.SPLAT_ATOMIC)
    ev = cm.DeviceEvents.from_host(hd.events)
    rho = torch.from_numpy(hd.inv_depth).cuda()
    ego = torch.from_numpy(hd.ego).cuda()
    ws = cm.Workspace(hd.cam, cfg, hd.events.n)
    out = {"dinv_depth": torch.empty_like(rho), "dego": torch.empty(6, device="cuda")}
    dl = torch.ones(1, device="cuda")
    cm.loss_forward(ws, ev, inv_depth=rho, ego=ego, dt=hd.dt)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    before = torch.cuda.memory_allocated()
    cm.loss_backward(ws, ev, dl, inv_depth=rho, ego=ego, dt=hd.dt, want_dflow=False, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.max_memory_allocated() == before  # the backward allocates nothing
    iwe = (hd.nbins + 1) * hd.cam.width * hd.cam.height * 16
    stored_warps = hd.events.n * (hd.nbins + 1) * 8
    # the workspace is the images of warped events plus a few per-pixel buffers
    # (the flow quads and gradient records, 32 bytes each, among them)
    assert iwe < ws.nbytes < iwe + 112 * hd.cam.width * hd.cam.height
    print(f"\nworkspace {ws.nbytes / 1e6:.1f} MB (IWE {iwe / 1e6:.1f} MB); stored trajectories would add "
          f"{stored_warps / 1e6:.1f} MB")
