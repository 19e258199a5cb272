"""GPU parity of the geometry-consistency loss (Eq. 3) and of its gradient to
both inverse depths and the camera motion, against the FP64 oracle, and its
composition into the total loss of Eq. 4 through autograd.  The oracle's
straddle analysis (oracle.geo_bounds) flags the pixels whose valid flag,
sample cell or branch of |a - b| an FP32 evaluation could decide the other
way: the loss must lie within 1e-5 of its interval; with the flagged pixels
made invalid in both views' input (a negative inverse depth puts the point
behind the camera, far from every threshold) the loss must match within 1e-5
and every gradient within 1e-4 relative L2."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_RTOL_L2, LOSS_RTOL, gpu_lib, rel_l2

pytestmark = pytest.mark.gpu


def _pair(W, H, seed):
    rng = np.random.default_rng(seed)
    rho0 = synth.inv_depth_map(rng, W, H)
    rho1 = (rho0 * rng.uniform(0.9, 1.1, rho0.shape)).astype(np.float32)
    ego = synth.ego_motion(rng)
    return rho0, rho1, ego


@pytest.mark.parametrize("W,H,seed,dt", [(640, 480, 1, 0.05), (346, 260, 2, 0.2), (96, 72, 3, 0.5)])
def test_geo_loss_and_gradients_match_oracle(W, H, seed, dt):
    import torch
    cm = gpu_lib()
    cam = synth.camera_for(W, H)
    rho0, rho1, ego = _pair(W, H, seed)
    r0 = torch.from_numpy(rho0).cuda().requires_grad_(True)
    r1 = torch.from_numpy(rho1).cuda().requires_grad_(True)
    e = torch.from_numpy(ego).cuda().requires_grad_(True)
    loss = cm.geo_loss(cam, r0, r1, e, dt)
    o = O.geo(cam, rho0, rho1, ego, dt)
    b = O.geo_bounds(cam, rho0, rho1, ego, dt)
    assert 0 < o["count"] < W * H  # some pixels leave the image
    assert b["count_lo"] <= o["count"] <= b["count_hi"] and b["loss_lo"] <= o["loss"] <= b["loss_hi"]
    assert b["loss_lo"] - LOSS_RTOL * o["loss"] <= loss.item() <= b["loss_hi"] + LOSS_RTOL * o["loss"]
    assert b["flagged"] < 3e-3 * W * H
    # the flagged pixels moved behind the camera in view 0: no decision in doubt
    rho0f = rho0.copy()
    rho0f[b["flags"] != 0] = -1.0
    assert O.geo_bounds(cam, rho0f, rho1, ego, dt)["flagged"] == 0
    r0 = torch.from_numpy(rho0f).cuda().requires_grad_(True)
    loss = cm.geo_loss(cam, r0, r1, e, dt)
    (2.5 * loss).backward()
    o = O.geo(cam, rho0f, rho1, ego, dt, grad=True, dloss=2.5)
    assert abs(loss.item() - o["loss"]) <= LOSS_RTOL * abs(o["loss"])
    assert rel_l2(r0.grad.cpu().numpy(), o["dinv_depth0"]) <= GRAD_RTOL_L2
    assert rel_l2(r1.grad.cpu().numpy(), o["dinv_depth1"]) <= GRAD_RTOL_L2
    assert rel_l2(e.grad.cpu().numpy(), o["dego"]) <= GRAD_RTOL_L2


def test_geo_camera_at_rest_is_exactly_zero():
    import torch
    cm = gpu_lib()
    cam = synth.camera_for(346, 260)
    rho0, _, _ = _pair(346, 260, 4)
    r = torch.from_numpy(rho0).cuda()
    loss = cm.geo_loss(cam, r, r.clone(), torch.zeros(6, device="cuda"), 0.01)
    assert loss.item() == 0.0


def test_total_loss_composes_through_autograd():
    import torch
    cm = gpu_lib()
    win = synth.davis_window(n=30000)
    rho1 = (win.inv_depth * 1.05).astype(np.float32)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    ws = cm.Workspace(win.cam, cfg, win.events.n, 1, "cuda")
    ev = cm.DeviceEvents.from_host(win.events, "cuda")
    r0 = torch.from_numpy(win.inv_depth).cuda().requires_grad_(True)
    r1 = torch.from_numpy(rho1).cuda().requires_grad_(True)
    e = torch.from_numpy(win.ego).cuda().requires_grad_(True)
    lcm = cm.cm_loss(ev, ws, inv_depth=r0, ego=e, dt=win.dt)
    lgeo = cm.geo_loss(win.cam, r0, r1, e, win.dt)
    total = lcm + cm.LAMBDA_GEO * lgeo  # Eq. 4
    total.backward()
    g0, ge = r0.grad.clone(), e.grad.clone()
    # the same gradients from the two terms separately
    r0.grad = None
    e.grad = None
    cm.cm_loss(ev, ws, inv_depth=r0, ego=e, dt=win.dt).backward()
    gc0, gce = r0.grad.clone(), e.grad.clone()
    r0.grad = None
    e.grad = None
    (cm.LAMBDA_GEO * cm.geo_loss(win.cam, r0, r1, e, win.dt)).backward()
    assert torch.allclose(g0, gc0 + r0.grad, rtol=1e-5, atol=1e-9)
    assert torch.allclose(ge, gce + e.grad, rtol=1e-5, atol=1e-9)
