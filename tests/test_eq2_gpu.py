"""GPU parity of the discrete flow (Eq. 2 with one pose per bin) and of its
adjoint: the flows within the oracle's bound on an FP32 evaluation of its FP64
definition, the adjoint against the FP64 oracle on a seeded dL/dflow, and the
whole chain (per-bin flows -> CM loss -> CM adjoint -> Eq. 2 adjoint) against
the oracle's chain through the autograd Function: the loss within 1e-5 of the
straddle interval (the flows' FP32 error bound included) and, on the window
without its flagged events, the loss and every gradient strictly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_EPS, GRAD_RTOL_L2, LOSS_RTOL, gpu_lib, rel_l2, unflagged

pytestmark = pytest.mark.gpu


def _poses(rng, nb):
    ego = np.stack([synth.ego_motion(rng) for _ in range(nb)]).astype(np.float32)
    return ego


def test_eq2_flow_within_its_fp32_error_bound():
    import torch
    cm = gpu_lib()
    cam = synth.camera_for(346, 260)
    rng = synth.rng_for(2)
    rho = synth.inv_depth_map(rng, 346, 260)
    ego = _poses(rng, 10)
    ego[7, 3:] *= 30.0  # one large rotation
    f = cm.flow_eq2(cam, torch.from_numpy(rho).cuda(), torch.from_numpy(ego).cuda(), 0.001, 10.0).cpu().numpy()
    f64 = O.flow_eq2_bins(cam, rho.astype(np.float64), ego.astype(np.float64), 0.001, 10.0)
    eb = O.flow_eq2_error_bound(cam, rho, ego, 0.001, 10.0)
    assert np.all(np.abs(f.astype(np.float64) - f64).max(axis=-1) <= eb)


@pytest.mark.parametrize("nb", [1, 10])
def test_eq2_adjoint_matches_oracle(nb):
    import torch
    cm = gpu_lib()
    cam = synth.camera_for(640, 480)
    rng = synth.rng_for(5)
    rho = synth.inv_depth_map(rng, 640, 480)
    ego = _poses(rng, nb)
    g = np.random.default_rng(8).normal(size=(nb, 480, 640, 2)).astype(np.float32)
    drho, dego = cm.flow_eq2_backward(cam, torch.from_numpy(rho).cuda(), torch.from_numpy(ego).cuda(), 0.001,
                                      float(nb), torch.from_numpy(g).cuda())
    orho, oego = O.flow_eq2_grad(cam, rho.astype(np.float64), ego.astype(np.float64), 0.001, float(nb), g)
    assert rel_l2(drho.cpu().numpy(), orho) <= 1e-5
    assert rel_l2(dego.cpu().numpy(), oego) <= 1e-5
    # deterministic: the same bits on a second call
    drho2, dego2 = cm.flow_eq2_backward(cam, torch.from_numpy(rho).cuda(), torch.from_numpy(ego).cuda(), 0.001,
                                        float(nb), torch.from_numpy(g).cuda())
    assert torch.equal(drho, drho2) and torch.equal(dego, dego2)


def _chain_oracle(win, ego, dt_bin, scale, eps=1e-9, grad=True, bounds=False):
    nb = ego.shape[0]
    rho = win.inv_depth.astype(np.float64)
    f64 = O.flow_eq2_bins(win.cam, rho, ego.astype(np.float64), dt_bin, scale)
    kw = dict(width=win.cam.width, height=win.cam.height, nbins=win.nbins, ref_mode=win.ref_mode, eps=eps)
    r = O.cm(win.events, f64 if nb > 1 else f64[0], grad=grad, **kw)
    if bounds:
        eb = O.flow_eq2_error_bound(win.cam, rho, ego, dt_bin, scale)
        r["bounds"] = O.cm_bounds(win.events, f64 if nb > 1 else f64[0], eflow=eb, **kw)
    if grad:
        r["dinv_depth"], r["dego"] = O.flow_eq2_grad(win.cam, rho, ego.astype(np.float64), dt_bin, scale,
                                                     np.asarray(r["dflow"]).reshape(nb, win.cam.height,
                                                                                    win.cam.width, 2))
    return r


def _chain_gpu(cm, win, ego, dt_bin, scale, eps):
    import torch
    nb = ego.shape[0]
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC, eps)
    ws = cm.Workspace(win.cam, cfg, max(win.events.n, 1), nb, "cuda")
    ev = cm.DeviceEvents.from_host(win.events, "cuda")
    rho = torch.from_numpy(win.inv_depth).cuda().requires_grad_(True)
    eg = torch.from_numpy(ego).cuda().requires_grad_(True)
    loss = cm.CMLossEq2.apply(rho, eg, ev, ws, dt_bin, scale)
    loss.backward()
    return loss.item(), rho.grad.cpu().numpy(), eg.grad.cpu().numpy()


@pytest.mark.parametrize("nb", [1, 10])
def test_eq2_chain_matches_oracle(nb):
    import torch
    cm = gpu_lib()
    rng = np.random.default_rng(60 + nb)
    win = synth.depth_window(rng, 160, 120, 20000, nbins=10)
    ego = _poses(rng, nb)
    dt_bin, scale = win.dt / nb, float(nb)
    L, _, _ = _chain_gpu(cm, win, ego, dt_bin, scale, 1e-9)
    o = _chain_oracle(win, ego, dt_bin, scale, grad=False, bounds=True)
    b = o["bounds"]
    assert b["loss_lo"] - LOSS_RTOL * o["loss"] <= L <= b["loss_hi"] + LOSS_RTOL * o["loss"]
    sub = unflagged(win, b["flags"])
    L, grho, gego = _chain_gpu(cm, sub, ego, dt_bin, scale, GRAD_EPS)
    o = _chain_oracle(sub, ego, dt_bin, scale, eps=GRAD_EPS)
    assert abs(L - o["loss"]) <= LOSS_RTOL * abs(o["loss"])
    assert rel_l2(grho, o["dinv_depth"]) <= GRAD_RTOL_L2
    assert rel_l2(gego, o["dego"]) <= GRAD_RTOL_L2


def test_eq2_rejects_bad_arguments():
    import torch
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    cam = cm.camera(synth.camera_for(64, 48))
    rho = torch.ones(48, 64, device="cuda")
    ego = torch.zeros(33, 6, device="cuda")
    out = torch.empty(33, 48, 64, 2, device="cuda")
    with pytest.raises(C.CMError) as e:
        C.cm_flow_eq2(cam, rho.data_ptr(), ego.data_ptr(), 33, 0.01, 1.0, out.data_ptr(), 0)
    assert e.value.status == C.CM_EINVAL
    need = C.cm_flow_eq2_scratch_query(cam, 2)
    small = torch.empty(max(need // 2, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(C.CMError) as e:
        C.cm_flow_eq2_backward(cam, rho.data_ptr(), ego.data_ptr(), 2, 0.01, 1.0, out.data_ptr(), rho.data_ptr(),
                               ego.data_ptr(), small.data_ptr(), small.numel(), 0)
    assert e.value.status == C.CM_ENOMEM
