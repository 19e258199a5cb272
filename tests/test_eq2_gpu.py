"""GPU parity of the discrete flow (Eq. 2 with one pose per bin) and of its
adjoint: the flows bit for bit against the oracle's FP32 operation sequence
(and within FP32 error of its FP64 definition), the adjoint against the FP64
oracle on a seeded dL/dflow, and the whole chain (per-bin flows -> CM loss ->
CM adjoint -> Eq. 2 adjoint) against the oracle's chain, also through the
autograd Function."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_RTOL_L2, LOSS_RTOL, gpu_lib, rel_l2

pytestmark = pytest.mark.gpu


def _poses(rng, nb):
    ego = np.stack([synth.ego_motion(rng) for _ in range(nb)]).astype(np.float32)
    return ego


def test_eq2_flow_bit_exact_and_close_to_fp64():
    import torch
    cm = gpu_lib()
    cam = synth.camera_for(346, 260)
    rng = synth.rng_for(2)
    rho = synth.inv_depth_map(rng, 346, 260)
    ego = _poses(rng, 10)
    ego[7, 3:] *= 30.0  # one large rotation
    f = cm.flow_eq2(cam, torch.from_numpy(rho).cuda(), torch.from_numpy(ego).cuda(), 0.001, 10.0).cpu().numpy()
    f32 = O.flow_eq2_bins_f32(cam, rho, ego, 0.001, 10.0)
    assert np.array_equal(f, f32)
    f64 = O.flow_eq2_bins(cam, rho.astype(np.float64), ego.astype(np.float64), 0.001, 10.0)
    zmax = 1.0 / float(rho.min())
    xmax = max(cam.cx, cam.width - cam.cx) / cam.fx
    assert np.abs(f - f64).max() < 8 * 10.0 * cam.fx * zmax * (1 + xmax) * 2.0 ** -24


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


def _chain_oracle(win, ego, dt_bin, scale, eps=1e-9):
    nb = ego.shape[0]
    f64 = O.flow_eq2_bins(win.cam, win.inv_depth.astype(np.float64), ego.astype(np.float64), dt_bin, scale)
    f32 = O.flow_eq2_bins_f32(win.cam, win.inv_depth, ego, dt_bin, scale)
    r = O.cm(win.events, f64 if nb > 1 else f64[0], width=win.cam.width, height=win.cam.height, nbins=win.nbins,
             ref_mode=win.ref_mode, eps=eps, positions="f32", flow32=f32 if nb > 1 else f32[0], grad=True)
    drho, dego = O.flow_eq2_grad(win.cam, win.inv_depth.astype(np.float64), ego.astype(np.float64), dt_bin, scale,
                                 np.asarray(r["dflow"]).reshape(nb, win.cam.height, win.cam.width, 2))
    return r["loss"], drho, dego


@pytest.mark.parametrize("nb", [1, 10])
def test_eq2_chain_matches_oracle(nb):
    import torch
    cm = gpu_lib()
    rng = np.random.default_rng(60 + nb)
    win = synth.depth_window(rng, 160, 120, 20000, nbins=10)
    ego = _poses(rng, nb)
    dt_bin, scale = win.dt / nb, float(nb)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    ws = cm.Workspace(win.cam, cfg, win.events.n, nb, "cuda")
    ev = cm.DeviceEvents.from_host(win.events, "cuda")
    rho = torch.from_numpy(win.inv_depth).cuda().requires_grad_(True)
    eg = torch.from_numpy(ego).cuda().requires_grad_(True)
    loss = cm.CMLossEq2.apply(rho, eg, ev, ws, dt_bin, scale)
    loss.backward()
    L, orho, oego = _chain_oracle(win, ego, dt_bin, scale)
    assert abs(loss.item() - L) <= LOSS_RTOL * abs(L)
    assert rel_l2(rho.grad.cpu().numpy(), orho) <= GRAD_RTOL_L2
    assert rel_l2(eg.grad.cpu().numpy(), oego) <= GRAD_RTOL_L2


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
