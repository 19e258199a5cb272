"""cm_loss_grad_static: the loss + flow gradient entry point that allocates
nothing (for callers that cannot call cudaMalloc where they evaluate the loss:
real-time loops, plug-ins inside a framework that owns the memory pool, code
with a fixed up-front budget).  Its output must equal the workspace path's
(cm_loss_forward + cm_loss_backward) within the parity tolerances, on two
calls in a row, whether this file runs alone in a fresh process or after the
other tests; its loss must lie within the FP64 oracle's interval; and after a
first call the calls must leave the device's free memory and torch's
allocation count unchanged.  Kept in its own file, collected last."""
import numpy as np
import pytest

from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_RTOL_L2, LOSS_RTOL, gpu_lib, rel_l2, run_oracle

pytestmark = pytest.mark.gpu


def _window(W, H, n, B, ref_mode, nfb, seed):
    rng = np.random.default_rng(seed)
    ev = synth.uniform_events(rng, W, H, n)
    flow = np.stack([synth.sinusoid_flow(rng, W, H, 4.0) for _ in range(nfb)])
    return synth.Window(synth.Camera(W, H, 0.7 * W, 0.7 * W, W / 2, H / 2), ev, B, ref_mode, flow=flow)


def _static_call(cm, win, flow, ev, dloss):
    import torch
    from paper_2412_06359_gb300 import _capi as C
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    loss = torch.empty(1, device="cuda")
    dflow = torch.empty_like(flow)
    nfb = 1 if flow.dim() == 3 else flow.shape[0]
    C.cm_loss_grad_static(cm.camera(win.cam), ev.c(), flow.data_ptr(), nfb, cfg, dloss.data_ptr(), loss.data_ptr(),
                          dflow.data_ptr(), cm.stream_handle())
    torch.cuda.synchronize()
    return float(loss.cpu()[0]), dflow.cpu().numpy()


def _workspace_call(cm, win, flow, ev, dloss):
    import torch
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    nfb = 1 if flow.dim() == 3 else flow.shape[0]
    ws = cm.Workspace(win.cam, cfg, max(ev.n, 1), nfb)
    loss = cm.loss_forward(ws, ev, flow=flow)
    g = cm.loss_backward(ws, ev, dloss, flow=flow)
    torch.cuda.synchronize()
    return float(loss.cpu()[0]), g["dflow"].cpu().numpy()


def test_static_entry_matches_workspace_path_two_calls():
    import torch
    cm = gpu_lib()
    cases = [
        # the 128x128 flow workload (20,000 events, one bin, window-end reference)
        synth.flow_window(),
        # a multi-bin, all-edges window with one flow per bin and a different size
        _window(160, 120, 12000, 6, synth.REF_ALL, 6, seed=99),
    ]
    for win in cases:
        ev = cm.DeviceEvents.from_host(win.events)
        flow = torch.from_numpy(np.ascontiguousarray(win.flow, np.float32)).cuda()
        if flow.shape[0] == 1:
            flow = flow[0].contiguous()
        dloss = torch.tensor([1.5], device="cuda")
        ref_loss, ref_g = _workspace_call(cm, win, flow, ev, dloss)
        # two calls in a row on the same input: the second sees the first call's leftovers
        for _ in range(2):
            loss, g = _static_call(cm, win, flow, ev, dloss)
            assert abs(loss - ref_loss) <= LOSS_RTOL * abs(ref_loss), (loss, ref_loss)
            assert rel_l2(g, ref_g) <= GRAD_RTOL_L2
        # and against the FP64 oracle's interval over FP32-sensitive decisions
        o = run_oracle(win, grad=False, bounds=True)
        b = o["bounds"]
        assert b["loss_lo"] - LOSS_RTOL * o["loss"] <= loss <= b["loss_hi"] + LOSS_RTOL * o["loss"]


def test_static_entry_allocates_nothing():
    import torch
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    win = synth.flow_window()
    ev = cm.DeviceEvents.from_host(win.events)
    flow = torch.from_numpy(np.ascontiguousarray(win.flow[0], np.float32)).cuda()
    dloss = torch.ones(1, device="cuda")
    loss = torch.empty(1, device="cuda")
    dflow = torch.empty_like(flow)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    # the set-up call (an empty window): reserves the array on this device
    empty = cm.DeviceEvents.from_host(win.events.take(np.arange(0)))
    C.cm_loss_grad_static(cm.camera(win.cam), empty.c(), flow.data_ptr(), 1, cfg, dloss.data_ptr(),
                          loss.data_ptr(), dflow.data_ptr(), cm.stream_handle())
    torch.cuda.synchronize()
    assert float(loss.cpu()[0]) == 0.0
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(5):
        C.cm_loss_grad_static(cm.camera(win.cam), ev.c(), flow.data_ptr(), 1, cfg, dloss.data_ptr(),
                              loss.data_ptr(), dflow.data_ptr(), cm.stream_handle())
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0
    assert float(loss.cpu()[0]) > 0.0


def test_static_entry_rejects_windows_beyond_its_array():
    import torch
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    # 640x480 with 11 references needs ~54 MB of images: more than the 32 MiB array
    win = _window(640, 480, 1000, 10, synth.REF_ALL, 1, seed=5)
    ev = cm.DeviceEvents.from_host(win.events)
    flow = torch.from_numpy(win.flow[0]).cuda()
    out = torch.empty(1, device="cuda")
    dflow = torch.empty_like(flow)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    with pytest.raises(C.CMError) as e:
        C.cm_loss_grad_static(cm.camera(win.cam), ev.c(), flow.data_ptr(), 1, cfg, out.data_ptr(), out.data_ptr(),
                              dflow.data_ptr(), cm.stream_handle())
    assert e.value.status == C.CM_ENOMEM
