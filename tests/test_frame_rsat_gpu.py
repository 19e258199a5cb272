"""GPU parity of the network's input frame (bit for bit against the oracle) and
of the RSAT metric (against the oracle's ratio of CM losses: within 2e-5 of
the interval the straddle analysis gives the numerator)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import gpu_lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,n", [(640, 480, 300000), (346, 260, 1), (64, 48, 0)])
def test_event_frame_bit_exact(W, H, n):
    cm = gpu_lib()
    rng = np.random.default_rng(W + n)
    e = synth.uniform_events(rng, W, H, n)
    if n > 10:  # a few events outside the sensor are skipped
        e.x[:5] = np.array([-1, W, 3, 0, W + 7], np.int16)
        e.y[:5] = np.array([2, 1, -3, H, 0], np.int16)
    ev = cm.DeviceEvents.from_host(e, "cuda")
    f = cm.event_frame(synth.camera_for(W, H), ev).cpu().numpy()
    assert np.array_equal(f, O.event_frame(e, W, H).astype(np.float32))


@pytest.mark.parametrize("wl", ["flow", "bins"])
def test_rsat_matches_oracle(wl):
    import torch
    cm = gpu_lib()
    if wl == "flow":
        win = synth.flow_window()
        flow = win.flow[0]
    else:
        rng = np.random.default_rng(9)
        W, H = 120, 90
        ev = synth.uniform_events(rng, W, H, 15000)
        flow = np.stack([synth.sinusoid_flow(rng, W, H, 4.0) for _ in range(5)])
        win = synth.Window(synth.Camera(W, H, 80.0, 80.0, W / 2, H / 2), ev, 5, synth.REF_ALL, flow=flow)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC)
    nfb = 1 if flow.ndim == 3 else flow.shape[0]
    ws = cm.Workspace(win.cam, cfg, win.events.n, nfb, "cuda")
    ev = cm.DeviceEvents.from_host(win.events, "cuda")
    fl = torch.from_numpy(np.ascontiguousarray(flow, np.float32)).cuda()
    r = float(cm.rsat(ws, ev, fl).item())
    o, lo, hi = O.rsat(win.events, flow, width=win.cam.width, height=win.cam.height, nbins=win.nbins,
                       ref_mode=win.ref_mode, bounds=True)
    assert lo <= o <= hi
    assert lo - 2e-5 * abs(o) <= r <= hi + 2e-5 * abs(o)
    # zero flow: the ratio of two evaluations of the same loss
    z = float(cm.rsat(ws, ev, torch.zeros_like(fl)).item())
    assert abs(z - 1.0) <= 1e-6
    # the workspace holds no forward for a backward afterwards
    from paper_2412_06359_gb300 import _capi as C
    with pytest.raises(C.CMError) as e:
        cm.loss_backward(ws, ev, torch.ones(1, device="cuda"), flow=fl)
    assert e.value.status == C.CM_ESTATE
