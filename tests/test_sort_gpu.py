"""The deterministic sort-by-pixel path (CM_SPLAT_SORT): parity with the FP64
oracle by the same checks as the atomic path (tests/gpu_util.py), and
bit-reproducibility run to run of the images of warped events, the loss and
every gradient."""
import numpy as np
import pytest

from paper_2412_06359_gb300 import synth
from tests.gpu_util import check_window, gpu_lib, plain, rel_l2, run_gpu, run_oracle, unflagged
from tests.test_parity_gpu import small_depth_window, small_flow_window

pytestmark = pytest.mark.gpu

END, ALL = synth.REF_END, synth.REF_ALL


def sort_mode():
    return gpu_lib().SPLAT_SORT


def test_sort_flow_window_128():
    win = synth.flow_window()
    check_window(win, plain(splat=sort_mode()))


def test_sort_davis_window_346():
    win = synth.davis_window()
    check_window(win, plain(splat=sort_mode()))


@pytest.mark.parametrize("B,ref_mode,nfb", [(4, ALL, 4), (5, END, 1), (3, ALL, 1), (20, ALL, 1)])
def test_sort_bins_refs_and_per_bin_flows(B, ref_mode, nfb):
    win = small_flow_window(70, 50, 5000, B, ref_mode, nfb=nfb, seed=B * 7 + nfb)
    check_window(win, plain(splat=sort_mode()))


@pytest.mark.parametrize("n", [1, 255, 2049, 4097])
def test_sort_ragged_event_counts(n):
    # entry counts below, at and across the sort's 2048-entry tiles
    win = small_depth_window(64, 48, n, 10, seed=n + 1)
    check_window(win, plain(splat=sort_mode()))


def test_sort_empty_and_all_masked():
    win = small_flow_window(32, 24, 0, 4, ALL)
    g = run_gpu(win, splat=sort_mode())
    assert g["loss"] == 0.0 and not np.any(g["dflow"])
    win = small_flow_window(40, 30, 2000, 4, ALL)
    win.flow = np.full_like(win.flow, 100.0)
    g = run_gpu(win, splat=sort_mode())
    assert g["loss"] == 0.0 and not np.any(g["nnz_r"]) and not np.any(g["dflow"])


def test_sort_iwe_matches_oracle_elementwise():
    win = small_depth_window(120, 90, 9000, 10, seed=4)
    win = unflagged(win, run_oracle(win, grad=False, bounds=True)["bounds"]["flags"])
    g = run_gpu(win, splat=sort_mode(), grad=False, want_iwe=True)
    o = run_oracle(win, grad=False, want_iwe=True)
    assert np.array_equal(g["iwe"] != 0, o["iwe"] != 0)
    np.testing.assert_allclose(g["iwe"], o["iwe"], rtol=1e-5, atol=2e-6)


def _sort_run_raw(win):
    """Every output of one sort-path evaluation, as raw bytes."""
    import torch
    cm = gpu_lib()
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_SORT)
    ws = cm.Workspace(win.cam, cfg, win.events.n)
    ev = cm.DeviceEvents.from_host(win.events)
    rho = torch.from_numpy(win.inv_depth).cuda()
    ego = torch.from_numpy(win.ego).cuda()
    loss = cm.loss_forward(ws, ev, inv_depth=rho, ego=ego, dt=win.dt)
    g = cm.loss_backward(ws, ev, torch.ones(1, device="cuda"), inv_depth=rho, ego=ego, dt=win.dt)
    torch.cuda.synchronize()
    out = {"loss": loss.cpu().numpy().tobytes(), "dflow": g["dflow"].cpu().numpy().tobytes(),
           "dinv_depth": g["dinv_depth"].cpu().numpy().tobytes(), "dego": g["dego"].cpu().numpy().tobytes()}
    lr, nz = ws.stats()
    out["loss_r"] = lr.tobytes()
    return out


def test_sort_path_is_bit_reproducible():
    import torch
    win = synth.davis_window()
    first = _sort_run_raw(win)
    # other work on the GPU in between, a different allocation pattern, then again
    junk = torch.randn(1 << 22, device="cuda")
    junk.mul_(2.0)
    second = _sort_run_raw(win)
    third = _sort_run_raw(win)
    for k in first:
        assert first[k] == second[k] == third[k], f"{k} differs between runs"


def test_sort_iwe_is_bit_reproducible():
    import torch
    cm = gpu_lib()
    win = small_flow_window(200, 150, 30000, 10, ALL, seed=5)
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_SORT)
    ws = cm.Workspace(win.cam, cfg, win.events.n)
    ev = cm.DeviceEvents.from_host(win.events)
    flow = torch.from_numpy(win.flow[0]).cuda()
    outs = []
    for _ in range(3):
        from paper_2412_06359_gb300 import _capi as C
        iwe = torch.empty((win.nbins + 1, 150, 200, 4), device="cuda")
        C.cm_warp_splat(cm.camera(win.cam), ev.c(), flow.data_ptr(), 1, cfg, ws.handle, iwe.data_ptr(),
                        cm.stream_handle())
        torch.cuda.synchronize()
        outs.append(iwe.cpu().numpy().tobytes())
    assert outs[0] == outs[1] == outs[2]


def test_sort_and_atomic_paths_agree():
    win = synth.davis_window()
    a = run_gpu(win, splat=gpu_lib().SPLAT_ATOMIC)
    s = run_gpu(win, splat=sort_mode())
    assert np.array_equal(a["nnz_r"], s["nnz_r"])
    assert abs(a["loss"] - s["loss"]) <= 1e-6 * abs(a["loss"])
    assert rel_l2(a["dinv_depth"], s["dinv_depth"]) < 1e-5
    assert rel_l2(a["dego"], s["dego"]) < 1e-5
