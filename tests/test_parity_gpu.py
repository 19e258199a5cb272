"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle, on
the same seeded inputs, element by element where the output is an image and on
the loss / gradients with the stated tolerances: on every full window N_nz
inside the oracle's straddle interval and the loss within 1e-5 of its
interval; on the window without its flagged events N_nz exact, the loss within
1e-5 relative and every gradient within 1e-4 relative L2 (tests/gpu_util.py)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth
from tests.gpu_util import (GRAD_EPS, check_strict, check_window, gpu_lib, plain, rel_l2, run_gpu, run_oracle,
                            unflagged)

pytestmark = pytest.mark.gpu

END, ALL = synth.REF_END, synth.REF_ALL


def small_flow_window(W, H, n, B, ref_mode, nfb=1, seed=0, mag=4.0):
    rng = np.random.default_rng(seed)
    ev = synth.uniform_events(rng, W, H, n)
    flow = np.stack([synth.sinusoid_flow(rng, W, H, mag) for _ in range(nfb)])
    return synth.Window(synth.Camera(W, H, 0.7 * W, 0.7 * W, W / 2, H / 2), ev, B, ref_mode, flow=flow)


def small_depth_window(W, H, n, B, ref_mode=ALL, seed=0):
    return synth.depth_window(np.random.default_rng(seed), W, H, n, nbins=B, ref_mode=ref_mode)


def test_flow_from_depth_within_its_fp32_error_bound():
    # every component within the oracle's bound on an FP32 evaluation of the
    # motion field (a few units of 2^-24 of the magnitudes of its terms)
    import torch
    cm = gpu_lib()
    for w in (synth.davis_window(n=10), synth.batch_windows(1)[0]):
        rho = torch.from_numpy(w.inv_depth).cuda()
        ego = torch.from_numpy(w.ego).cuda()
        f = cm.flow_from_depth(w.cam, rho, ego, w.dt).cpu().numpy().astype(np.float64)
        f64 = O.flow_from_depth(w.cam, w.inv_depth, w.ego, w.dt)
        eb = O.flow_error_bound(w.cam, w.inv_depth, w.ego, w.dt)
        assert np.all(np.abs(f - f64).max(axis=-1) <= eb)


@pytest.mark.parametrize("wl", ["flow", "depth"])
def test_iwe_elementwise(wl):
    if wl == "flow":
        win = small_flow_window(96, 80, 7000, 6, ALL, seed=3)
    else:
        win = small_depth_window(120, 90, 9000, 10, seed=4)
    # on the window without its flagged events every support decision is the
    # same in FP32 and FP64: identical support, values within FP32 error
    sub = unflagged(win, run_oracle(win, grad=False, bounds=True)["bounds"]["flags"])
    assert sub.events.n > 0.99 * win.events.n
    g = run_gpu(sub, grad=False, want_iwe=True)
    o = run_oracle(sub, grad=False, want_iwe=True)
    gi, oi = g["iwe"], o["iwe"]
    assert gi.shape == oi.shape
    assert np.array_equal(gi != 0, oi != 0)
    np.testing.assert_allclose(gi, oi, rtol=1e-5, atol=2e-6)


def test_flow_window_128():
    # 128x128 sensor, 20,000 events, sinusoid flow, one bin, window-end reference
    win = synth.flow_window()
    check_window(win)


def test_davis_window_346():
    # 346x260 DAVIS sensor, 100,000 gradient-sampled events, depth + ego, 10 bins, 11 references
    win = synth.davis_window()
    assert check_window(win) < 0.001 * win.events.n


@pytest.mark.parametrize("B,ref_mode,nfb", [(4, ALL, 4), (5, END, 1), (5, END, 5), (3, ALL, 1), (2, ALL, 2)])
def test_bins_refs_and_per_bin_flows(B, ref_mode, nfb):
    win = small_flow_window(70, 50, 5000, B, ref_mode, nfb=nfb, seed=B * 10 + nfb)
    check_window(win)


@pytest.mark.parametrize("B", [20, 32])
def test_many_bins(B):
    win = small_depth_window(160, 120, 6000, B, seed=B)
    check_window(win)


@pytest.mark.parametrize("n", [1, 31, 255, 257, 1023])
def test_ragged_event_counts(n):
    win = small_depth_window(64, 48, n, 10, seed=n)
    check_window(win)


def test_empty_window():
    win = small_flow_window(32, 24, 0, 4, ALL)
    g = run_gpu(win)
    assert g["loss"] == 0.0 and not np.any(g["dflow"]) and not np.any(g["nnz_r"])


def test_all_events_masked():
    # a flow of 100 px per window pushes every event out of a 40x30 image
    win = small_flow_window(40, 30, 2000, 4, ALL)
    win.flow = np.full_like(win.flow, 100.0)
    g = run_gpu(win)
    o = run_oracle(win)
    assert o["valid"].sum() == 0
    assert g["loss"] == 0.0 and not np.any(g["nnz_r"]) and not np.any(g["dflow"])


def test_zero_flow_window():
    # every point is the event's own pixel, exact in any precision: nothing is
    # flagged and the full window must match exactly
    win = small_flow_window(50, 40, 3000, 5, ALL)
    win.flow = np.zeros_like(win.flow)
    assert check_window(win) == 0


def test_out_of_range_events_are_masked():
    win = small_flow_window(48, 32, 1000, 3, ALL, seed=8)
    win.events.x[:10] = 48       # one past the last column
    win.events.y[10:20] = -1     # above the first row
    win.events.x[20:30] = 32767
    o = run_oracle(win, grad=False)
    assert not o["valid"][:30].any()
    check_window(win)


def test_smallest_sensor():
    win = small_flow_window(2, 2, 50, 2, ALL, mag=0.3)
    check_window(win)


def test_events_on_window_edges():
    win = small_flow_window(64, 48, 600, 8, ALL, seed=12)
    t = win.events.t.copy()
    t[:100] = win.events.t0
    t[-100:] = win.events.t1
    t[200:300] = np.float32(0.005)  # an interior bin edge (tau = 0.5 for 8 bins)
    win.events.t = np.sort(t)
    check_window(win)


def test_dloss_scales_gradient():
    win = small_depth_window(80, 60, 4000, 10, seed=5)
    g1 = run_gpu(win, dloss=1.0)
    g2 = run_gpu(win, dloss=-2.5)
    assert g1["loss"] == g2["loss"]
    assert rel_l2(g2["dinv_depth"], -2.5 * g1["dinv_depth"]) < 1e-6
    assert rel_l2(g2["dego"], -2.5 * g1["dego"]) < 1e-6


def test_eps_is_used():
    win = small_flow_window(60, 45, 3000, 4, ALL, seed=6)
    check_window(win, eps=1e-3)
    # and the loss does depend on it
    assert run_gpu(win, eps=1e-3, grad=False)["loss"] != run_gpu(win, eps=1e-9, grad=False)["loss"]


def test_autograd_function_matches_backward():
    import torch
    cm = gpu_lib()
    win = small_depth_window(100, 80, 5000, 10, seed=7)
    win = unflagged(win, run_oracle(win, grad=False, bounds=True)["bounds"]["flags"])
    cfg = cm.loss_cfg(win.nbins, win.ref_mode, cm.SPLAT_ATOMIC, GRAD_EPS)
    ws = cm.Workspace(win.cam, cfg, win.events.n)
    ev = cm.DeviceEvents.from_host(win.events)
    rho = torch.from_numpy(win.inv_depth).cuda().requires_grad_(True)
    ego = torch.from_numpy(win.ego).cuda().requires_grad_(True)
    loss = cm.cm_loss(ev, ws, inv_depth=rho, ego=ego, dt=win.dt)
    (3.0 * loss).backward()
    o = run_oracle(win, dloss=3.0, eps=GRAD_EPS)
    assert abs(loss.item() - o["loss"]) <= 1e-5 * o["loss"]
    assert rel_l2(rho.grad.cpu().numpy(), o["dinv_depth"]) < 1e-4
    assert rel_l2(ego.grad.cpu().numpy(), o["dego"]) < 1e-4


# ---- stored warps (the forward keeps the trajectory points for the backward) ----

@pytest.mark.parametrize("B,ref_mode,nfb", [(10, ALL, 1), (5, END, 1), (4, ALL, 4), (1, END, 1)])
def test_stored_warps_flow_window(B, ref_mode, nfb):
    win = small_flow_window(90, 70, 6000, B, ref_mode, nfb=nfb, seed=40 + B, mag=6.0)
    check_window(win, plain(store_warps=True))


def test_stored_warps_depth_window_and_masked_events():
    # a strong ego-motion pushes part of the events out of the image: the mask
    # read back from the stored points must repeat the forward's decision
    win = small_depth_window(120, 90, 9000, 10, seed=41)
    win.ego[:3] *= 4.0
    assert run_oracle(win, grad=False)["valid"].mean() < 0.9
    check_window(win, plain(store_warps=True))
    g = run_gpu(win, store_warps=True)
    r = run_gpu(win)  # recompute: same decisions, same values up to the reduction order
    assert np.array_equal(g["nnz_r"], r["nnz_r"])
    assert rel_l2(g["dinv_depth"], r["dinv_depth"]) <= 1e-5


def test_stored_warps_sort_path_is_bitwise_recompute():
    # the sort path is deterministic, and the stored points are the recomputed
    # points: both backwards give the same bits
    cm = gpu_lib()
    win = small_depth_window(100, 80, 7000, 10, seed=42)
    a = run_gpu(win, splat=cm.SPLAT_SORT, store_warps=True)
    b = run_gpu(win, splat=cm.SPLAT_SORT)
    assert a["loss"] == b["loss"]
    for k in ("dflow", "dinv_depth", "dego"):
        assert np.array_equal(a[k], b[k]), k
