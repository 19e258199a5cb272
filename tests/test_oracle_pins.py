"""Pins of the CPU oracle against what the paper and the mathematics fix.

The paper prints no worked numeric example for the loss, so every pin here is
a closed form, a brute-force evaluation written independently in the test, an
invariant the paper's own data augmentations imply (polarity flip, left-right
flip, time reversal; supp. "Implementation details"), or a finite-difference
check of the analytic gradient.  Each is chosen so that a plausible mistake
in the oracle (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth

END, ALL = O.REF_END, O.REF_ALL


def ev(xs, ys, ts, ps, t0=0.0, t1=1.0):
    return synth.Events(np.array(xs, np.int16), np.array(ys, np.int16), np.array(ts, np.float32),
                        np.array(ps, np.int8), t0, t1)


def uniform_flow(W, H, ux, uy, nfb=None):
    f = np.zeros((H, W, 2))
    f[..., 0], f[..., 1] = ux, uy
    return f if nfb is None else np.broadcast_to(f, (nfb, H, W, 2)).copy()


def brute_weights(px, py):
    """Bilinear splat of a point, written out independently: {(col, row): weight}."""
    x0, y0 = math.floor(px), math.floor(py)
    ax, ay = px - x0, py - y0
    out = {}
    for dx, wx in ((0, 1 - ax), (1, ax)):
        for dy, wy in ((0, 1 - ay), (1, ay)):
            if wx * wy != 0:
                out[(x0 + dx, y0 + dy)] = out.get((x0 + dx, y0 + dy), 0.0) + wx * wy
    return out


# --------------------------------------------------------------------------
# S4 bilinear splat and S5 loss: brute force on tiny inputs


def test_single_event_splat_brute_force():
    # one event at pixel (5, 7), tau = 0.25, uniform flow (2.5, -1.25) px/window;
    # one reference at the window end:
    # warped position (5 + 0.75*2.5, 7 - 0.75*1.25) = (6.875, 6.0625)
    W, H = 16, 12
    e = ev([5], [7], [0.25], [1])
    r = O.cm(e, uniform_flow(W, H, 2.5, -1.25), width=W, height=H, nbins=1, ref_mode=END,
             want_iwe=True)
    expect = brute_weights(6.875, 6.0625)
    tbar = 0.25  # 1 - |1 - 0.25|
    iwe = r["iwe"][0]
    assert len(expect) == 4
    for (cx, cy), w in expect.items():
        assert iwe[cy, cx, 0] == pytest.approx(w, abs=1e-15)
        assert iwe[cy, cx, 1] == pytest.approx(w * tbar, abs=1e-15)
    mask = np.ones((H, W), bool)
    for cx, cy in expect:
        mask[cy, cx] = False
    assert np.all(iwe[mask] == 0) and np.all(iwe[..., 2:] == 0)
    # four isolated pixels each with T = w tbar / (w + eps); N_nz = 4
    eps = 1e-9
    L = sum((w * tbar / (w + eps)) ** 2 for w in expect.values()) / (4 + eps)
    assert r["loss"] == pytest.approx(L, rel=1e-14)
    assert r["nnz_r"][0] == 4


def test_two_events_one_pixel_hand_example():
    # zero flow, two positive events at the same pixel, one at the window end reference:
    # t-bar = tau, C = 2, S = tau1 + tau2, T = S / (2 + eps), N_nz = 1
    W, H = 8, 8
    e = ev([3, 3], [4, 4], [0.25, 0.75], [1, 1])
    r = O.cm(e, uniform_flow(W, H, 0, 0), width=W, height=H, nbins=1, ref_mode=END)
    eps = 1e-9
    T = (0.25 + 0.75) / (2 + eps)
    assert r["loss"] == pytest.approx(T * T / (1 + eps), rel=1e-15)
    # opposite polarities at the same pixel: two polarity images, one non-empty pixel
    e = ev([3, 3], [4, 4], [0.25, 0.75], [1, -1])
    r = O.cm(e, uniform_flow(W, H, 0, 0), width=W, height=H, nbins=1, ref_mode=END)
    Tp, Tm = 0.25 / (1 + eps), 0.75 / (1 + eps)
    assert r["loss"] == pytest.approx((Tp * Tp + Tm * Tm) / (1 + eps), rel=1e-15)


def test_zero_flow_gives_raw_event_image():
    # zero flow: every reference image is the per-polarity event-count image, and
    # S_p(x) = sum over the events at x of 1 - |tau_r - tau_k|
    W, H, B = 20, 15, 4
    rng = np.random.default_rng(7)
    n = 300
    e = synth.uniform_events(rng, W, H, n, 0.0, 0.01)
    r = O.cm(e, uniform_flow(W, H, 0, 0), width=W, height=H, nbins=B, ref_mode=ALL,
             want_iwe=True)
    tau = (e.t.astype(np.float64) - e.t0) / (e.t1 - e.t0)
    pix = e.y.astype(np.int64) * W + e.x
    eps = 1e-9
    L = 0.0
    for rr in range(B + 1):
        tbar = 1 - np.abs(rr / B - tau)
        for pol, sgn in ((0, 1), (1, -1)):
            sel = e.p == sgn
            C = np.bincount(pix[sel], minlength=W * H)
            S = np.bincount(pix[sel], weights=tbar[sel], minlength=W * H)
            assert np.array_equal(r["iwe"][rr, ..., 2 * pol].ravel(), C)
            np.testing.assert_allclose(r["iwe"][rr, ..., 2 * pol + 1].ravel(), S, rtol=1e-14, atol=1e-15)
        Cp = np.bincount(pix[e.p > 0], minlength=W * H)
        Cm = np.bincount(pix[e.p < 0], minlength=W * H)
        Sp = np.bincount(pix[e.p > 0], weights=tbar[e.p > 0], minlength=W * H)
        Sm = np.bincount(pix[e.p < 0], weights=tbar[e.p < 0], minlength=W * H)
        nnz = np.count_nonzero(Cp + Cm)
        assert r["nnz_r"][rr] == nnz
        L += ((Sp / (Cp + eps)) ** 2 + (Sm / (Cm + eps)) ** 2).sum() / (nnz + eps)
    assert r["loss"] == pytest.approx(L / (B + 1), rel=1e-13)
    assert r["valid"].all()


def test_splat_conserves_mass():
    # per reference: sum of counts = number of valid events (per polarity), and
    # sum of timestamp images = sum of the valid events' average timestamps
    W, H, B = 48, 36, 5
    rng = np.random.default_rng(11)
    e = synth.uniform_events(rng, W, H, 3000, 0.0, 0.01)
    flow = synth.sinusoid_flow(rng, W, H, 4.0)
    r = O.cm(e, flow, width=W, height=H, nbins=B, ref_mode=ALL, want_iwe=True)
    valid = r["valid"].astype(bool)
    assert 0.5 < valid.mean() < 1.0  # some events leave the image, most stay
    tau = (e.t.astype(np.float64) - e.t0) / (e.t1 - e.t0)
    for rr in range(B + 1):
        tbar = 1 - np.abs(rr / B - tau)
        for pol, sgn in ((0, 1), (1, -1)):
            sel = valid & (e.p == sgn)
            assert r["iwe"][rr, ..., 2 * pol].sum() == pytest.approx(sel.sum(), rel=1e-12)
            assert r["iwe"][rr, ..., 2 * pol + 1].sum() == pytest.approx(tbar[sel].sum(), rel=1e-12)


def test_mask_at_any_point():
    # an event pushed out of the image by the forward chain is dropped from every
    # reference image, including the ones where it would lie inside (Sec. 3.1)
    W, H, B = 16, 8, 4
    e = ev([1, 8], [4, 4], [0.5, 0.5], [1, 1])
    r = O.cm(e, uniform_flow(W, H, -10.0, 0.0), width=W, height=H, nbins=B, ref_mode=ALL,
             want_iwe=True)
    # event 0: x at tau=1 is 1 - 5 = -4 (outside); at tau=0 it is 6 (inside); event 1 stays inside
    assert list(r["valid"]) == [0, 1]
    for rr in range(B + 1):
        assert r["iwe"][rr, ..., 0].sum() == pytest.approx(1.0)
    # the window-end-only reference never looks at the backward chain
    e2 = ev([14], [4], [0.5], [1])
    r2 = O.cm(e2, uniform_flow(W, H, 10.0, 0.0), width=W, height=H, nbins=B, ref_mode=END)
    assert list(r2["valid"]) == [0]  # 14 + 5 = 19 > 15
    r3 = O.cm(e2, uniform_flow(W, H, -10.0, 0.0), width=W, height=H, nbins=B, ref_mode=END)
    assert list(r3["valid"]) == [1]  # 14 - 5 = 9; the backward point (19) is not computed


def test_closed_image_interval():
    # a point exactly on the last column is inside (closed interval), one ulp beyond is not
    W, H = 10, 6
    e = ev([5, 5], [2, 2], [0.0, 0.0], [1, 1])
    r = O.cm(e, uniform_flow(W, H, 4.0, 0.0), width=W, height=H, nbins=1, ref_mode=END,
             want_iwe=True)
    assert list(r["valid"]) == [1, 1]
    assert r["iwe"][0, 2, 9, 0] == 2.0  # all weight on the border pixel
    r = O.cm(e, uniform_flow(W, H, 4.0 + 1e-12, 0.0), width=W, height=H, nbins=1, ref_mode=END)
    assert list(r["valid"]) == [0, 0]


def test_bin_of_edge_events():
    # b = min(floor(tau B), B - 1): an event at tau = 1 sits in the last bin and is
    # not moved to the window end; an event on an interior edge starts its backward
    # chain with a zero-length push
    W, H, B = 32, 8, 4
    e = ev([10, 10], [3, 3], [1.0, 0.5], [1, 1])
    r = O.cm(e, uniform_flow(W, H, 2.0, 0.0), width=W, height=H, nbins=B, ref_mode=ALL,
             want_pos=True)
    np.testing.assert_allclose(r["pos"][0, :, 0], [10 - 2.0 * (1 - j / B) for j in range(B + 1)], atol=1e-14)
    np.testing.assert_allclose(r["pos"][1, :, 0], [10 + 2.0 * (j / B - 0.5) for j in range(B + 1)], atol=1e-14)


# --------------------------------------------------------------------------
# S2 trajectory


@pytest.mark.parametrize("B", [1, 3, 10])
def test_iterative_warp_uniform_flow_is_linear(B):
    # sampling a constant field is position independent, so the bin-by-bin push
    # equals the single linear warp x_j = x_k + (tau_j - tau_k) u
    W, H = 64, 48
    rng = np.random.default_rng(3)
    e = synth.uniform_events(rng, W - 20, H - 20, 200, 0.0, 0.01)
    e.x += 10
    e.y += 10
    u = (3.25, -2.5)
    r = O.cm(e, uniform_flow(W, H, *u), width=W, height=H, nbins=B, ref_mode=ALL, want_pos=True)
    tau = (e.t.astype(np.float64) - e.t0) / (e.t1 - e.t0)
    for j in range(B + 1):
        np.testing.assert_allclose(r["pos"][:, j, 0], e.x + (j / B - tau) * u[0], atol=1e-12)
        np.testing.assert_allclose(r["pos"][:, j, 1], e.y + (j / B - tau) * u[1], atol=1e-12)


def test_iterative_warp_affine_flow_is_euler():
    # bilinear interpolation reproduces an affine field exactly, so the iterative
    # warp is explicit Euler for dx/dtau = A x + c with step 1/B after a partial
    # first step from the event: written out here independently
    W, H, B = 80, 60, 6
    A = np.array([[0.05, -0.08], [0.06, 0.03]])
    c = np.array([-1.5, 0.75])
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    flow = np.stack([A[0, 0] * xx + A[0, 1] * yy + c[0], A[1, 0] * xx + A[1, 1] * yy + c[1]], -1)
    rng = np.random.default_rng(5)
    e = synth.uniform_events(rng, 30, 20, 50, 0.0, 0.01)
    e.x += 25
    e.y += 20
    r = O.cm(e, flow, width=W, height=H, nbins=B, ref_mode=ALL, want_pos=True)
    tau = (e.t.astype(np.float64) - e.t0) / (e.t1 - e.t0)
    for k in range(e.n):
        b = min(int(math.floor(tau[k] * B)), B - 1)
        xk = np.array([e.x[k], e.y[k]], float)
        u = A @ xk + c
        pos = {b + 1: xk + ((b + 1) / B - tau[k]) * u, b: xk - (tau[k] - b / B) * u}
        for j in range(b + 1, B):
            pos[j + 1] = pos[j] + (A @ pos[j] + c) / B
        for j in range(b, 0, -1):
            pos[j - 1] = pos[j] - (A @ pos[j] + c) / B
        for j in range(B + 1):
            np.testing.assert_allclose(r["pos"][k, j], pos[j], atol=1e-11)


def test_per_bin_flows_use_bin_field():
    # with one field per bin, the push across bin j uses field j (forward and backward)
    W, H, B = 64, 32, 4
    speeds = [1.0, -2.0, 4.0, 0.5]
    flow = np.stack([uniform_flow(W, H, s, 0.0) for s in speeds])
    e = ev([30], [10], [0.3], [1])  # bin 1
    r = O.cm(e, flow, width=W, height=H, nbins=B, ref_mode=ALL, want_pos=True)
    x = {1: 30.0}
    # forward: partial bin 1 (0.3 -> 0.5), then bins 2, 3; backward: partial bin 1 (0.3 -> 0.25), then bin 0
    x[2] = 30 + (0.5 - 0.3) * speeds[1]
    x[3] = x[2] + 0.25 * speeds[2]
    x[4] = x[3] + 0.25 * speeds[3]
    x[1] = 30 - (0.3 - 0.25) * speeds[1]
    x[0] = x[1] - 0.25 * speeds[0]
    np.testing.assert_allclose(r["pos"][0, :, 0], [x[j] for j in range(B + 1)], atol=1e-6)


# --------------------------------------------------------------------------
# straddles: the flags and the loss interval of orc_cm_bounds


def test_bounds_hand_case_one_event_next_to_an_integer():
    # one event at (3, 3), tau = 0.5, B = 1, window-end reference, uniform flow
    # (4 - 2e-8, 0): the end point is (5 - 1e-8, 3).  Its x lies 1e-8 from the
    # integer 5, far inside the FP32 error margin of a 2-px push, so bit 0 is set;
    # y is exact (zero flow component, no rounding), so no row is in doubt.
    # FP64 support: (5, 3) with weight 1 - 1e-8 and (4, 3) with 1e-8.  Outcomes
    # of the flagged floor: the small weight at (4, 3), at (6, 3) or nowhere, so
    # N_nz lies in [1, 3], (5, 3) is sure, and each of the other two pixels adds
    # a term T^2 in [0, (tbar w/(w + eps))^2] for its weight w up to the margin.
    W, H, eps = 10, 8, 1e-9
    d = 1e-8
    e = ev([3], [3], [0.5], [1])
    flow = uniform_flow(W, H, 2 * (2 - d), 0.0)
    kw = dict(width=W, height=H, nbins=1, ref_mode=END, eps=eps)
    b = O.cm_bounds(e, flow, want_err=True, **kw)
    r = O.cm(e, flow, **kw)
    assert list(b["flags"]) == [1] and b["counts"] == (1, 0, 0, 1)
    assert list(b["nnz_lo"]) == [1] and list(b["nnz_hi"]) == [3]
    assert list(r["nnz_r"]) == [2]
    tbar = 0.5
    w_sure = 1 - d
    t_sure = tbar * w_sure / (w_sure + eps)
    m = O.SAFETY * (b["err"][0, 1, 0] + 2.0 ** -24)  # the margin of the flagged x
    assert b["err"][0, 1, 1] == 0.0 and 1e-7 < m < 1e-4
    t_hi = [tbar * (d + m) / (d + m + eps), tbar * (m - d) / (m - d + eps)]  # (4, 3) and (6, 3)
    assert b["loss_lo"] == pytest.approx(t_sure ** 2 / (3 + eps), rel=1e-12)
    assert b["loss_hi"] == pytest.approx((t_sure ** 2 + t_hi[0] ** 2 + t_hi[1] ** 2) / (1 + eps), rel=1e-12)
    assert b["loss_lo"] <= r["loss"] <= b["loss_hi"]


def test_bounds_collapse_to_the_fp64_loss_without_error():
    # zero flow: every point is the event's own pixel, exact in any precision, so
    # nothing is flagged and the interval is the FP64 loss itself; a margin of 0
    # (safety 0) collapses the interval for any flow
    W, H, B = 30, 20, 4
    rng = np.random.default_rng(3)
    e = synth.uniform_events(rng, W, H, 800)
    for flow, safety in ((np.zeros((H, W, 2)), O.SAFETY), (synth.sinusoid_flow(rng, W, H, 3.0), 0.0)):
        kw = dict(width=W, height=H, nbins=B, ref_mode=ALL)
        b = O.cm_bounds(e, flow, safety=safety, **kw)
        r = O.cm(e, flow, **kw)
        assert not b["flags"].any()
        assert np.array_equal(b["nnz_lo"], r["nnz_r"]) and np.array_equal(b["nnz_hi"], r["nnz_r"])
        assert b["loss_lo"] == pytest.approx(r["loss"], rel=1e-14)
        assert b["loss_hi"] == pytest.approx(r["loss"], rel=1e-14)


@pytest.mark.parametrize("wl", ["flow", "depth", "end"])
def test_bounds_contain_every_perturbed_evaluation(wl):
    # brute force over the error model: perturb the flow by up to the stated
    # bound (random per pixel, 1e-3 relative, large enough that many floors and
    # supports flip) and evaluate the FP64 definition on each perturbed flow:
    # every trajectory point moves by at most its error bound, and every
    # N_nz(r) and loss lands in the interval computed from the unperturbed flow
    rng = np.random.default_rng({"flow": 1, "depth": 2, "end": 3}[wl])
    if wl == "depth":
        w = synth.depth_window(rng, 64, 48, 3000, nbins=6)
        flow = O.flow_from_depth(w.cam, w.inv_depth, w.ego, w.dt)[None]
    else:
        W, H = 56, 40
        w = synth.Window(synth.Camera(W, H, 40.0, 40.0, W / 2, H / 2), synth.uniform_events(rng, W, H, 3000),
                         5, END if wl == "end" else ALL, flow=synth.sinusoid_flow(rng, W, H, 4.0)[None])
        flow = w.flow.astype(np.float64)
    eb = 1e-3 * np.abs(flow).max(axis=-1) + 1e-6
    kw = dict(width=w.cam.width, height=w.cam.height, nbins=w.nbins, ref_mode=w.ref_mode)
    b = O.cm_bounds(w.events, flow, eflow=eb, want_err=True, **kw)
    base = O.cm(w.events, flow, want_pos=True, **kw)
    assert b["counts"][3] > 50  # the perturbation scale flags many events
    flips = 0
    for s in range(6):
        u = np.random.default_rng(100 + s).uniform(-1, 1, flow.shape)
        r = O.cm(w.events, flow + u * eb[..., None], want_pos=True, **kw)
        both = np.isfinite(r["pos"]) & np.isfinite(base["pos"])
        assert np.all(np.abs(r["pos"] - base["pos"])[both] <= b["err"][both])
        assert np.all((b["nnz_lo"] <= r["nnz_r"]) & (r["nnz_r"] <= b["nnz_hi"]))
        assert b["loss_lo"] <= r["loss"] <= b["loss_hi"]
        flips += int(np.sum(np.floor(r["pos"][both]) != np.floor(base["pos"][both])))
    assert flips > 0  # the perturbations did move points across cell boundaries


@pytest.mark.parametrize("wl", ["flow", "davis", "batch"])
def test_bounds_contain_the_fp64_result_and_flag_few_events(wl):
    if wl == "flow":
        w = synth.flow_window(n=4000)
    elif wl == "davis":
        w = synth.depth_window(np.random.default_rng(9), 120, 90, 4000)
    else:
        w = synth.batch_windows(2)[1]
    r = O.cm_window(w, bounds=True)
    b = r["bounds"]
    assert np.all((b["nnz_lo"] <= r["nnz_r"]) & (r["nnz_r"] <= b["nnz_hi"]))
    assert b["loss_lo"] <= r["loss"] <= b["loss_hi"]
    assert np.all((b["loss_r_lo"] <= r["loss_r"]) & (r["loss_r"] <= b["loss_r_hi"]))
    assert b["counts"][3] < 0.01 * w.events.n


# --------------------------------------------------------------------------
# S1 motion field


def test_flow_pure_translation_and_rotation():
    cam = synth.Camera(40, 30, 50.0, 50.0, 19.5, 14.0)
    rho = np.full((30, 40), 0.8)
    dt = 0.01
    u, v = np.meshgrid(np.arange(40.0), np.arange(30.0))
    xn, yn = (u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy
    # lateral translation: uniform flow -dt fx rho vx
    f = O.flow_from_depth(cam, rho, [1.5, 0, 0, 0, 0, 0], dt)
    np.testing.assert_allclose(f[..., 0], -dt * cam.fx * 0.8 * 1.5, rtol=1e-14)
    np.testing.assert_allclose(f[..., 1], 0, atol=1e-15)
    # forward translation: radial field through the principal point
    f = O.flow_from_depth(cam, rho, [0, 0, 2.0, 0, 0, 0], dt)
    np.testing.assert_allclose(f[..., 0], dt * 0.8 * 2.0 * (u - cam.cx), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(f[..., 1], dt * 0.8 * 2.0 * (v - cam.cy), rtol=1e-13, atol=1e-15)
    # roll about the optical axis (fx = fy): rotation field about (cx, cy), independent of rho
    rho2 = np.random.default_rng(0).uniform(0.2, 2, (30, 40))
    f = O.flow_from_depth(cam, rho2, [0, 0, 0, 0, 0, 3.0], dt)
    np.testing.assert_allclose(f[..., 0], dt * 3.0 * (v - cam.cy), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(f[..., 1], -dt * 3.0 * (u - cam.cx), rtol=1e-13, atol=1e-15)
    # yaw alone
    f = O.flow_from_depth(cam, rho2, [0, 0, 0, 0, 1.0, 0], dt)
    np.testing.assert_allclose(f[..., 0], -dt * cam.fx * (1 + xn * xn), rtol=1e-13)
    np.testing.assert_allclose(f[..., 1], -dt * cam.fy * xn * yn, rtol=1e-13, atol=1e-15)


def test_motion_field_is_first_order_eq2():
    # Eq. 2 with the camera displaced by (v dt, w dt) agrees with the motion field
    # to first order: the difference shrinks as dt^2
    cam = synth.camera_for(346, 260)
    rng = synth.rng_for(2)
    rho = synth.inv_depth_map(rng, 346, 260).astype(np.float64)
    ego = np.array([0.7, -0.4, 1.1, 0.5, -0.8, 0.3])
    errs = []
    for dt in (0.02, 0.01, 0.005):
        d = np.abs(O.flow_eq2(cam, rho, ego, dt) - O.flow_from_depth(cam, rho, ego, dt)).max()
        scale = np.abs(O.flow_from_depth(cam, rho, ego, dt)).max()
        assert d < 0.05 * scale
        errs.append(d)
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_motion_field_error_bound_covers_a_single_precision_evaluation():
    # the bound is for any FP32 evaluation: check it against numpy float32
    # arithmetic of the textbook formula (a different order from any kernel)
    cam = synth.camera_for(346, 260)
    rng = synth.rng_for(2)
    rho = synth.inv_depth_map(rng, 346, 260)
    ego = synth.ego_motion(rng)
    f64 = O.flow_from_depth(cam, rho, ego, 0.01)
    eb = O.flow_error_bound(cam, rho, ego, 0.01)
    f = np.float32
    v, u = np.mgrid[0:260, 0:346].astype(np.float32)
    xn, yn = (u - f(cam.cx)) / f(cam.fx), (v - f(cam.cy)) / f(cam.fy)
    e = ego.astype(np.float32)
    r = rho.astype(np.float32)
    xd = r * (-e[0] + xn * e[2]) + xn * yn * e[3] - (f(1) + xn * xn) * e[4] + yn * e[5]
    yd = r * (-e[1] + yn * e[2]) + (f(1) + yn * yn) * e[3] - xn * yn * e[4] - xn * e[5]
    f32 = np.stack([f(0.01) * f(cam.fx) * xd, f(0.01) * f(cam.fy) * yd], -1)
    d = np.abs(f32.astype(np.float64) - f64).max(axis=-1)
    assert np.all(d <= eb)
    assert eb.max() < 1e-5 * np.abs(f64).max()  # and the bound is FP32-tight


# --------------------------------------------------------------------------
# invariants from the paper's augmentations (polarity flip, left-right flip,
# time reversal) and from the loss being a sum over events


def _small_case(seed=21, B=4, nfb=1):
    W, H = 40, 30
    rng = np.random.default_rng(seed)
    e = synth.uniform_events(rng, W, H, 1500, 0.0, 0.01)
    flows = [synth.sinusoid_flow(rng, W, H, 3.0).astype(np.float64) for _ in range(nfb)]
    return W, H, B, e, np.stack(flows)


@pytest.mark.parametrize("nfb", [1, 4])
def test_polarity_flip_invariance(nfb):
    W, H, B, e, f = _small_case(nfb=nfb)
    kw = dict(width=W, height=H, nbins=B, ref_mode=ALL, grad=True)
    r1 = O.cm(e, f, **kw)
    e2 = synth.Events(e.x, e.y, e.t, (-e.p).astype(np.int8), e.t0, e.t1)
    r2 = O.cm(e2, f, **kw)
    assert r2["loss"] == pytest.approx(r1["loss"], rel=1e-14)
    np.testing.assert_allclose(r2["dflow"], r1["dflow"], rtol=1e-10, atol=1e-14 * np.abs(r1["dflow"]).max())


@pytest.mark.parametrize("nfb", [1, 4])
def test_left_right_flip_invariance(nfb):
    W, H, B, e, f = _small_case(nfb=nfb)
    kw = dict(width=W, height=H, nbins=B, ref_mode=ALL, grad=True)
    r1 = O.cm(e, f, **kw)
    e2 = synth.Events((W - 1 - e.x).astype(np.int16), e.y, e.t, e.p, e.t0, e.t1)
    f2 = f[:, :, ::-1].copy()
    f2[..., 0] *= -1
    r2 = O.cm(e2, f2, **kw)
    assert r2["loss"] == pytest.approx(r1["loss"], rel=1e-12)
    g2 = r2["dflow"][:, :, ::-1].copy()
    g2[..., 0] *= -1
    np.testing.assert_allclose(g2, r1["dflow"], rtol=1e-7, atol=1e-9 * np.abs(r1["dflow"]).max())


@pytest.mark.parametrize("nfb", [1, 4])
def test_time_reversal_invariance(nfb):
    # tau -> 1 - tau, flow -> -flow (and bin j's field -> bin B-1-j), all edges
    W, H, B, e, f = _small_case(nfb=nfb)
    kw = dict(width=W, height=H, nbins=B, ref_mode=ALL)
    r1 = O.cm(e, f, **kw)
    # reverse in a window [0, 1] with timestamps on a 2^-20 grid, so that t -> 1 - t is exact
    e1 = synth.Events(e.x, e.y, (np.round(e.t / np.float32(0.01) * 2**20) / 2**20).astype(np.float32), e.p,
                      0.0, 1.0)
    r1b = O.cm(e1, f, **kw)
    order = np.arange(e.n)[::-1]
    e2 = synth.Events(e1.x[order], e1.y[order], (np.float32(1.0) - e1.t[order]).astype(np.float32), e1.p[order],
                      0.0, 1.0)
    r2 = O.cm(e2, -f[::-1], **kw)
    assert r2["loss"] == pytest.approx(r1b["loss"], rel=1e-12)
    assert r1b["loss"] == pytest.approx(r1["loss"], rel=1e-4)


def test_event_permutation_invariance():
    W, H, B, e, f = _small_case()
    kw = dict(width=W, height=H, nbins=B, ref_mode=ALL, grad=True)
    r1 = O.cm(e, f, **kw)
    perm = np.random.default_rng(1).permutation(e.n)
    r2 = O.cm(e.take(perm), f, **kw)
    assert r2["loss"] == pytest.approx(r1["loss"], rel=1e-13)
    np.testing.assert_allclose(r2["dflow"], r1["dflow"], rtol=1e-9, atol=1e-13 * np.abs(r1["dflow"]).max())


# --------------------------------------------------------------------------
# S6 / S7 gradients: frozen-branch finite differences of the oracle itself


def _fd_directional(fun, x0, v, h):
    return (fun(x0 + h * v) - fun(x0 - h * v)) / (2 * h)


@pytest.mark.parametrize("nfb,ref_mode,eps", [(1, ALL, 1e-3), (4, ALL, 1e-3), (1, END, 1e-3), (1, ALL, 1e-9)])
def test_flow_gradient_matches_frozen_fd(nfb, ref_mode, eps):
    W, H, B, e, f = _small_case(seed=33, nfb=nfb)
    kw = dict(width=W, height=H, nbins=B, ref_mode=ref_mode, eps=eps)
    base = O.cm(e, f, grad=True, record=True, **kw)
    br = base["branch"]
    g = base["dflow"]

    def L(flow):
        return O.cm(e, flow, replay=br, **kw)["loss"]

    assert L(f) == base["loss"]
    rng = np.random.default_rng(2)
    for _ in range(4):
        v = rng.standard_normal(f.shape)
        fd = _fd_directional(L, f, v, 1e-6)
        an = float((g * v).sum())
        assert fd == pytest.approx(an, rel=2e-6 if eps > 1e-6 else 1e-4)
    # single entries with the largest gradients
    flat = np.argsort(np.abs(g).ravel())[-6:]
    for i in flat:
        v = np.zeros(f.size)
        v[i] = 1
        v = v.reshape(f.shape)
        assert _fd_directional(L, f, v, 1e-6) == pytest.approx(g.ravel()[i], rel=1e-5)


def test_depth_ego_gradient_matches_frozen_fd():
    cam = synth.Camera(48, 36, 40.0, 40.0, 24.0, 18.0)
    rng = np.random.default_rng(44)
    e = synth.gradient_events(rng, 48, 36, 1200)
    rho = synth.inv_depth_map(rng, 48, 36).astype(np.float64)
    ego = np.array([0.4, -0.3, 0.8, 0.5, 0.2, -0.6])
    dt, B, eps = 0.05, 5, 1e-3
    base = O.cm_depth(e, cam, rho, ego, dt, nbins=B, ref_mode=ALL, eps=eps, grad=True, record=True)
    br = base["branch"]

    def L(rho_, ego_):
        fl = O.flow_from_depth(cam, rho_, ego_, dt)
        return O.cm(e, fl, width=48, height=36, nbins=B, ref_mode=ALL, eps=eps, replay=br)["loss"]

    for i in range(6):
        v = np.zeros(6)
        v[i] = 1
        fd = (L(rho, ego + 1e-6 * v) - L(rho, ego - 1e-6 * v)) / 2e-6
        assert fd == pytest.approx(base["dego"][i], rel=1e-5, abs=1e-9 * np.abs(base["dego"]).max())
    for _ in range(3):
        v = rng.standard_normal(rho.shape)
        fd = (L(rho + 1e-6 * v, ego) - L(rho - 1e-6 * v, ego)) / 2e-6
        assert fd == pytest.approx(float((base["dinv_depth"] * v).sum()), rel=1e-5)


# --------------------------------------------------------------------------
# hand-derived worked cases (tests/golden/hand_cases.json, each with its
# derivation and the passage it follows)


def _golden_cases():
    import json
    import os
    p = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")
    return json.load(open(p))["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_hand_cases(case):
    W, H = case["W"], case["H"]
    xs, ys, ts, ps = zip(*case["events"])
    e = ev(xs, ys, ts, ps)
    mode = END if case["ref_mode"] == "end" else ALL
    r = O.cm(e, uniform_flow(W, H, *case["flow"]), width=W, height=H, nbins=case["nbins"], ref_mode=mode,
             want_iwe=True)
    assert list(r["nnz_r"]) == case["nnz"]
    assert r["loss"] == pytest.approx(case["loss"], rel=case["loss_rtol"], abs=1e-12)
    iwe = r["iwe"]
    expect = np.zeros_like(iwe)
    for rr, x, y, pol, C, S in case["iwe"]:
        k = 0 if pol > 0 else 2
        expect[rr, y, x, k] += C
        expect[rr, y, x, k + 1] += S
    np.testing.assert_allclose(iwe, expect, rtol=0, atol=1e-12)
