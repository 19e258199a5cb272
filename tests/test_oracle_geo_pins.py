"""Pins of the oracle's geometry-consistency loss (Eq. 3): closed forms for a
camera at rest (equal and uniformly scaled depth), for forward motion over a
fronto-parallel plane (consistent depths give zero loss; the valid count from
the closed-form projection), for a pan over a plane, central differences of
the loss on frozen decisions for every inverse-depth pixel of both views and
every pose component, and the straddle analysis (flags, the interval of the
valid count and of the loss) against perturbed evaluations."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth


def _cam(W=23, H=17, f=19.0):
    return synth.Camera(W, H, f, f * 1.05, W / 2 - 0.4, H / 2 + 0.3)


def test_camera_at_rest():
    cam = _cam()
    rho = np.random.default_rng(1).uniform(0.3, 2.0, (cam.height, cam.width))
    r = O.geo(cam, rho, rho, np.zeros(6), 0.01)
    assert r["loss"] < 1e-14 and r["count"] == cam.width * cam.height  # x' = x up to FP64 rounding
    for c in (0.5, 1.7):
        r = O.geo(cam, rho, c * rho, np.zeros(6), 0.01)
        assert r["loss"] == pytest.approx(abs(c - 1) / (c + 1), rel=1e-12)


def test_forward_motion_over_a_plane():
    cam = _cam()
    Z0, vz, dt = 2.0, 3.0, 0.05
    rho0 = np.full((cam.height, cam.width), 1 / Z0)
    rho1 = np.full_like(rho0, 1 / (Z0 - vz * dt))  # the plane's depth after the motion
    r = O.geo(cam, rho0, rho1, np.array([0, 0, vz, 0, 0, 0]), dt)
    assert r["loss"] < 1e-14
    s = Z0 / (Z0 - vz * dt)  # points move away from the principal point by s
    v, u = np.mgrid[0:cam.height, 0:cam.width]
    xp, yp = cam.cx + (u - cam.cx) * s, cam.cy + (v - cam.cy) * s
    inside = (xp >= 0) & (xp <= cam.width - 1) & (yp >= 0) & (yp <= cam.height - 1)
    assert r["count"] == int(inside.sum())


def test_pan_over_a_plane():
    cam = _cam()
    Z0, wy, dt = 1.5, 0.9, 0.1
    rho = np.full((cam.height, cam.width), 1 / Z0)
    ego = np.array([0, 0, 0, 0, wy, 0])
    r = O.geo(cam, rho, rho, ego, dt)
    th = -wy * dt
    v, u = np.mgrid[0:cam.height, 0:cam.width]
    xn = (u - cam.cx) / cam.fx
    a = Z0 * (-np.sin(th) * xn + np.cos(th))  # depth of the rotated point; view 1 sees the plane at Z0
    f = np.abs(a - Z0) / (a + Z0)
    # the projection of the rotated plane point, in closed form
    xp = cam.fx * (np.cos(th) * xn + np.sin(th)) / (-np.sin(th) * xn + np.cos(th)) + cam.cx
    yp = cam.fy * ((v - cam.cy) / cam.fy) / (-np.sin(th) * xn + np.cos(th)) + cam.cy
    ok = (xp >= 0) & (xp <= cam.width - 1) & (yp >= 0) & (yp <= cam.height - 1) & (a > 0)
    assert r["count"] == int(ok.sum()) > 0
    assert r["loss"] == pytest.approx(f[ok].mean(), rel=1e-12)


def _loss(cam, r0, r1, e, dt, dec):
    return O.geo(cam, r0, r1, e, dt, replay=dec)["loss"]


def test_gradient_matches_central_differences_on_frozen_decisions():
    cam = _cam(13, 9, 11.0)
    rng = np.random.default_rng(5)
    r0 = rng.uniform(0.5, 1.5, (cam.height, cam.width))
    r1 = r0 * rng.uniform(0.8, 1.2, r0.shape)
    e = np.array([0.3, -0.2, 0.8, 0.4, -0.6, 0.2])
    dt = 0.05
    base = O.geo(cam, r0, r1, e, dt, record=True)
    dec = base["decisions"]
    assert 0 < dec["ok"].sum() < r0.size  # some pixels leave the image
    g = O.geo(cam, r0, r1, e, dt, replay=dec, grad=True, dloss=1.7)
    assert g["loss"] == pytest.approx(base["loss"], rel=1e-14)
    for name, x in (("dinv_depth0", r0), ("dinv_depth1", r1)):
        fd = np.empty_like(x)
        for q in range(x.size):
            h = 1e-6 * x.flat[q]
            xp, xm = x.copy(), x.copy()
            xp.flat[q] += h
            xm.flat[q] -= h
            args_p = (xp, r1) if name == "dinv_depth0" else (r0, xp)
            args_m = (xm, r1) if name == "dinv_depth0" else (r0, xm)
            fd.flat[q] = 1.7 * (_loss(cam, *args_p, e, dt, dec) - _loss(cam, *args_m, e, dt, dec)) / (2 * h)
        np.testing.assert_allclose(g[name], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    fde = np.empty(6)
    for q in range(6):
        h = 1e-6
        ep, em = e.copy(), e.copy()
        ep[q] += h
        em[q] -= h
        fde[q] = 1.7 * (_loss(cam, r0, r1, ep, dt, dec) - _loss(cam, r0, r1, em, dt, dec)) / (2 * h)
    np.testing.assert_allclose(g["dego"], fde, rtol=1e-5, atol=1e-6 * np.abs(fde).max())


def test_bounds_contain_the_loss_and_every_perturbed_evaluation():
    # a sideways translation over a fronto-parallel plane moves every pixel by
    # exactly -3 px, so every projection lies on an integer and column 3 lands
    # on the border x' = 0: every pixel is flagged (cell), column 3 also in the
    # valid set.  Inverse depths perturbed by 1e-7 relative (x' moves by 3e-7 px,
    # inside the margins) move column 3 in and out of the image: every
    # perturbed count and loss lies in the interval
    cam = _cam(40, 30, 30.0)
    dt, rho0 = 0.05, 0.8
    vx = 3.0 / (cam.fx * dt * rho0)
    e = np.array([vx, 0, 0, 0, 0, 0])
    r0 = np.full((cam.height, cam.width), rho0)
    r1 = r0 * np.random.default_rng(11).uniform(0.9, 1.1, r0.shape)
    base = O.geo(cam, r0, r1, e, dt)
    b = O.geo_bounds(cam, r0, r1, e, dt, safety=100.0)
    f = b["flags"]
    # every cell in doubt along x (y' = v is exact: no rows in doubt), column 3
    # also valid or not; columns 0-2 land beyond the margin: invalid in any evaluation
    assert np.all(f[:, 3:] & 1) and np.all(f[:, 3] & 2) and not np.any(f[:, 4:] & 2)
    assert not np.any(f[:, :3])
    assert b["count_hi"] - b["count_lo"] == cam.height
    assert b["count_lo"] <= base["count"] <= b["count_hi"]
    assert b["loss_lo"] <= base["loss"] <= b["loss_hi"]
    counts = set()
    for s in range(8):
        g = np.random.default_rng(50 + s)
        p0 = r0 * (1 + 1e-7 * g.uniform(-1, 1, r0.shape))
        pr = O.geo(cam, p0, r1, e, dt)
        assert b["count_lo"] <= pr["count"] <= b["count_hi"]
        assert b["loss_lo"] <= pr["loss"] <= b["loss_hi"]
        counts.add(pr["count"])
    assert len(counts) > 1  # the perturbations did move pixels across the border
