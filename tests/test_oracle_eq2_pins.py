"""Pins of the oracle's discrete flow (Eq. 2 with one pose per bin) and of its
adjoint through the projection, the rigid transform and Rodrigues' formula:
closed forms for pure translation and pure rotations written out here,
consistency with the single-pose form, the FP32 operation sequence within FP32
error of FP64, and central finite differences of the FP64 flow for every
inverse-depth pixel and every pose component (including a near-zero and a
large rotation angle)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2412_06359_gb300 import synth


def _cam(W=23, H=17, f=19.0):
    return synth.Camera(W, H, f, f * 1.1, W / 2 - 0.3, H / 2 + 0.2)


def _pix(cam):
    v, u = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
    return u, v, (u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy


def test_one_bin_unit_scale_is_the_single_pose_form():
    cam = synth.camera_for(64, 48)
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.3, 2.0, (48, 64))
    ego = np.array([0.4, -0.2, 0.9, 0.3, -0.5, 0.2])
    a = O.flow_eq2_bins(cam, rho, ego[None], 0.01, 1.0)[0]
    b = O.flow_eq2(cam, rho, ego, 0.01)
    assert np.array_equal(a, b)
    c = O.flow_eq2_bins(cam, rho, np.stack([ego, 2 * ego]), 0.01, 3.0)
    np.testing.assert_allclose(c[0], 3.0 * b, rtol=1e-15, atol=1e-15)


def test_pure_translation_closed_form():
    cam = _cam()
    u, v, xn, yn = _pix(cam)
    rho = np.random.default_rng(4).uniform(0.5, 1.5, u.shape)
    vel, dt = np.array([0.3, -0.2, 0.5]), 0.02
    Z = 1.0 / rho
    # the point moves by -v dt in the camera frame
    X, Y, Zp = Z * xn - vel[0] * dt, Z * yn - vel[1] * dt, Z - vel[2] * dt
    fx = cam.fx * X / Zp + cam.cx - u
    fy = cam.fy * Y / Zp + cam.cy - v
    f = O.flow_eq2_bins(cam, rho, np.r_[vel, 0, 0, 0][None], dt, 1.0)[0]
    np.testing.assert_allclose(f[..., 0], fx, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(f[..., 1], fy, rtol=1e-12, atol=1e-12)


def test_roll_rotates_about_the_principal_point():
    cam = synth.Camera(21, 15, 17.0, 17.0, 10.0, 7.0)
    u, v, xn, yn = _pix(cam)
    rho = np.random.default_rng(5).uniform(0.2, 2.0, u.shape)  # depth plays no part
    wz, dt = 0.8, 0.05
    ang = -wz * dt
    xr = np.cos(ang) * (u - cam.cx) - np.sin(ang) * (v - cam.cy)
    yr = np.sin(ang) * (u - cam.cx) + np.cos(ang) * (v - cam.cy)
    f = O.flow_eq2_bins(cam, rho, np.array([[0, 0, 0, 0, 0, wz]]), dt, 1.0)[0]
    np.testing.assert_allclose(f[..., 0], xr - (u - cam.cx), atol=1e-12)
    np.testing.assert_allclose(f[..., 1], yr - (v - cam.cy), atol=1e-12)


def test_pan_closed_form():
    cam = _cam()
    u, v, xn, yn = _pix(cam)
    rho = np.random.default_rng(6).uniform(0.2, 2.0, u.shape)
    wy, dt = -1.3, 0.1
    th = -wy * dt  # rotation about the camera's y axis by th
    c, s = np.cos(th), np.sin(th)
    X, Y, Z = xn, yn, np.ones_like(xn)  # depth cancels for a pure rotation
    Xp, Yp, Zp = c * X + s * Z, Y, -s * X + c * Z
    f = O.flow_eq2_bins(cam, rho, np.array([[0, 0, 0, 0, wy, 0]]), dt, 1.0)[0]
    np.testing.assert_allclose(f[..., 0], cam.fx * Xp / Zp + cam.cx - u, atol=1e-11)
    np.testing.assert_allclose(f[..., 1], cam.fy * Yp / Zp + cam.cy - v, atol=1e-11)


def _eq2_float32(cam, rho, e, dt, scale):
    """Eq. 2 displacement in numpy float32 arithmetic, written in the
    cancellation-free form (Z s0 + t0 - xn t2) / P2 with s0 = ((R - I) m)_0 -
    xn ((R - I) m)_2, m = (xn, yn, 1), and the rotation's coefficients in the
    stable forms sin(th)/th and 2 sin^2(th/2)/th^2."""
    f = np.float32
    k = (-e[3:] * f(dt)).astype(np.float32)
    t = (-e[:3] * f(dt)).astype(np.float32)
    th = np.sqrt((k * k).sum(dtype=np.float32))
    a = np.sin(th) / th if th > 0 else f(1)
    b = f(2) * np.sin(th / f(2)) ** 2 / (th * th) if th > 0 else f(0.5)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]], np.float32)
    A = (a * K + b * (K @ K)).astype(np.float32)  # R - I
    v, u = np.mgrid[0:cam.height, 0:cam.width].astype(np.float32)
    xn, yn = (u - f(cam.cx)) / f(cam.fx), (v - f(cam.cy)) / f(cam.fy)
    Z = f(1) / rho.astype(np.float32)
    Am = [A[i, 0] * xn + A[i, 1] * yn + A[i, 2] for i in range(3)]
    P2 = Z * (f(1) + Am[2]) + t[2]
    e0 = Z * (Am[0] - xn * Am[2]) + (t[0] - xn * t[2])
    e1 = Z * (Am[1] - yn * Am[2]) + (t[1] - yn * t[2])
    return np.stack([f(scale) * (f(cam.fx) * (e0 / P2)), f(scale) * (f(cam.fy) * (e1 / P2))], -1)


def test_error_bound_covers_a_single_precision_evaluation():
    cam = synth.camera_for(346, 260)
    rng = synth.rng_for(2)
    rho = synth.inv_depth_map(rng, 346, 260)
    ego = np.stack([synth.ego_motion(rng) for _ in range(4)])
    ego[3, 3:] *= 40.0  # a large rotation angle (about 0.5 rad over the bin)
    scale = 4.0
    f64 = O.flow_eq2_bins(cam, rho, ego, 0.01, scale)
    eb = O.flow_eq2_error_bound(cam, rho, ego, 0.01, scale)
    for i in range(4):
        f32 = _eq2_float32(cam, rho, ego[i].astype(np.float32), 0.01, scale)
        d = np.abs(f32.astype(np.float64) - f64[i]).max(axis=-1)
        assert np.all(d <= eb[i]), (i, (d / eb[i]).max())
        assert eb[i].max() < 1e-5 * np.abs(f64[i]).max() + 1e-5  # FP32-tight


def _loss(cam, rho, ego, dt, scale, g):
    return float((O.flow_eq2_bins(cam, rho, ego, dt, scale) * g).sum())


@pytest.mark.parametrize("angles", ["moderate", "tiny_and_large"])
def test_adjoint_matches_central_differences(angles):
    cam = _cam(13, 9)
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.3, 1.8, (cam.height, cam.width))
    ego = rng.normal(size=(3, 6))
    if angles == "tiny_and_large":
        ego[0, 3:] = [1e-6, -2e-6, 1.5e-6]  # th ~ 1e-8 over the bin: the series branch
        ego[2, 3:] *= 60.0                    # th ~ 1 rad
    dt, scale = 0.01, 3.0
    g = rng.normal(size=(3, cam.height, cam.width, 2))
    drho, dego = O.flow_eq2_grad(cam, rho, ego, dt, scale, g)
    # every inverse-depth pixel
    fd = np.empty_like(rho)
    for q in range(rho.size):
        h = 1e-6 * rho.flat[q]
        rp, rm = rho.copy(), rho.copy()
        rp.flat[q] += h
        rm.flat[q] -= h
        fd.flat[q] = (_loss(cam, rp, ego, dt, scale, g) - _loss(cam, rm, ego, dt, scale, g)) / (2 * h)
    np.testing.assert_allclose(drho, fd, rtol=2e-6, atol=1e-6 * np.abs(fd).max())
    # every pose component of every bin
    fde = np.empty_like(ego)
    for q in range(ego.size):
        h = 1e-6 * max(1.0, abs(ego.flat[q]))
        ep, em = ego.copy(), ego.copy()
        ep.flat[q] += h
        em.flat[q] -= h
        fde.flat[q] = (_loss(cam, rho, ep, dt, scale, g) - _loss(cam, rho, em, dt, scale, g)) / (2 * h)
    np.testing.assert_allclose(dego, fde, rtol=2e-6, atol=1e-6 * np.abs(fde).max())
