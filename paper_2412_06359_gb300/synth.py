"""Seeded synthetic event windows, inverse-depth maps, ego-motions and flows.

These stand in for the event-camera datasets the paper trains and evaluates on
(MVSEC, DSEC, UZH-FPV; supplementary Sec. "Implementation details"), which are
not available here.  Shapes follow the paper: 10 bins per window (supp.,
Training), 1k-100k events per bin (Sec. 3.3, supp. DSEC bin cap), the
346x260 DAVIS and 640x480 DVXplorer sensors (Sec. 3.5).

This module holds NO arithmetic of the method (no warp, splat, loss or flow
construction): it only draws inputs.  Both the CUDA path and the CPU oracle
take their inputs from here, so it is the one module the two share.

Seeds: numpy PCG64.  Workload c uses base seed 1000 + c; window i of a
multi-window workload uses (1000 + c) * 1000 + i.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

try:  # scipy is present here and on the GPU hosts; the blur is a plain convolution otherwise
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover
    _gaussian_filter = None

WINDOW_S = 0.01  # 10 ms windows (supp., DSEC / UZH-FPV bins)


@dataclasses.dataclass
class Camera:
    """Pinhole intrinsics of an undistorted, rectified sensor."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


@dataclasses.dataclass
class Events:
    """One window of events in structure-of-arrays form, timestamps ascending.

    x, y: int16 pixel column / row; t: float32 seconds; p: int8 polarity (+1/-1);
    the window is [t0, t1] (float32 values).
    """
    x: np.ndarray
    y: np.ndarray
    t: np.ndarray
    p: np.ndarray
    t0: float
    t1: float

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def take(self, idx) -> "Events":
        return Events(self.x[idx], self.y[idx], self.t[idx], self.p[idx], self.t0, self.t1)


@dataclasses.dataclass
class Window:
    """One evaluation: events plus either a flow field or (inverse depth, ego-motion)."""
    cam: Camera
    events: Events
    nbins: int
    ref_mode: int            # 0: window end only; 1: all bin edges
    flow: np.ndarray | None = None       # [nfb, H, W, 2] float32, px per window
    inv_depth: np.ndarray | None = None  # [H, W] float32, 1/m
    ego: np.ndarray | None = None        # [6] float32: (vx, vy, vz, wx, wy, wz)
    dt: float = WINDOW_S


REF_END = 0
REF_ALL = 1


def camera_for(width: int, height: int) -> Camera:
    """Intrinsics used for each sensor size.

    346x260: fx = fy = 226, principal point (173, 130).  640x480: fx = fy = 450.
    1280x720: fx = fy = 900.  The principal point is the image centre, and for
    other sizes the focal length is 0.7 * width (the ratio of the other sensors).
    """
    if (width, height) == (346, 260):
        return Camera(346, 260, 226.0, 226.0, 173.0, 130.0)
    if (width, height) == (640, 480):
        return Camera(640, 480, 450.0, 450.0, 320.0, 240.0)
    if (width, height) == (1280, 720):
        return Camera(1280, 720, 900.0, 900.0, 640.0, 360.0)
    f = float(round(0.7 * width))
    return Camera(width, height, f, f, width / 2.0, height / 2.0)


def rng_for(workload: int, window: int | None = None) -> np.random.Generator:
    base = 1000 + workload
    seed = base if window is None else base * 1000 + window
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# events


def _timestamps(rng: np.random.Generator, n: int, t0: float, t1: float) -> np.ndarray:
    t = np.sort(rng.uniform(t0, t1, size=n)).astype(np.float32)
    return np.clip(t, np.float32(t0), np.float32(t1))


def _polarity(rng: np.random.Generator, n: int) -> np.ndarray:
    return np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)


def uniform_events(rng: np.random.Generator, width: int, height: int, n: int,
                   t0: float = 0.0, t1: float = WINDOW_S) -> Events:
    """x, y uniform integer pixels; t uniform in [t0, t1], sorted; p = +-1 with p = 0.5."""
    x = rng.integers(0, width, size=n).astype(np.int16)
    y = rng.integers(0, height, size=n).astype(np.int16)
    return Events(x, y, _timestamps(rng, n, t0, t1), _polarity(rng, n), float(np.float32(t0)), float(np.float32(t1)))


def _blur(img: np.ndarray, sigma: float) -> np.ndarray:
    if _gaussian_filter is not None:
        return _gaussian_filter(img, sigma, mode="reflect")
    r = int(3 * sigma) + 1
    k = np.exp(-0.5 * (np.arange(-r, r + 1) / sigma) ** 2)
    k /= k.sum()
    out = np.apply_along_axis(lambda v: np.convolve(np.pad(v, r, mode="reflect"), k, "valid"), 0, img)
    return np.apply_along_axis(lambda v: np.convolve(np.pad(v, r, mode="reflect"), k, "valid"), 1, out)


def texture(rng: np.random.Generator, width: int, height: int) -> np.ndarray:
    """Sum of 4 octaves of Gaussian-blurred white noise (sigma 16, 8, 4, 2 px)."""
    img = np.zeros((height, width), np.float64)
    for octave, sigma in enumerate((16.0, 8.0, 4.0, 2.0)):
        img += (0.5 ** octave) * _blur(rng.standard_normal((height, width)), sigma) * sigma
    return img


def gradient_events(rng: np.random.Generator, width: int, height: int, n: int,
                    t0: float = 0.0, t1: float = WINDOW_S) -> Events:
    """Events at integer pixels drawn with probability proportional to the
    image-gradient magnitude of a random texture (edges fire events);
    t uniform in [t0, t1], sorted; p = +-1 with p = 0.5."""
    img = texture(rng, width, height)
    gy, gx = np.gradient(img)
    mag = np.hypot(gx, gy).ravel()
    prob = mag / mag.sum()
    flat = rng.choice(width * height, size=n, p=prob)
    x = (flat % width).astype(np.int16)
    y = (flat // width).astype(np.int16)
    return Events(x, y, _timestamps(rng, n, t0, t1), _polarity(rng, n), float(np.float32(t0)), float(np.float32(t1)))


# --------------------------------------------------------------------------
# flow, inverse depth, ego-motion


def sinusoid_flow(rng: np.random.Generator, width: int, height: int, max_mag: float = 5.0) -> np.ndarray:
    """Sum of 3 low-frequency sinusoids, rescaled so that max |flow| = max_mag
    px per window.  Returns [H, W, 2] float32."""
    yy, xx = np.meshgrid(np.arange(height) / height, np.arange(width) / width, indexing="ij")
    f = np.zeros((height, width, 2))
    for _ in range(3):
        kx, ky = rng.integers(1, 4, size=2)
        amp = rng.uniform(0.5, 1.0)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        arg = 2 * np.pi * (kx * xx + ky * yy)
        f[..., 0] += amp * np.sin(arg + ph[0])
        f[..., 1] += amp * np.cos(arg + ph[1])
    mag = np.sqrt((f ** 2).sum(-1)).max()
    return (f * (max_mag / mag)).astype(np.float32)


def inv_depth_map(rng: np.random.Generator, width: int, height: int,
                  lo: float = 0.2, hi: float = 2.0) -> np.ndarray:
    """Piecewise-smooth inverse depth in [lo, hi] 1/m: a Voronoi partition over
    6 random seeds, each cell a random plane, plus 5 Gaussian bumps (sigma
    10-40 px), clipped.  Returns [H, W] float32."""
    yy, xx = np.meshgrid(np.arange(height, dtype=np.float64), np.arange(width, dtype=np.float64), indexing="ij")
    seeds = np.stack([rng.uniform(0, width, 6), rng.uniform(0, height, 6)], 1)
    d2 = (xx[None] - seeds[:, 0, None, None]) ** 2 + (yy[None] - seeds[:, 1, None, None]) ** 2
    label = np.argmin(d2, axis=0)
    rho = np.zeros((height, width))
    for i in range(6):
        base = rng.uniform(lo + 0.1, hi - 0.3)
        gx, gy = rng.uniform(-0.5, 0.5, size=2)
        plane = base + gx * (xx / width - 0.5) + gy * (yy / height - 0.5)
        rho = np.where(label == i, plane, rho)
    for _ in range(5):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        sig = rng.uniform(10, 40)
        amp = rng.uniform(-0.4, 0.6)
        rho += amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * sig * sig))
    return np.clip(rho, lo, hi).astype(np.float32)


def ego_motion(rng: np.random.Generator) -> np.ndarray:
    """Linear velocity ~ N(0, 1) m/s and angular velocity ~ N(0, 1) rad/s,
    camera frame.  Returns float32 (vx, vy, vz, wx, wy, wz)."""
    return rng.standard_normal(6).astype(np.float32)


# --------------------------------------------------------------------------
# the workloads


def log_uniform_count(rng: np.random.Generator, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def flow_window(n: int = 20_000, size=(128, 128), seed_workload: int = 1) -> Window:
    """Flow-input workload: sensor 128x128, 20,000 uniform events over 10 ms,
    a given sinusoid flow (|flow| <= 5 px per window), one bin, one
    reference time at the window end."""
    rng = rng_for(seed_workload)
    w, h = size
    ev = uniform_events(rng, w, h, n)
    flow = sinusoid_flow(rng, w, h)[None]
    cam = Camera(w, h, 0.7 * w, 0.7 * w, w / 2, h / 2)
    return Window(cam, ev, nbins=1, ref_mode=REF_END, flow=flow)


def depth_window(rng: np.random.Generator, width: int, height: int, n: int, nbins: int = 10,
                 ref_mode: int = REF_ALL) -> Window:
    """Depth + ego-motion workload: events drawn on texture edges, a
    piecewise-smooth inverse depth and a random ego-motion, 10 ms window."""
    cam = camera_for(width, height)
    ev = gradient_events(rng, width, height, n)
    rho = inv_depth_map(rng, width, height)
    ego = ego_motion(rng)
    return Window(cam, ev, nbins=nbins, ref_mode=ref_mode, inv_depth=rho, ego=ego)


def motion_window(rng: np.random.Generator, width: int, height: int, n: int, nbins: int = 10,
                  per_point: int = 50, max_mag: float = 8.0) -> Window:
    """Motion-consistent events (the contention stress case): n / per_point
    scene points at random sub-pixel positions, each with one polarity, fire
    events at uniform times as they move along a given smooth flow (a
    sinusoid field, px per window); each event is the point's position at its
    time, rounded to a pixel.  With that flow as the window's flow every
    point's events gather in a small spot at each reference: the sharp images
    of a converged estimate, with many events per pixel."""
    flow = sinusoid_flow(rng, width, height, max_mag)
    npts = max(1, n // per_point)
    px = rng.uniform(0, width - 1, npts)
    py = rng.uniform(0, height - 1, npts)
    pol = np.where(rng.random(npts) < 0.5, 1, -1).astype(np.int8)
    k = rng.integers(0, npts, size=n)
    t = _timestamps(rng, n, 0.0, WINDOW_S)
    tau = (t.astype(np.float64) - 0.0) / WINDOW_S
    ix, iy = np.rint(px[k]).astype(np.int64), np.rint(py[k]).astype(np.int64)
    u = flow[iy, ix].astype(np.float64)
    x = np.clip(np.rint(px[k] + tau * u[:, 0]), 0, width - 1).astype(np.int16)
    y = np.clip(np.rint(py[k] + tau * u[:, 1]), 0, height - 1).astype(np.int16)
    ev = Events(x, y, t, pol[k], 0.0, float(np.float32(WINDOW_S)))
    return Window(camera_for(width, height), ev, nbins=nbins, ref_mode=REF_ALL, flow=flow[None])


def batch_windows_motion(count: int = 64, width: int = 640, height: int = 480, lo: float = 5e3, hi: float = 5e5,
                         first: int = 0) -> list[Window]:
    """The uneven batch with motion-consistent events (flow input, the true
    flow): the contention stress variant of batch_windows."""
    out = []
    for i in range(first, first + count):
        rng = rng_for(6, i)
        n = log_uniform_count(rng, lo, hi)
        out.append(motion_window(rng, width, height, n))
    return out


def davis_window(n: int = 100_000) -> Window:
    """346x260 DAVIS sensor, 100,000 events, 10 bins, all 11 bin edges as references."""
    return depth_window(rng_for(2), 346, 260, n)


def batch_windows(count: int = 64, width: int = 640, height: int = 480,
                  lo: float = 5e3, hi: float = 5e5, first: int = 0) -> list[Window]:
    """Uneven batch: `count` 640x480 windows with log-uniform event counts in
    [5k, 500k], each with its own depth map and ego-motion, 10 bins.  Windows
    first .. first+count-1 of the seeded sequence."""
    out = []
    for i in range(first, first + count):
        rng = rng_for(3, i)
        n = log_uniform_count(rng, lo, hi)
        out.append(depth_window(rng, width, height, n))
    return out


def hd_window(n: int = 2_000_000, nbins: int = 20) -> Window:
    """1280x720 sensor, 2,000,000 events, 20 bins, all 21 edges as references."""
    return depth_window(rng_for(4), 1280, 720, n, nbins=nbins)


SERVE_RESOLUTIONS = ((346, 260), (640, 480), (1280, 720))


@dataclasses.dataclass
class Arrival:
    stream: int
    t_arrival: float
    window: Window


def serving_trace(streams: int = 32, rate_hz: float = 100.0, duration_s: float = 2.0,
                  lo: float = 1e4, hi: float = 2e6, nbins: int = 10, seed_workload: int = 5,
                  max_requests: int | None = None) -> list[Arrival]:
    """Poisson arrivals (exponential gaps, mean 1/rate) on `streams` streams
    whose resolutions cycle through 346x260 / 640x480 / 1280x720; every request
    carries its own events (log-uniform count in [lo, hi]), depth and ego-motion."""
    arrivals = []
    for s in range(streams):
        rng = rng_for(seed_workload, s)
        w, h = SERVE_RESOLUTIONS[s % len(SERVE_RESOLUTIONS)]
        t = rng.exponential(1.0 / rate_hz)
        while t < duration_s:
            n = log_uniform_count(rng, lo, hi)
            arrivals.append((t, s, depth_window(rng, w, h, n, nbins=nbins)))
            t += rng.exponential(1.0 / rate_hz)
    arrivals.sort(key=lambda a: (a[0], a[1]))
    if max_requests is not None:
        arrivals = arrivals[:max_requests]
    return [Arrival(s, t, win) for t, s, win in arrivals]
