"""Pins of the oracle's event frame (the network input) and of the RSAT metric
(ratio of squared average timestamps): an independent per-pixel count, hand
examples worked out from Eq. 1, and the ratio's fixed points."""
import numpy as np

from oracle import oracle as O
from paper_2412_06359_gb300 import synth


def _ev(xs, ys, ts, ps):
    return synth.Events(np.array(xs, np.int16), np.array(ys, np.int16), np.array(ts, np.float32),
                        np.array(ps, np.int8), 0.0, 1.0)


def test_event_frame_counts_each_polarity():
    rng = np.random.default_rng(3)
    W, H = 31, 17
    e = synth.uniform_events(rng, W, H, 4000)
    f = O.event_frame(e, W, H)
    pos, neg = e.p > 0, e.p <= 0
    for ch, sel in ((0, pos), (1, neg)):
        ref = np.zeros(H * W)
        np.add.at(ref, e.y[sel].astype(np.int64) * W + e.x[sel], 1.0)
        assert np.array_equal(f[ch].ravel(), ref)
    assert f.sum() == e.n


def test_event_frame_skips_events_outside_the_sensor():
    e = _ev([0, 5, -1, 7, 3], [0, 2, 1, 0, 9], [0.1, 0.2, 0.3, 0.4, 0.5], [1, -1, 1, 1, -1])
    f = O.event_frame(e, 6, 4)  # x = 7 and y = 9 fall outside
    assert f.sum() == 2 and f[0, 0, 0] == 1 and f[1, 2, 5] == 1


def test_rsat_of_zero_flow_is_one():
    rng = np.random.default_rng(4)
    e = synth.uniform_events(rng, 20, 15, 500)
    assert O.rsat(e, np.zeros((15, 20, 2)), width=20, height=15, nbins=4, ref_mode=O.REF_ALL) == 1.0


def test_rsat_hand_example_two_events_aligned_by_the_flow():
    # A at (2, 3), tau = 0 and B at (3, 3), tau = 1; flow (1, 0) px per window,
    # one bin, reference at the window end.  t-bar: A 0, B 1.
    # zero flow: two pixels, T = 0 and T = 1, L = (0 + 1) / 2 = 0.5
    # with the flow A lands on B's pixel: C = 2, S = 1, T = 0.5, L = 0.25 / 1
    # RSAT = 0.25 / 0.5 = 0.5
    e = _ev([2, 3], [3, 3], [0.0, 1.0], [1, 1])
    flow = np.zeros((8, 8, 2))
    flow[..., 0] = 1.0
    r = O.rsat(e, flow, width=8, height=8, nbins=1, ref_mode=O.REF_END)
    assert abs(r - 0.5) < 1e-8


def test_rsat_of_one_isolated_event_is_one():
    # any in-image flow spreads one event over its bilinear corners, each with
    # T = t-bar as eps -> 0 (T = t-bar w / (w + eps) at a corner of weight w),
    # so L_r = t-bar^2 with or without the flow
    e = _ev([4], [4], [0.3], [-1])
    flow = np.zeros((10, 10, 2))
    flow[..., 0], flow[..., 1] = 0.37, -0.61
    r = O.rsat(e, flow, width=10, height=10, nbins=3, ref_mode=O.REF_ALL, eps=1e-15)
    assert abs(r - 1.0) < 1e-8
    # at the default eps the smallest corner weight (~0.0008 here) shows up
    assert abs(O.rsat(e, flow, width=10, height=10, nbins=3, ref_mode=O.REF_ALL) - 1.0) < 1e-5
