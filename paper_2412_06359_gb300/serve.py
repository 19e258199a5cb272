"""Python front end of the serving API (cm_server_* / cm_batch_submit / poll /
wait): host buffers for requests and a thin Server wrapper.  Marshalling only;
the scheduler, memory pool and kernels are in libcm.so."""
from __future__ import annotations

import dataclasses

import numpy as np

from . import _capi as C


@dataclasses.dataclass
class HostRequest:
    """One request's host buffers (kept alive until the request is done)."""
    stream_id: int
    window: object                 # synth.Window with inv_depth / ego
    x: np.ndarray
    y: np.ndarray
    t: np.ndarray
    p: np.ndarray
    rho: np.ndarray
    ego: np.ndarray
    loss: np.ndarray
    drho: np.ndarray
    dego: np.ndarray

    @staticmethod
    def from_window(stream_id: int, win) -> "HostRequest":
        ev = win.events
        H, W = win.inv_depth.shape
        return HostRequest(stream_id, win, np.ascontiguousarray(ev.x, np.int16), np.ascontiguousarray(ev.y, np.int16),
                           np.ascontiguousarray(ev.t, np.float32), np.ascontiguousarray(ev.p, np.int8),
                           np.ascontiguousarray(win.inv_depth, np.float32), np.ascontiguousarray(win.ego, np.float32),
                           np.zeros(1, np.float32), np.zeros((H, W), np.float32), np.zeros(6, np.float32))

    def c(self) -> C.cm_request:
        w = self.window
        cam = C.cm_camera(w.cam.width, w.cam.height, w.cam.fx, w.cam.fy, w.cam.cx, w.cam.cy)
        n = self.x.shape[0]
        ptr = (lambda a: a.ctypes.data if n else None)
        return C.cm_request(self.stream_id, cam, ptr(self.x), ptr(self.y), ptr(self.t), ptr(self.p), n,
                            float(w.events.t0), float(w.events.t1), self.rho.ctypes.data, self.ego.ctypes.data,
                            float(w.dt), self.loss.ctypes.data, self.drho.ctypes.data, self.dego.ctypes.data)


class Server:
    def __init__(self, hbm_budget: int, *, max_batch: int = 8, lanes: int = 2, max_queue: int = 4096,
                 nbins: int = 10, ref_mode: int = C.CM_REF_ALL_EDGES, eps: float = 1e-9, device: int = 0,
                 group_events: int = 0):
        cfg = C.cm_server_cfg(int(hbm_budget), max_batch, lanes, max_queue, nbins, ref_mode, eps, device,
                              int(group_events))
        self.handle = C.cm_server_create(cfg)
        self.live = {}

    def submit(self, req: HostRequest) -> int:
        t = C.cm_batch_submit(self.handle, req.c())
        self.live[t] = req
        return t

    def poll(self, ticket: int):
        r = C.cm_batch_poll(self.handle, ticket)
        if r is not None:
            self.live.pop(ticket, None)
        return r

    def wait(self, ticket: int, timeout_s: float = 60.0):
        r = C.cm_batch_wait(self.handle, ticket, timeout_s)
        self.live.pop(ticket, None)
        return r

    def stats(self) -> C.cm_server_stats:
        return C.cm_server_get_stats(self.handle)

    def close(self):
        if self.handle:
            C.cm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
