"""ctypes binding of libcm.so with the names of include/cm.h.

Argument marshalling only: every function takes plain integers for device
pointers and streams and returns what the C call returns (raising CMError on a
non-zero status).  Loading fails loudly when libcm.so is missing; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcm.so")

CM_OK, CM_EINVAL, CM_ENOMEM, CM_EBUSY, CM_ETIMEOUT, CM_ECUDA, CM_ENOTFOUND, CM_ESTATE = range(8)
CM_REF_END, CM_REF_ALL_EDGES = 0, 1
CM_SPLAT_AUTO, CM_SPLAT_ATOMIC, CM_SPLAT_SORT, CM_SPLAT_TILES = 0, 1, 2, 3
CM_MAX_BINS = 32
CM_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


class CMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib_or_none().cm_status_string(status).decode() if _lib_or_none() else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class cm_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class cm_events(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("t0", ctypes.c_float), ("t1", ctypes.c_float)]


class cm_loss_cfg(ctypes.Structure):
    _fields_ = [("nbins", ctypes.c_int32), ("ref_mode", ctypes.c_int32), ("splat", ctypes.c_int32),
                ("store_warps", ctypes.c_int32), ("eps", ctypes.c_float)]


class cm_window(ctypes.Structure):
    _fields_ = [("cam", cm_camera), ("ev", cm_events), ("flow", ctypes.c_void_p), ("inv_depth", ctypes.c_void_p),
                ("ego6", ctypes.c_void_p), ("dt_window", ctypes.c_float), ("dloss", ctypes.c_void_p),
                ("loss_out", ctypes.c_void_p), ("dflow", ctypes.c_void_p), ("dinv_depth", ctypes.c_void_p),
                ("dego6", ctypes.c_void_p), ("scratch", ctypes.c_void_p)]


class cm_batch_schedule(ctypes.Structure):
    _fields_ = [("chains", ctypes.c_int32), ("group", ctypes.c_int32), ("bin", ctypes.c_int32),
                ("persist", ctypes.c_int32)]


class cm_server_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("nbins", ctypes.c_int32), ("ref_mode", ctypes.c_int32),
                ("eps", ctypes.c_float), ("device", ctypes.c_int32), ("group_events", ctypes.c_int64)]


class cm_request(ctypes.Structure):
    _fields_ = [("stream_id", ctypes.c_int32), ("cam", cm_camera), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("p", ctypes.c_void_p), ("n", ctypes.c_int64), ("t0", ctypes.c_float),
                ("t1", ctypes.c_float), ("inv_depth", ctypes.c_void_p), ("ego6", ctypes.c_void_p),
                ("dt_window", ctypes.c_float), ("loss_out", ctypes.c_void_p), ("dinv_depth_out", ctypes.c_void_p),
                ("dego6_out", ctypes.c_void_p)]


class cm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class cm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64), ("evictions", ctypes.c_int64),
                ("memory_waits", ctypes.c_int64), ("queued", ctypes.c_int64), ("pool_bytes", ctypes.c_size_t),
                ("pool_used", ctypes.c_size_t), ("pool_peak", ctypes.c_size_t)]


class cm_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None

_vp, _i32, _i64, _f32, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
_P = ctypes.POINTER

# name -> (argtypes, restype); restype int means a status code
SIGNATURES = {
    "cm_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "cm_abi_version": ([], ctypes.c_int),
    "cm_workspace_query": ([_P(cm_camera), _P(cm_loss_cfg), _i64, _i32, _P(_sz)], ctypes.c_int),
    "cm_workspace_create": ([_vp, _sz, _P(cm_camera), _P(cm_loss_cfg), _i64, _i32, _P(_vp)], ctypes.c_int),
    "cm_workspace_destroy": ([_vp], ctypes.c_int),
    "cm_workspace_stats": ([_vp, _P(_vp), _P(_vp)], ctypes.c_int),
    "cm_flow_from_depth": ([_P(cm_camera), _vp, _vp, _f32, _vp, _vp], ctypes.c_int),
    "cm_warp_splat": ([_P(cm_camera), _P(cm_events), _vp, _i32, _P(cm_loss_cfg), _vp, _vp, _vp], ctypes.c_int),
    "cm_loss_forward": ([_P(cm_camera), _P(cm_events), _vp, _i32, _vp, _vp, _f32, _P(cm_loss_cfg), _vp, _vp, _vp],
                        ctypes.c_int),
    "cm_loss_backward": ([_P(cm_camera), _P(cm_events), _vp, _i32, _vp, _vp, _f32, _P(cm_loss_cfg), _vp, _vp,
                          _vp, _vp, _vp, _vp], ctypes.c_int),
    "cm_window_scratch_query": ([_P(cm_camera), _P(cm_loss_cfg), _P(_sz)], ctypes.c_int),
    "cm_batch_query": ([_P(cm_window), _i32, _P(cm_loss_cfg), _P(_sz)], ctypes.c_int),
    "cm_batch_create": ([_vp, _sz, _P(cm_window), _i32, _P(cm_loss_cfg), _P(_vp)], ctypes.c_int),
    "cm_batch_set_windows": ([_vp, _P(cm_window), _i32], ctypes.c_int),
    "cm_batch_run": ([_vp, _vp], ctypes.c_int),
    "cm_batch_status": ([_vp, _vp], ctypes.c_int),
    "cm_batch_inject_stall": ([_vp, _i32], ctypes.c_int),
    "cm_batch_set_schedule": ([_vp, _P(cm_batch_schedule)], ctypes.c_int),
    "cm_batch_get_schedule": ([_vp, _P(cm_batch_schedule)], ctypes.c_int),
    "cm_batch_autotune": ([_vp, _vp, _P(cm_batch_schedule)], ctypes.c_int),
    "cm_batch_stats": ([_vp, _i32, _P(_vp), _P(_vp)], ctypes.c_int),
    "cm_batch_destroy": ([_vp], ctypes.c_int),
    "cm_server_create": ([_P(cm_server_cfg), _P(_vp)], ctypes.c_int),
    "cm_batch_submit": ([_vp, _P(cm_request), _P(ctypes.c_uint64)], ctypes.c_int),
    "cm_batch_poll": ([_vp, ctypes.c_uint64, _P(cm_result), _P(_i32)], ctypes.c_int),
    "cm_batch_wait": ([_vp, ctypes.c_uint64, ctypes.c_double, _P(cm_result)], ctypes.c_int),
    "cm_server_get_stats": ([_vp, _P(cm_server_stats)], ctypes.c_int),
    "cm_server_destroy": ([_vp], ctypes.c_int),
    "cm_loss_grad_static": ([_P(cm_camera), _P(cm_events), _vp, _i32, _P(cm_loss_cfg), _vp, _vp, _vp, _vp],
                            ctypes.c_int),
    "cm_profile_enable": ([ctypes.c_int], ctypes.c_int),
    "cm_profile_collect": ([_P(cm_kernel_stat), _i32, _P(_i32)], ctypes.c_int),
    "cm_profile_reset": ([], ctypes.c_int),
    "cm_launch_count": ([], ctypes.c_int64),
    "cm_flow_eq2": ([_P(cm_camera), _vp, _vp, _i32, _f32, _f32, _vp, _vp], ctypes.c_int),
    "cm_event_frame": ([_P(cm_camera), _P(cm_events), _vp, _vp], ctypes.c_int),
    "cm_geo_scratch_query": ([_P(cm_camera), _P(_sz)], ctypes.c_int),
    "cm_geo_forward": ([_P(cm_camera), _vp, _vp, _vp, _f32, _vp, _sz, _vp, _vp], ctypes.c_int),
    "cm_geo_backward": ([_P(cm_camera), _vp, _vp, _vp, _f32, _vp, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "cm_rsat": ([_P(cm_camera), _P(cm_events), _vp, _i32, _P(cm_loss_cfg), _vp, _vp, _vp], ctypes.c_int),
    "cm_flow_eq2_scratch_query": ([_P(cm_camera), _i32, _P(_sz)], ctypes.c_int),
    "cm_flow_eq2_backward": ([_P(cm_camera), _vp, _vp, _i32, _f32, _f32, _vp, _vp, _vp, _vp, _sz, _vp],
                             ctypes.c_int),
    "cm_measure_l2_rates": ([_vp, _sz, _vp, _P(ctypes.c_double), _P(ctypes.c_double)], ctypes.c_int),
}


def _lib_or_none():
    return _lib


def lib():
    """Load libcm.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libcm.so is not built ({LIB_PATH}); run paper_2412_06359_gb300.build.build()")
        l = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(l, name)
            fn.argtypes = args
            fn.restype = res
        _lib = l
    return _lib


def _check(status: int, where: str):
    if status != CM_OK:
        raise CMError(status, where)


# ---------------------------------------------------------------------------
# the entry points (same names as include/cm.h)


def cm_status_string(status: int) -> str:
    return lib().cm_status_string(status).decode()


def cm_abi_version() -> int:
    return lib().cm_abi_version()


def cm_workspace_query(cam: cm_camera, cfg: cm_loss_cfg, max_events: int, n_flow_bins: int) -> int:
    out = _sz(0)
    _check(lib().cm_workspace_query(ctypes.byref(cam), ctypes.byref(cfg), max_events, n_flow_bins,
                                    ctypes.byref(out)), "cm_workspace_query")
    return out.value


def cm_workspace_create(dev_mem: int, nbytes: int, cam: cm_camera, cfg: cm_loss_cfg, max_events: int,
                        n_flow_bins: int) -> int:
    h = _vp(0)
    _check(lib().cm_workspace_create(dev_mem, nbytes, ctypes.byref(cam), ctypes.byref(cfg), max_events,
                                     n_flow_bins, ctypes.byref(h)), "cm_workspace_create")
    return h.value


def cm_workspace_destroy(ws: int) -> None:
    _check(lib().cm_workspace_destroy(ws), "cm_workspace_destroy")


def cm_workspace_stats(ws: int) -> tuple[int, int]:
    a, b = _vp(0), _vp(0)
    _check(lib().cm_workspace_stats(ws, ctypes.byref(a), ctypes.byref(b)), "cm_workspace_stats")
    return a.value, b.value


def cm_flow_from_depth(cam, inv_depth: int, ego6: int, dt_window: float, flow_out: int, stream: int) -> None:
    _check(lib().cm_flow_from_depth(ctypes.byref(cam), inv_depth, ego6, dt_window, flow_out, stream),
           "cm_flow_from_depth")


def cm_warp_splat(cam, ev, flow: int, n_flow_bins: int, cfg, ws: int | None, iwe_out: int | None, stream: int):
    _check(lib().cm_warp_splat(ctypes.byref(cam), ctypes.byref(ev), flow, n_flow_bins, ctypes.byref(cfg), ws,
                               iwe_out, stream), "cm_warp_splat")


def cm_loss_forward(cam, ev, flow, n_flow_bins, inv_depth, ego6, dt_window, cfg, ws, loss_out, stream):
    _check(lib().cm_loss_forward(ctypes.byref(cam), ctypes.byref(ev), flow, n_flow_bins, inv_depth, ego6,
                                 dt_window, ctypes.byref(cfg), ws, loss_out, stream), "cm_loss_forward")


def cm_loss_backward(cam, ev, flow, n_flow_bins, inv_depth, ego6, dt_window, cfg, ws, dloss, dflow, dinv_depth,
                     dego6, stream):
    _check(lib().cm_loss_backward(ctypes.byref(cam), ctypes.byref(ev), flow, n_flow_bins, inv_depth, ego6,
                                  dt_window, ctypes.byref(cfg), ws, dloss, dflow, dinv_depth, dego6, stream),
           "cm_loss_backward")


def _win_array(wins):
    arr = (cm_window * len(wins))(*wins)
    return arr


def cm_window_scratch_query(cam, cfg) -> int:
    out = _sz(0)
    _check(lib().cm_window_scratch_query(ctypes.byref(cam), ctypes.byref(cfg), ctypes.byref(out)),
           "cm_window_scratch_query")
    return out.value


def cm_batch_query(wins, cfg) -> int:
    out = _sz(0)
    _check(lib().cm_batch_query(_win_array(wins), len(wins), ctypes.byref(cfg), ctypes.byref(out)), "cm_batch_query")
    return out.value


def cm_batch_create(dev_mem: int, nbytes: int, wins, cfg) -> int:
    h = _vp(0)
    _check(lib().cm_batch_create(dev_mem, nbytes, _win_array(wins), len(wins), ctypes.byref(cfg), ctypes.byref(h)),
           "cm_batch_create")
    return h.value


def cm_batch_set_windows(plan: int, wins) -> None:
    _check(lib().cm_batch_set_windows(plan, _win_array(wins), len(wins)), "cm_batch_set_windows")


def cm_batch_run(plan: int, stream: int) -> None:
    _check(lib().cm_batch_run(plan, stream), "cm_batch_run")


def cm_batch_set_schedule(plan: int, chains: int, group: int, bin: int = 0, persist: int = 0) -> None:
    s = cm_batch_schedule(chains, group, bin, persist)
    _check(lib().cm_batch_set_schedule(plan, ctypes.byref(s)), "cm_batch_set_schedule")


def cm_batch_get_schedule(plan: int) -> tuple[int, int, int, int]:
    s = cm_batch_schedule()
    _check(lib().cm_batch_get_schedule(plan, ctypes.byref(s)), "cm_batch_get_schedule")
    return s.chains, s.group, s.bin, s.persist


def cm_batch_autotune(plan: int, stream: int) -> tuple[int, int, int, int]:
    s = cm_batch_schedule()
    _check(lib().cm_batch_autotune(plan, stream, ctypes.byref(s)), "cm_batch_autotune")
    return s.chains, s.group, s.bin, s.persist


def cm_batch_status(plan: int, stream: int) -> int:
    """CM_OK, or CM_ETIMEOUT when a bounded device wait of the last run gave up
    (other failures raise)."""
    st = lib().cm_batch_status(plan, stream)
    if st not in (CM_OK, CM_ETIMEOUT):
        _check(st, "cm_batch_status")
    return st


def cm_batch_inject_stall(plan: int, window: int) -> None:
    _check(lib().cm_batch_inject_stall(plan, window), "cm_batch_inject_stall")


def cm_batch_stats(plan: int, window: int) -> tuple[int, int]:
    a, b = _vp(0), _vp(0)
    _check(lib().cm_batch_stats(plan, window, ctypes.byref(a), ctypes.byref(b)), "cm_batch_stats")
    return a.value, b.value


def cm_batch_destroy(plan: int) -> None:
    _check(lib().cm_batch_destroy(plan), "cm_batch_destroy")


def cm_server_create(cfg: cm_server_cfg) -> int:
    h = _vp(0)
    _check(lib().cm_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cm_server_create")
    return h.value


def cm_batch_submit(server: int, req: cm_request) -> int:
    t = ctypes.c_uint64(0)
    _check(lib().cm_batch_submit(server, ctypes.byref(req), ctypes.byref(t)), "cm_batch_submit")
    return t.value


def cm_batch_poll(server: int, ticket: int):
    """None while the request runs, else its cm_result."""
    r = cm_result()
    done = _i32(0)
    _check(lib().cm_batch_poll(server, ticket, ctypes.byref(r), ctypes.byref(done)), "cm_batch_poll")
    return r if done.value else None


def cm_batch_wait(server: int, ticket: int, timeout_s: float) -> cm_result:
    r = cm_result()
    _check(lib().cm_batch_wait(server, ticket, float(timeout_s), ctypes.byref(r)), "cm_batch_wait")
    return r


def cm_server_get_stats(server: int) -> cm_server_stats:
    s = cm_server_stats()
    _check(lib().cm_server_get_stats(server, ctypes.byref(s)), "cm_server_get_stats")
    return s


def cm_server_destroy(server: int) -> None:
    _check(lib().cm_server_destroy(server), "cm_server_destroy")


def cm_loss_grad_static(cam, ev, flow: int, n_flow_bins: int, cfg, dloss: int, loss_out: int, dflow_out: int,
                        stream: int) -> None:
    """Loss and dL/dflow of one window with no workspace and no allocation
    (the library's fixed internal array; see include/cm.h for the limits)."""
    _check(lib().cm_loss_grad_static(ctypes.byref(cam), ctypes.byref(ev), flow, n_flow_bins, ctypes.byref(cfg),
                                     dloss, loss_out, dflow_out, stream), "cm_loss_grad_static")


def cm_profile_enable(on: bool) -> None:
    _check(lib().cm_profile_enable(1 if on else 0), "cm_profile_enable")


def cm_profile_collect() -> dict:
    """{kernel name: (launches, total milliseconds)} since the last reset."""
    n = _i32(0)
    _check(lib().cm_profile_collect(None, 0, ctypes.byref(n)), "cm_profile_collect")
    arr = (cm_kernel_stat * max(n.value, 1))()
    _check(lib().cm_profile_collect(arr, n.value, ctypes.byref(n)), "cm_profile_collect")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def cm_profile_reset() -> None:
    _check(lib().cm_profile_reset(), "cm_profile_reset")


def cm_launch_count() -> int:
    return int(lib().cm_launch_count())


def cm_measure_l2_rates(buf: int, nbytes: int, stream: int) -> tuple[float, float]:
    """(random reductions / s, random loads / s) measured over device memory `buf`."""
    red, ld = ctypes.c_double(), ctypes.c_double()
    _check(lib().cm_measure_l2_rates(buf, nbytes, stream, ctypes.byref(red), ctypes.byref(ld)),
           "cm_measure_l2_rates")
    return red.value, ld.value


def cm_flow_eq2(cam, inv_depth: int, ego6: int, nb: int, dt_bin: float, scale: float, flow_out: int,
                stream: int) -> None:
    _check(lib().cm_flow_eq2(ctypes.byref(cam), inv_depth, ego6, nb, dt_bin, scale, flow_out, stream), "cm_flow_eq2")


def cm_flow_eq2_scratch_query(cam, nb: int) -> int:
    n = _sz()
    _check(lib().cm_flow_eq2_scratch_query(ctypes.byref(cam), nb, ctypes.byref(n)), "cm_flow_eq2_scratch_query")
    return n.value


def cm_flow_eq2_backward(cam, inv_depth: int, ego6: int, nb: int, dt_bin: float, scale: float, dflow: int,
                         dinv_depth: int, dego6: int, scratch: int, scratch_bytes: int, stream: int) -> None:
    _check(lib().cm_flow_eq2_backward(ctypes.byref(cam), inv_depth, ego6, nb, dt_bin, scale, dflow, dinv_depth,
                                      dego6, scratch, scratch_bytes, stream), "cm_flow_eq2_backward")


def cm_event_frame(cam, ev, frame_out: int, stream: int) -> None:
    _check(lib().cm_event_frame(ctypes.byref(cam), ctypes.byref(ev), frame_out, stream), "cm_event_frame")


def cm_rsat(cam, ev, flow: int, n_flow_bins: int, cfg, ws: int, rsat_out: int, stream: int) -> None:
    _check(lib().cm_rsat(ctypes.byref(cam), ctypes.byref(ev), flow, n_flow_bins, ctypes.byref(cfg), ws, rsat_out,
                         stream), "cm_rsat")


def cm_geo_scratch_query(cam) -> int:
    n = _sz()
    _check(lib().cm_geo_scratch_query(ctypes.byref(cam), ctypes.byref(n)), "cm_geo_scratch_query")
    return n.value


def cm_geo_forward(cam, rho0: int, rho1: int, ego6: int, dt: float, scratch: int, scratch_bytes: int, loss_out: int,
                   stream: int) -> None:
    _check(lib().cm_geo_forward(ctypes.byref(cam), rho0, rho1, ego6, dt, scratch, scratch_bytes, loss_out, stream),
           "cm_geo_forward")


def cm_geo_backward(cam, rho0: int, rho1: int, ego6: int, dt: float, dloss: int, drho0: int, drho1: int, dego6: int,
                    scratch: int, scratch_bytes: int, stream: int) -> None:
    _check(lib().cm_geo_backward(ctypes.byref(cam), rho0, rho1, ego6, dt, dloss, drho0, drho1, dego6, scratch,
                                 scratch_bytes, stream), "cm_geo_backward")
