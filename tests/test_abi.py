"""The C ABI: libcm.so builds for sm_103a, loads, exports every function that
include/cm.h declares, and validates arguments on the host (no GPU needed:
every call here fails validation or only computes sizes, before any CUDA call)."""
import ctypes
import os
import re

import pytest

from paper_2412_06359_gb300 import _capi as C
from paper_2412_06359_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(cm_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported by libcm.so"
    # and the binding covers them under the same names
    for n in names:
        assert hasattr(C, n) or n in C.SIGNATURES, n


def test_status_strings(lib):
    assert C.cm_status_string(0) == "ok"
    assert "invalid" in C.cm_status_string(C.CM_EINVAL)
    assert C.cm_abi_version() == 1


def cam(w=346, h=260):
    return C.cm_camera(w, h, 226.0, 226.0, 173.0, 130.0)


def test_workspace_query_sizes(lib):
    cfg = C.cm_loss_cfg(10, C.CM_REF_ALL_EDGES, C.CM_SPLAT_ATOMIC, 0, 1e-9)
    n = C.cm_workspace_query(cam(), cfg, 100000, 1)
    # the IWE alone is R x H x W x 16 bytes
    assert n >= 11 * 346 * 260 * 16
    n_end = C.cm_workspace_query(cam(), C.cm_loss_cfg(10, C.CM_REF_END, 1, 0, 0.0), 100000, 1)
    assert n_end < n
    n_bins = C.cm_workspace_query(cam(), cfg, 100000, 10)
    assert n_bins > n


@pytest.mark.parametrize("bad", [
    dict(nbins=0), dict(nbins=33), dict(ref_mode=2), dict(splat=7), dict(store_warps=2),
])
def test_invalid_cfg_rejected(lib, bad):
    kw = dict(nbins=10, ref_mode=1, splat=1, store_warps=0, eps=1e-9)
    kw.update(bad)
    cfg = C.cm_loss_cfg(kw["nbins"], kw["ref_mode"], kw["splat"], kw["store_warps"], kw["eps"])
    with pytest.raises(C.CMError) as e:
        C.cm_workspace_query(cam(), cfg, 10, 1)
    assert e.value.status == C.CM_EINVAL


@pytest.mark.parametrize("w,h,fx", [(1, 10, 100.0), (10, 0, 100.0), (40000, 10, 100.0), (10, 10, 0.0),
                                    (10, 10, float("nan"))])
def test_invalid_camera_rejected(lib, w, h, fx):
    cfg = C.cm_loss_cfg(1, 0, 1, 0, 1e-9)
    with pytest.raises(C.CMError):
        C.cm_workspace_query(C.cm_camera(w, h, fx, 100.0, 5.0, 5.0), cfg, 10, 1)


def test_workspace_create_checks(lib):
    cfg = C.cm_loss_cfg(4, 1, 1, 0, 1e-9)
    need = C.cm_workspace_query(cam(64, 48), cfg, 1000, 4)
    fake = 1 << 40  # never dereferenced: creation only lays out offsets on the host
    with pytest.raises(C.CMError) as e:
        C.cm_workspace_create(fake, need - 1, cam(64, 48), cfg, 1000, 4)
    assert e.value.status == C.CM_ENOMEM
    with pytest.raises(C.CMError) as e:
        C.cm_workspace_create(fake + 8, need, cam(64, 48), cfg, 1000, 4)
    assert e.value.status == C.CM_EINVAL
    with pytest.raises(C.CMError):
        C.cm_workspace_create(fake, need, cam(64, 48), cfg, 1000, 3)  # n_flow_bins neither 1 nor B
    h = C.cm_workspace_create(fake, need, cam(64, 48), cfg, 1000, 4)
    a, b = C.cm_workspace_stats(h)
    assert fake <= a < fake + need and fake <= b < fake + need
    C.cm_workspace_destroy(h)


def test_entry_points_validate_before_launch(lib):
    cfg = C.cm_loss_cfg(4, 1, 1, 0, 1e-9)
    c = cam(64, 48)
    fake = 1 << 40
    ev = C.cm_events(fake, fake, fake, fake, 100, 0.0, 0.01)
    bad_ev = C.cm_events(fake, fake, fake, fake, 100, 0.01, 0.01)  # t1 == t0
    null_ev = C.cm_events(None, None, None, None, 100, 0.0, 0.01)
    ws = C.cm_workspace_create(fake, C.cm_workspace_query(c, cfg, 1000, 1), c, cfg, 1000, 1)
    try:
        for e in (bad_ev, null_ev):
            with pytest.raises(C.CMError) as x:
                C.cm_loss_forward(c, e, fake, 1, None, None, 0.01, cfg, ws, fake, None)
            assert x.value.status == C.CM_EINVAL
        # depth input needs inv_depth and ego
        with pytest.raises(C.CMError):
            C.cm_loss_forward(c, ev, None, 1, fake, None, 0.01, cfg, ws, fake, None)
        # too many events for this workspace
        big = C.cm_events(fake, fake, fake, fake, 1001, 0.0, 0.01)
        with pytest.raises(C.CMError) as x:
            C.cm_loss_forward(c, big, fake, 1, None, None, 0.01, cfg, ws, fake, None)
        assert x.value.status == C.CM_ENOMEM
        # shape mismatch with the workspace
        with pytest.raises(C.CMError):
            C.cm_loss_forward(cam(65, 48), ev, fake, 1, None, None, 0.01, cfg, ws, fake, None)
        # backward before any forward on this workspace
        with pytest.raises(C.CMError) as x:
            C.cm_loss_backward(c, ev, fake, 1, None, None, 0.01, cfg, ws, fake, fake, None, None, None)
        assert x.value.status == C.CM_ESTATE
        with pytest.raises(C.CMError):
            C.cm_flow_from_depth(c, None, fake, 0.01, fake, None)
        with pytest.raises(C.CMError):
            C.cm_warp_splat(c, ev, fake, 2, cfg, None, fake, None)  # n_flow_bins neither 1 nor B
    finally:
        C.cm_workspace_destroy(ws)


def test_batch_query_and_status_validate_on_the_host(lib):
    # sizes only (no device memory is touched): the deterministic mode holds
    # one image and quad slab per chain (at most eight), so a 64-window plan
    # needs far less than the atomic plan's slab per window, plus its sort
    # buffers; the status and stall-hook calls refuse a null plan
    fake = 1 << 40
    wins = []
    for i in range(64):
        ev = C.cm_events(fake, fake, fake, fake, 5000 + 1000 * i, 0.0, 0.01)
        wins.append(C.cm_window(cam(640, 480), ev, None, fake, fake, 0.01, fake, fake, None, fake, fake, None))
    atomic = C.cm_batch_query(wins, C.cm_loss_cfg(10, 1, 1, 0, 1e-9))
    sort = C.cm_batch_query(wins, C.cm_loss_cfg(10, 1, 2, 0, 1e-9))
    images = 64 * 11 * 640 * 480 * 16
    assert atomic > images
    assert sort < atomic / 2
    one = C.cm_batch_query(wins[:1], C.cm_loss_cfg(10, 1, 2, 0, 1e-9))
    assert one < sort
    assert lib.cm_batch_status(None, None) == C.CM_EINVAL
    assert lib.cm_batch_inject_stall(None, 0) == C.CM_EINVAL
    with pytest.raises(C.CMError) as x:  # a splat strategy batches do not know
        C.cm_batch_query(wins, C.cm_loss_cfg(10, 1, 7, 0, 1e-9))
    assert x.value.status == C.CM_EINVAL
