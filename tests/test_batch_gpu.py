"""The batched path (cm_batch_*): every window of an uneven batch, the phases
replayed from a CUDA graph, against the FP64 oracle (tests/gpu_util.py:
intervals on the full windows, strict on the windows without their flagged
events) and against the plain single-window path."""
import numpy as np
import pytest

from paper_2412_06359_gb300 import synth
from tests.gpu_util import GRAD_RTOL_L2, LOSS_RTOL, check_windows, gpu_lib, rel_l2, run_gpu

pytestmark = pytest.mark.gpu


def _dev_windows(cm, wins):
    import torch
    out = []
    for w in wins:
        d = {"cam": w.cam, "ev": cm.DeviceEvents.from_host(w.events)}
        if w.flow is not None:
            d["flow"] = torch.from_numpy(np.ascontiguousarray(w.flow[0])).cuda()
        else:
            d["inv_depth"] = torch.from_numpy(w.inv_depth).cuda()
            d["ego"] = torch.from_numpy(w.ego).cuda()
            d["dt"] = w.dt
        out.append(d)
    return out


def _batch_result(plan, i, win=None):
    import torch
    torch.cuda.synchronize()
    r = {"loss": float(plan.loss[i].item())}
    r["loss_r"], r["nnz_r"] = plan.stats(i)
    for k, v in plan.outputs[i].items():
        r[k] = v.cpu().numpy()
    if win is not None and win.flow is not None and "dflow" in r:
        r["dflow"] = r["dflow"][None]
    return r


def batch_runner(B=10, ref_mode=synth.REF_ALL, schedule=None, store_warps=False, want_dflow=False, reps=1,
                 autotune=False, splat=None):
    """A runner for check_windows: one batch plan over the windows."""
    def run(wins, eps):
        cm = gpu_lib()
        sp = cm.SPLAT_ATOMIC if splat is None else splat
        plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(B, ref_mode, sp, eps, store_warps),
                            want_dflow=want_dflow)
        if schedule is not None:
            plan.set_schedule(*schedule)
        if autotune:
            plan.autotune()
        for _ in range(reps):
            plan.run()
        return [_batch_result(plan, i, w) for i, w in enumerate(wins)]
    return run


def plan_results(plan, wins):
    return [_batch_result(plan, i, w) for i, w in enumerate(wins)]


def _mixed_windows(count, seed):
    rng = np.random.default_rng(seed)
    wins = []
    for i in range(count):
        W, H = [(96, 72), (120, 90), (64, 48), (160, 100)][i % 4]
        n = int(rng.integers(0, 6000)) if i % 5 else 0  # some empty windows
        wins.append(synth.depth_window(np.random.default_rng(seed * 100 + i), W, H, n, nbins=10))
    return wins


def test_batch_of_mixed_windows_matches_oracle():
    cm = gpu_lib()
    wins = _mixed_windows(9, 1)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    for rep in range(2):  # capture, then replay
        plan.run()
        for i, w in enumerate(wins):
            g = _batch_result(plan, i)
            if w.events.n == 0:
                assert g["loss"] == 0.0 and not np.any(g["dinv_depth"]) and not np.any(g["dego"])
        check_windows(wins, batch_runner(reps=2), full=plan_results(plan, wins))


def test_batch_flow_windows_end_reference():
    cm = gpu_lib()
    rng = np.random.default_rng(4)
    wins = []
    for i in range(5):
        W, H = 80 + 8 * i, 60
        ev = synth.uniform_events(rng, W, H, 3000 + 500 * i)
        flow = synth.sinusoid_flow(rng, W, H, 4.0)[None]
        wins.append(synth.Window(synth.Camera(W, H, 50.0, 50.0, W / 2, H / 2), ev, 4, synth.REF_END, flow=flow))
    check_windows(wins, batch_runner(B=4, ref_mode=cm.REF_END))


def test_batch_equals_plain_path_on_the_640x480_windows():
    # four windows of the 64-window workload: each batched result equals the plain
    # single-window result within the parity tolerances
    cm = gpu_lib()
    wins = synth.batch_windows(4)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.run()
    for i, w in enumerate(wins):
        g = _batch_result(plan, i)
        p = run_gpu(w)
        assert np.array_equal(g["nnz_r"], p["nnz_r"])
        assert abs(g["loss"] - p["loss"]) <= LOSS_RTOL * abs(p["loss"])
        assert rel_l2(g["dinv_depth"], p["dinv_depth"]) <= GRAD_RTOL_L2
        assert rel_l2(g["dego"], p["dego"]) <= GRAD_RTOL_L2


def test_band_grouping_on_the_640x480_windows_equals_the_plain_path():
    # bin 2: each window's events regrouped by 32-row band with a counting
    # sort over many 4096-event super-chunks (up to ~120 per window)
    cm = gpu_lib()
    wins = synth.batch_windows(4)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(2, 1, 2)
    for _ in range(2):
        plan.run()
    for i, w in enumerate(wins):
        g = _batch_result(plan, i)
        p = run_gpu(w)
        assert np.array_equal(g["nnz_r"], p["nnz_r"])
        assert abs(g["loss"] - p["loss"]) <= LOSS_RTOL * abs(p["loss"])
        assert rel_l2(g["dinv_depth"], p["dinv_depth"]) <= GRAD_RTOL_L2
        assert rel_l2(g["dego"], p["dego"]) <= GRAD_RTOL_L2


def test_batch_set_windows_reuses_the_graph():
    import torch
    cm = gpu_lib()
    first = _mixed_windows(6, 7)
    plan = cm.BatchPlan(_dev_windows(cm, first), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.run()
    # a smaller set of windows that fits the plan: reversed order, fewer windows
    second = list(reversed(first))[:4]
    plan.set_windows(_dev_windows(cm, second))
    plan.run()
    check_windows(second, batch_runner(), full=plan_results(plan, second))
    # windows larger than the plan's image memory are refused
    big = [synth.depth_window(np.random.default_rng(3), 640, 480, 100, nbins=10)] * 6
    from paper_2412_06359_gb300 import _capi as C
    with pytest.raises(C.CMError) as e:
        plan.set_windows(_dev_windows(cm, big))
    assert e.value.status == C.CM_ENOMEM
    torch.cuda.synchronize()


def test_batch_profiling_records_every_phase():
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    wins = _mixed_windows(4, 11)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(2, 1, 1)
    plan.run()
    C.cm_profile_reset()
    n0 = C.cm_launch_count()
    C.cm_profile_enable(True)
    for _ in range(3):
        plan.run()
    C.cm_profile_enable(False)
    plan.run()
    prof = C.cm_profile_collect()
    per_run = 7 * len(wins)  # seven kernels per window group (with tile grouping), one window per group
    assert C.cm_launch_count() - n0 == 4 * per_run
    assert set(prof) == {"k_prep_batch", "k_bin_count_batch", "k_bin_scatter_batch", "k_splat_batch", "k_loss_batch",
                         "k_adjoint_batch", "k_grad_batch"}
    assert all(v[0] == 3 * len(wins) and v[1] > 0 for v in prof.values())
    # results still right after switching the timing events back
    check_windows(wins, batch_runner(schedule=(2, 1, 1)), full=plan_results(plan, wins), grad=False)


@pytest.mark.parametrize("chains,group,bin", [(1, 0, 0), (1, 1, 0), (2, 1, 0), (3, 2, 0), (4, 1, 0),
                                              (1, 0, 1), (2, 1, 1), (3, 2, 1), (1, 0, 2), (2, 1, 2), (4, 2, 2),
                                              (1, 0, 3), (2, 1, 3), (3, 2, 3)])
def test_every_schedule_gives_the_same_results(chains, group, bin):
    cm = gpu_lib()
    wins = _mixed_windows(7, 21)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(chains, group, bin)
    assert plan.schedule() == (chains, group, bin, 0)
    plan.run()
    plan.run()
    check_windows(wins, batch_runner(schedule=(chains, group, bin), reps=2), full=plan_results(plan, wins))


def test_autotune_picks_a_schedule_and_stays_correct():
    cm = gpu_lib()
    wins = synth.batch_windows(6)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    chains, group, bin, persist = plan.autotune()
    assert 1 <= chains <= 8 and group >= 0 and bin in (0, 1, 2, 3) and 0 <= persist <= 8
    assert plan.autotune() == (chains, group, bin, persist)  # cached for this shape
    plan.run()
    sched = (chains, group, bin, persist)
    check_windows([wins[0], wins[3]], batch_runner(schedule=sched),
                  full=[_batch_result(plan, 0), _batch_result(plan, 3)])


@pytest.mark.parametrize("chains,group", [(1, 0), (2, 1)])
def test_batch_with_stored_warps(chains, group):
    cm = gpu_lib()
    wins = _mixed_windows(6, 31)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC, store_warps=True))
    plan.set_schedule(chains, group)
    for _ in range(2):
        plan.run()
    check_windows(wins, batch_runner(schedule=(chains, group), store_warps=True, reps=2),
                  full=plan_results(plan, wins))


def test_batch_of_motion_consistent_windows_matches_oracle():
    # many events per pixel after the warp (hot spots under the true flow):
    # the unordered reductions add more terms per address, same tolerances
    cm = gpu_lib()
    wins = [synth.motion_window(np.random.default_rng(70 + i), 160, 120, 20000 + 15000 * i) for i in range(3)]
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    for sched in ((2, 1, 0), (1, 0, 1), (2, 1, 2), (2, 1, 3)):
        plan.set_schedule(*sched)
        plan.run()
        check_windows(wins, batch_runner(schedule=sched), full=plan_results(plan, wins))


def test_batch_odd_sized_images_and_requested_dflow():
    # images with an odd pixel count (the loss pass then reads single pixels,
    # not 16-byte pairs) among even ones, depth and flow windows mixed; depth
    # windows also return dL/dflow when asked for it
    cm = gpu_lib()
    rng = np.random.default_rng(41)
    wins = []
    for i, (W, H) in enumerate([(97, 61), (96, 72), (81, 45), (131, 99)]):
        n = 2500 + 700 * i
        if i == 2:
            ev = synth.uniform_events(rng, W, H, n)
            flow = synth.sinusoid_flow(rng, W, H, 3.0)[None]
            wins.append(synth.Window(synth.Camera(W, H, 60.0, 60.0, W / 2, H / 2), ev, 10, synth.REF_ALL,
                                     flow=flow))
        else:
            wins.append(synth.depth_window(np.random.default_rng(4100 + i), W, H, n, nbins=10))
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC), want_dflow=True)
    for rep in range(2):
        plan.run()
        full = plan_results(plan, wins)
        assert all("dflow" in g for g in full)
    check_windows(wins, batch_runner(want_dflow=True, reps=2), full=full)  # dflow included


@pytest.mark.parametrize("B,ref_mode", [(32, synth.REF_ALL), (20, synth.REF_ALL), (32, synth.REF_END),
                                        (1, synth.REF_END), (1, synth.REF_ALL)])
def test_batch_bin_counts_up_to_the_maximum(B, ref_mode):
    # every event-kernel instantiation (1, 10, 20 and 32 bins) and the loss
    # pass's reference rounds (R = 1, 2, 21, 33) in the batched plan
    cm = gpu_lib()
    wins = [synth.depth_window(np.random.default_rng(5200 + i), W, H, n, nbins=B, ref_mode=ref_mode)
            for i, (W, H, n) in enumerate([(120, 90, 3000), (97, 61, 1500), (160, 100, 4000)])]
    check_windows(wins, batch_runner(B=B, ref_mode=ref_mode))


def test_band_grouping_with_events_outside_the_sensor_and_a_1280x720_window():
    # bin 2 with events whose (x, y) lies outside the sensor (their band is
    # that of the nearest row; they are masked as in the oracle) and with a
    # 1280x720 window (23 bands, 74 super-chunks) against the plain path
    cm = gpu_lib()
    small = synth.depth_window(np.random.default_rng(92), 160, 100, 5000, nbins=10)
    e = small.events
    x, y = e.x.copy(), e.y.copy()
    x[::97] = -2
    y[1::89] = 103
    x[2::101] = 161
    y[3::103] = -5
    small.events = synth.Events(x, y, e.t, e.p, e.t0, e.t1)
    hd = synth.depth_window(np.random.default_rng(93), 1280, 720, 300000, nbins=10)
    plan = cm.BatchPlan(_dev_windows(cm, [small, hd]), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(2, 1, 2)
    for _ in range(2):
        plan.run()
    check_windows([small], batch_runner(schedule=(2, 1, 2), reps=2), full=[_batch_result(plan, 0)])
    g, p = _batch_result(plan, 1), run_gpu(hd)
    assert np.array_equal(g["nnz_r"], p["nnz_r"])
    assert abs(g["loss"] - p["loss"]) <= LOSS_RTOL * abs(p["loss"])
    assert rel_l2(g["dinv_depth"], p["dinv_depth"]) <= GRAD_RTOL_L2
    assert rel_l2(g["dego"], p["dego"]) <= GRAD_RTOL_L2


def test_band_grouping_across_set_windows_and_schedule_changes():
    # bin 2 across new windows (event counts that change, some beyond the plan's
    # grouping memory, which then run in their given order) and across
    # switches between the grouping modes; every run against the oracle
    cm = gpu_lib()
    first = _mixed_windows(6, 57)
    plan = cm.BatchPlan(_dev_windows(cm, first), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(2, 1, 2)
    plan.run()
    second = []
    for i, w in enumerate(reversed(first)):
        # some grow past the grouping memory; at least 500 events (a lone event's gradient is eps-bound)
        n = w.events.n * 2 + 300 if i % 2 else max(w.events.n // 3, 500)
        second.append(synth.depth_window(np.random.default_rng(5800 + i), w.cam.width, w.cam.height, n, nbins=10))
    plan.set_windows(_dev_windows(cm, second))
    for sched in ((2, 1, 2), (1, 0, 1), (3, 2, 2), (1, 0, 0), (2, 1, 2)):
        plan.set_schedule(*sched)
        plan.run()
        check_windows(second, batch_runner(schedule=sched), full=plan_results(plan, second), grad=sched == (1, 0, 0))


@pytest.mark.parametrize("chains,group,bin,persist", [(0, 1, 0, 0), (9, 1, 0, 0), (2, -1, 0, 0), (2, 0, 0, 0),
                                                      (1, 1, 4, 0), (1, 1, -1, 0), (1, 0, 0, 9), (1, 0, 0, -1),
                                                      (2, 1, 0, 2), (1, 0, 1, 2), (1, 0, 3, 1)])
def test_invalid_schedules_are_refused_and_leave_the_plan_as_it_was(chains, group, bin, persist):
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    wins = _mixed_windows(3, 61)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(1, 1, 2)
    with pytest.raises(C.CMError) as e:
        plan.set_schedule(chains, group, bin, persist)
    assert e.value.status == C.CM_EINVAL
    assert plan.schedule() == (1, 1, 2, 0)
    plan.run()
    check_windows(wins, batch_runner(schedule=(1, 1, 2)), full=plan_results(plan, wins), grad=False)


def test_the_bench_windows_against_the_oracle():
    # the headline workload's own windows (640x480, 10 bins, 11 references) in
    # the bench's launch configuration (autotuned schedule, which picks band
    # grouping on this workload): four of the 64 windows, among them the one
    # with the most events, against the FP64 oracle
    wins = synth.batch_windows(64)
    idx = sorted({int(np.argmax([w.events.n for w in wins])), 0, 17, 40})
    sub = [wins[i] for i in idx]
    assert max(w.events.n for w in sub) > 400_000
    flagged = check_windows(sub, batch_runner(schedule=(6, 2, 2)))
    assert all(f < 0.005 * w.events.n for f, w in zip(flagged, sub))
    check_windows(sub[:2], batch_runner(autotune=True), grad=False)


@pytest.mark.parametrize("B,ref_mode", [(10, synth.REF_ALL), (20, synth.REF_ALL), (5, synth.REF_END),
                                        (1, synth.REF_END)])
def test_shared_memory_tiles_strategy(B, ref_mode):
    # CM_SPLAT_TILES: the plan starts on bin 3 (events grouped by 32x32 tile,
    # the splat and the adjoint's pushes accumulated per tile in shared memory);
    # 20 bins have 21 references, of which the first 12 are held in shared
    # memory and the rest go straight to the images
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    wins = [synth.depth_window(np.random.default_rng(7300 + i), W, H, n, nbins=B, ref_mode=ref_mode)
            for i, (W, H, n) in enumerate([(120, 90, 6000), (97, 61, 1500), (200, 150, 20000)])]
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(B, ref_mode, cm.SPLAT_TILES))
    assert plan.schedule()[2] == 3 and plan.schedule()[3] == 0
    plan.run()
    check_windows(wins, batch_runner(B=B, ref_mode=ref_mode, splat=cm.SPLAT_TILES),
                  full=plan_results(plan, wins))
    # the single-window entry points refuse the strategy
    cfg = cm.loss_cfg(B, ref_mode, cm.SPLAT_TILES)
    with pytest.raises(C.CMError) as e:
        cm.Workspace(wins[0].cam, cfg, 100)
    assert e.value.status == C.CM_EINVAL


def test_shared_memory_tiles_on_the_bench_windows_and_hot_spots():
    # the 640x480 bench windows (incl. the largest) and motion-consistent windows
    # (many events per pixel after the warp: the warp-aggregated path) under bin 3
    cm = gpu_lib()
    wins = synth.batch_windows(64)
    sub = [wins[int(np.argmax([w.events.n for w in wins]))], wins[3]]
    check_windows(sub, batch_runner(schedule=(2, 1, 3)), grad=False)
    mot = [synth.motion_window(np.random.default_rng(80 + i), 160, 120, 40000) for i in range(2)]
    check_windows(mot, batch_runner(schedule=(2, 1, 3)))


@pytest.mark.parametrize("persist,bin", [(1, 0), (2, 2), (3, 2), (7, 0)])
def test_persistent_step_matches_the_oracle(persist, bin):
    # one persistent kernel per run: mixed windows (some empty), replayed, then
    # new windows through set_windows (the queue's size is read from the
    # uploaded header, so the graph stays)
    cm = gpu_lib()
    wins = _mixed_windows(9, 83)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(1, 0, bin, persist)
    assert plan.schedule() == (1, 0, bin, persist)
    for _ in range(2):
        plan.run()
    check_windows(wins, batch_runner(schedule=(1, 0, bin, persist), reps=2), full=plan_results(plan, wins))
    second = list(reversed(wins))[:6]
    plan.set_windows(_dev_windows(cm, second))
    plan.run()
    check_windows(second, batch_runner(schedule=(1, 0, bin, persist)), full=plan_results(plan, second), grad=False)


def test_persistent_step_on_the_bench_windows_with_stored_warps_and_many_bins():
    cm = gpu_lib()
    wins = synth.batch_windows(64)
    sub = [wins[int(np.argmax([w.events.n for w in wins]))], wins[5], wins[9]]
    check_windows(sub, batch_runner(schedule=(1, 0, 2, 2)))
    mixed = _mixed_windows(5, 91)
    check_windows(mixed, batch_runner(schedule=(1, 0, 2, 3), store_warps=True), grad=False)
    deep = [synth.depth_window(np.random.default_rng(9400 + i), W, H, n, nbins=20)
            for i, (W, H, n) in enumerate([(120, 90, 3000), (160, 100, 5000)])]
    check_windows(deep, batch_runner(B=20, schedule=(1, 0, 2, 2)))


def test_persistent_wait_gives_up_reports_and_the_plan_recovers():
    # failure path of the persistent step's bounded waits: a window whose prep
    # pass is left out of the queue (test hook) blocks its later phases; the
    # first wait to reach its bound (about 4 s) sets the error word, every
    # other wait returns at once, the kernel ends and the run reports
    # CM_ETIMEOUT.  With the queue restored the same plan is correct again.
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    wins = _mixed_windows(5, 97)
    plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_ATOMIC))
    plan.set_schedule(1, 0, 2, 2)
    plan.run()
    assert plan.status() == C.CM_OK
    plan.inject_stall(1)
    plan.run()
    assert plan.status() == C.CM_ETIMEOUT
    plan.inject_stall(-1)
    plan.run()
    assert plan.status() == C.CM_OK
    check_windows(wins, batch_runner(schedule=(1, 0, 2, 2)), full=plan_results(plan, wins), grad=False)
    plan.set_schedule(6, 1, 2, 0)  # the graph path has no device waits
    plan.run()
    assert plan.status() == C.CM_OK


def _bitwise_equal(a, b):
    for k in a:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        assert x.dtype == y.dtype and x.shape == y.shape and x.tobytes() == y.tobytes(), k


@pytest.mark.parametrize("want_dflow", [False, True])
def test_batched_deterministic_mode_is_bit_reproducible_and_matches_the_oracle(want_dflow):
    # CM_SPLAT_SORT in a batch: the windows one after another through the sort
    # path, every sum in a fixed order; the same bits on every replay and after
    # the windows are set again, and the oracle's verdict on every window
    from paper_2412_06359_gb300 import _capi as C
    cm = gpu_lib()
    wins = _mixed_windows(6, 101)
    wins.append(synth.motion_window(np.random.default_rng(102), 90, 70, 4000))  # a flow-input window too
    dev = _dev_windows(cm, wins)
    plan = cm.BatchPlan(dev, cm.loss_cfg(10, cm.REF_ALL, cm.SPLAT_SORT), want_dflow=want_dflow)
    assert plan.schedule() == (min(len(wins), 8), 1, 0, 0)  # one window at a time on each chain
    for bad in [(9, 1, 0, 0), (2, 2, 0, 0), (2, 1, 2, 0), (1, 0, 0, 1)]:
        with pytest.raises(C.CMError):
            plan.set_schedule(*bad)
    plan.run()
    first = plan_results(plan, wins)
    for _ in range(2):
        plan.run()
    for a, b in zip(first, plan_results(plan, wins)):
        _bitwise_equal(a, b)
    # the same bits whatever the number of chains, after the windows are set again, and autotuned
    for chains in (1, 3):
        plan.set_schedule(chains, 1, 0, 0)
        plan.run()
        for a, b in zip(first, plan_results(plan, wins)):
            _bitwise_equal(a, b)
    plan.set_windows(dev)
    plan.run()
    for a, b in zip(first, plan_results(plan, wins)):
        _bitwise_equal(a, b)
    c, g, bn, p = plan.autotune()
    assert 1 <= c <= 8 and (g, bn, p) == (1, 0, 0)
    plan.run()
    for a, b in zip(first, plan_results(plan, wins)):
        _bitwise_equal(a, b)
    check_windows(wins, batch_runner(splat=cm.SPLAT_SORT, want_dflow=want_dflow), full=first)


def test_batched_deterministic_mode_many_bins_and_stored_warps():
    # 20 bins (21 references) and the stored-warp backward in the deterministic
    # mode: the same bits twice, the oracle's verdict on every window
    cm = gpu_lib()
    wins = [synth.depth_window(np.random.default_rng(9600 + i), W, H, n, nbins=20)
            for i, (W, H, n) in enumerate([(120, 90, 3000), (160, 100, 5000), (64, 48, 0), (96, 72, 2500)])]
    for sw in (False, True):
        plan = cm.BatchPlan(_dev_windows(cm, wins), cm.loss_cfg(20, cm.REF_ALL, cm.SPLAT_SORT, store_warps=sw))
        plan.run()
        first = plan_results(plan, wins)
        plan.run()
        for a, b in zip(first, plan_results(plan, wins)):
            _bitwise_equal(a, b)
        check_windows(wins, batch_runner(B=20, splat=cm.SPLAT_SORT, store_warps=sw), full=first)
