#!/usr/bin/env python
"""Throughput of the contrast-maximisation loss + gradient on one GB300.

Workload: the uneven 64-window batch (640x480 sensor, fx = fy = 450, event
counts log-uniform in [5k, 500k] per window, each window with its own
inverse-depth map and ego-motion, 10 bins, all 11 bin edges as references).
A step is one full forward + backward (loss, dL/d inverse depth, dL/d
ego-motion) of every window of the batch; the metric is input events of such
evaluations per second (Mev/s).  Inputs are seeded synthetic windows resident
in HBM before the timed region.

Printed as one JSON line (rank 0).  --impl reference times the CPU oracle on
the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CM loss+grad Mevents/s batched vs plain per-window at ≤1e-5 rel err; p50/p99 latency"
WORKLOAD = "batch64_640x480_b10"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--windows", type=int, default=64, help="windows per step (64 for the headline workload)")
    ap.add_argument("--no-plain", action="store_true", help="skip the per-window plain comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bound of the CPU oracle sample")
    ap.add_argument("--schedule", default="auto",
                    help="batch schedule 'chains,windows_per_kernel,grouping[,persist]' (grouping 0: given order, "
                         "1: 32x32 tiles, 2: 32-row bands, 3: tiles in shared memory; persist k > 0: one persistent "
                         "kernel staggering the windows by k - 1 phases, with 1,0,g; e.g. 6,2,2 or 1,0,2,2), or 'auto'")
    ap.add_argument("--events", default="iid", choices=["iid", "motion"],
                    help="iid: the headline workload; motion: motion-consistent events with their true flow "
                         "(flow input, many events per pixel after the warp: the contention stress variant)")
    ap.add_argument("--store-warps", type=int, default=0, choices=[0, 1],
                    help="1: the forward stores the trajectory points for the backward (no recompute)")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead (one line per rate)")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving leg of the default line")
    ap.add_argument("--latency", action="store_true",
                    help="single-window latency of the parity workloads (128x128 flow, 346x260 and 1280x720 depth)")
    ap.add_argument("--reps", type=int, default=200, help="repetitions per workload of --latency")
    ap.add_argument("--other-kernels", action="store_true",
                    help="time only the kernels beside the CM path (Eq. 2 flow, geometry loss, event frame)")
    ap.add_argument("--serve-scales", default="0.25,0.5,1.0", help="arrival-rate multipliers of 100 Hz per stream")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-pool", type=int, default=2, help="pre-generated windows per stream")
    ap.add_argument("--serve-lanes", type=int, default=6, help="concurrent lanes of the server")
    ap.add_argument("--serve-batch", type=int, default=8, help="requests per batch of a lane")
    ap.add_argument("--serve-group", type=int, default=16_000_000,
                    help="events per lane batch regrouped by 32-row band before the splat (0: given order)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---------------------------------------------------------------------------
# several GPUs: replicas.  Windows are independent, so every rank evaluates its
# own windows (weak scaling) and the only collective is the timing reduction.


def first_window_of(rank: int, windows: int) -> int:
    """Rank r evaluates windows r*windows .. (r+1)*windows - 1 of the seeded sequence."""
    return rank * windows


def reduce_over_ranks(total_ms: float, events: int, device):
    """(max over ranks of the timed region, sum over ranks of the events)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, events
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    e = torch.tensor([float(events)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(e.item()))


# ---------------------------------------------------------------------------
# GPU clocks during the timed region


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic bytes per kernel launch (strict model: events read by the forward
# splat and by the adjoint, 9 B each; inverse depth read by the flow kernel and
# its gradient written by the depth/ego kernel, 4 B per pixel each; the IWE is
# intermediate state).  The materialised-IWE model adds the dense IWE traffic
# of this design: 16 B per pixel and reference written by the splat, read and
# rewritten by the loss pass, gathered by the adjoint.


def kernel_bytes(name: str, n: int, hw: int, R: int, model: str) -> float:
    """Algorithmic bytes of one launch of `name` that processes n events over
    hw pixels (summed over the windows the launch covers) with R references.
    strict: events read by the splat and the adjoint (9 B each), inverse depth
    read by the prep pass and its gradient written by the gradient pass (4 B
    per pixel each).  iwe adds the dense traffic of this design: the images
    (16 B per pixel and reference) zeroed by the prep pass, reduced into by the
    splat, read by the loss pass and gathered by the adjoint; the 32-byte flow
    quads and gradient records written by the prep pass and read by the
    gradient pass, which also writes dL/dflow (8 B per pixel)."""
    iwe = model == "iwe"
    base = name.replace("_batch", "")
    if base in ("k_splat", "k_adjoint"):
        return 9.0 * n + (16.0 * R * hw if iwe else 0.0)
    if base == "k_prep":
        return 4.0 * hw + ((16.0 * R + 64.0) * hw if iwe else 0.0)
    if base == "k_loss":
        return 16.0 * R * hw if iwe else 0.0
    if base == "k_grad":
        return 4.0 * hw + (40.0 * hw if iwe else 0.0)
    return 0.0


def kernel_bytes_step(n: int, hw: int, R: int) -> float:
    """Strict algorithmic bytes of a whole step: 18 B per event (read by the
    splat and by the adjoint) and 8 B per pixel (inverse depth read, its
    gradient written)."""
    return 18.0 * n + 8.0 * hw


def workload_config(wins, events_kind: str, events_per_step: int) -> dict:
    """The workload as both arms name it (the `config` of the JSON line)."""
    R = wins[0].nbins + 1 if wins[0].ref_mode == 1 else 1
    hw = wins[0].cam.width * wins[0].cam.height
    return {"workload": WORKLOAD if events_kind == "iid" else WORKLOAD + "_motion",
            "events": "iid (gradient-sampled pixels, uniform times)" if events_kind == "iid"
            else "motion-consistent, flow input with the true flow (contention stress variant)",
            "windows": len(wins), "events_per_step": int(events_per_step),
            "sensor": f"{wins[0].cam.width}x{wins[0].cam.height}", "bins": wins[0].nbins, "refs": R,
            "l2": "per-step IWE working set %.2f GB > L2 (no flush needed)" % (len(wins) * R * hw * 16 / 1e9)}


# the batch schedule's event grouping modes (cm_batch_schedule.bin)
GROUPING = ("given order", "32x32 tiles", "32-row bands", "32x32 tiles, shared-memory accumulation")


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the device sources of the batched plan's kernels: recorded ncu
    counters hold while it is unchanged."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2412_06359_gb300", "csrc")
    for f in ("cm_device.cuh", "cm_bands.cuh", "cm_batch_kernels.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_counters(kernel: str):
    """Per-event ncu counters of an event kernel from the committed summary
    (profiles/event_kernels_ncu_counters.md: DRAM bytes and L2 requests per
    input event), or None when the kernel sources changed since they were taken."""
    p = os.path.join(ROOT, "profiles", "event_kernels_ncu_counters.md")
    try:
        text = open(p).read()
        block = text.split("```json", 1)[1].split("```", 1)[0]
        d = json.loads(block)
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("kernels", {}).get(kernel)


def l2_rates(device):
    """Random-request rates of this GPU's L2 (reductions/s, loads/s), measured
    by the library's probe over a 64 MiB buffer (about one window's images)."""
    import torch
    from paper_2412_06359_gb300 import _capi as C
    buf = torch.empty(64 << 20, dtype=torch.uint8, device=device)
    red, ld = C.cm_measure_l2_rates(buf.data_ptr(), buf.numel(), torch.cuda.current_stream(device).cuda_stream)
    del buf
    return red, ld


# ---------------------------------------------------------------------------
# CPU oracle baseline


def oracle_sample(windows, seconds: float):
    """Time the FP64 oracle (single thread) on windows of the workload until
    `seconds` of CPU work are done; returns (events, seconds, windows used)."""
    from oracle import oracle as O
    O.build()
    ev = 0
    t_total = 0.0
    used = 0
    for w in windows:
        t0 = time.perf_counter()
        O.cm_window(w, grad=True)
        t_total += time.perf_counter() - t0
        ev += w.events.n
        used += 1
        if t_total >= seconds:
            break
    return ev, t_total, used


def _oracle_share(j: int, idx: list, motion: bool, ready_q, go, out_q):
    """Worker of oracle_all_cores: the workload's windows `idx`, generated
    first, evaluated once `go` is set."""
    from paper_2412_06359_gb300 import synth
    from oracle import oracle as O
    gen = synth.batch_windows_motion if motion else synth.batch_windows
    wins = [gen(1, first=i)[0] for i in idx]
    ready_q.put(j)
    go.wait()
    ev = 0
    for w in wins:
        O.cm_window(w, grad=True)
        ev += w.events.n
    out_q.put(ev)


def oracle_all_cores(sizes: list, motion: bool, limit_s: float = 300.0):
    """The FP64 oracle as it stands on every host core: one spawned process per
    core, each evaluating its share of the workload's windows (loss + gradient,
    one thread each; windows of event counts `sizes` dealt largest first to the
    least loaded process); wall time from the moment every process holds its
    windows to the last result.  Returns (events, seconds, processes), or None
    when a process fails or exceeds `limit_s`."""
    import multiprocessing as mp
    import queue
    from oracle import oracle as O
    O.build()  # compiled once here, loaded by the workers
    nproc = max(1, min(os.cpu_count() or 1, len(sizes)))
    share, load = [[] for _ in range(nproc)], [0] * nproc
    for i in sorted(range(len(sizes)), key=lambda i: -sizes[i]):
        j = load.index(min(load))
        share[j].append(i)
        load[j] += sizes[i]
    ctx = mp.get_context("spawn")
    ready_q, out_q, go = ctx.Queue(), ctx.Queue(), ctx.Event()
    procs = [ctx.Process(target=_oracle_share, args=(j, share[j], motion, ready_q, go, out_q)) for j in range(nproc)]
    for q in procs:
        q.start()
    try:
        for _ in procs:
            ready_q.get(timeout=limit_s)
        t0 = time.perf_counter()
        go.set()
        ev = sum(out_q.get(timeout=limit_s) for _ in procs)
        sec = time.perf_counter() - t0
        return ev, sec, nproc
    except queue.Empty:
        return None
    finally:
        for q in procs:
            q.join(timeout=10)
            if q.is_alive():
                q.terminate()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2412_06359_gb300 import synth
    wins = synth.batch_windows(args.windows)
    from oracle import oracle as O
    O.build()
    # each step: the oracle on one window of the batch (rotating), a bounded sample
    for i in range(args.warmup):
        O.cm_window(wins[i % len(wins)], grad=True)
    ev = 0
    t0 = time.perf_counter()
    times = []
    for i in range(args.steps):
        w = wins[i % len(wins)]
        s = time.perf_counter()
        O.cm_window(w, grad=True)
        times.append(time.perf_counter() - s)
        ev += w.events.n
    el = time.perf_counter() - t0
    v = ev / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Mev/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wins, "iid", sum(w.events.n for w in wins)),
        "sample": "one window of the batch per step (rotating through the batch)",
        "cpu_baseline": {"value": v, "unit": "Mev/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} windows of the 64-window batch, one per step, loss + gradient"},
        "e2e": {"value": v, "unit": "Mev/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our path


class Batch:
    """The windows of one step resident on the device: a batched plan over all
    of them (the timed path) and one workspace per window for the plain
    per-window comparison through the single-window entry points.  Windows
    take inverse depth and ego-motion, or a given flow (the motion-consistent
    stress variant)."""

    def __init__(self, wins, device, store_warps=False):
        import torch

        from paper_2412_06359_gb300 import cm
        self.cm = cm
        self.wins = wins
        self.dev = device
        self.items = []
        self.flow_input = wins[0].flow is not None
        dev_wins = []
        for w in wins:
            cfg = cm.loss_cfg(w.nbins, w.ref_mode, cm.SPLAT_ATOMIC, store_warps=store_warps)
            ws = cm.Workspace(w.cam, cfg, w.events.n, 1, device)
            ev = cm.DeviceEvents.from_host(w.events, device)
            loss = torch.empty(1, device=device)
            if self.flow_input:
                flow = torch.from_numpy(np.ascontiguousarray(w.flow[0])).to(device)
                self.items.append((w, ws, ev, flow, None, {"dflow": torch.empty_like(flow)}, loss))
                dev_wins.append({"cam": w.cam, "ev": ev, "flow": flow})
            else:
                rho = torch.from_numpy(w.inv_depth).to(device)
                ego = torch.from_numpy(w.ego).to(device)
                out = {"dinv_depth": torch.empty_like(rho), "dego": torch.empty(6, device=device)}
                self.items.append((w, ws, ev, rho, ego, out, loss))
                dev_wins.append({"cam": w.cam, "ev": ev, "inv_depth": rho, "ego": ego, "dt": w.dt})
        self.dloss = torch.ones(1, device=device)
        self.dev_wins = dev_wins
        self.plan = cm.BatchPlan(dev_wins, cm.loss_cfg(wins[0].nbins, wins[0].ref_mode, cm.SPLAT_ATOMIC,
                                                       store_warps=store_warps), device)
        self.events = sum(w.events.n for w in wins)

    def step(self):
        self.plan.run()

    def window_call(self, it):
        """Loss and gradient of one window through the single-window calls."""
        w, ws, ev, a, b, out, loss = it
        if self.flow_input:
            self.cm.loss_forward(ws, ev, flow=a, out=loss)
            self.cm.loss_backward(ws, ev, self.dloss, flow=a, out=out)
        else:
            self.cm.loss_forward(ws, ev, inv_depth=a, ego=b, dt=w.dt, out=loss)
            self.cm.loss_backward(ws, ev, self.dloss, inv_depth=a, ego=b, dt=w.dt, want_dflow=False, out=out)

    def plain_window(self, i):
        import torch
        self.window_call(self.items[i])
        torch.cuda.current_stream().synchronize()


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2412_06359_gb300 import _capi as C
    from paper_2412_06359_gb300 import build, synth
    build.build()
    C.lib()

    # weak scaling: every rank evaluates its own 64 windows
    if args.events == "motion":
        wins = synth.batch_windows_motion(args.windows, first=first_window_of(rank, args.windows))
    else:
        wins = synth.batch_windows(args.windows, first=first_window_of(rank, args.windows))
    batch = Batch(wins, dev, store_warps=bool(args.store_warps))
    hw = wins[0].cam.width * wins[0].cam.height
    R = wins[0].nbins + 1
    stream = torch.cuda.current_stream()

    l2 = l2_rates(dev)
    if args.schedule == "auto":
        schedule = batch.plan.autotune()  # picks chains / windows per kernel for this batch (cached per shape)
    else:
        batch.plan.set_schedule(*[int(v) for v in args.schedule.split(",")])
        schedule = batch.plan.schedule()
    for _ in range(args.warmup):
        batch.step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, CUDA events on the launching stream ----
    ev_steps = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    C.cm_profile_reset()
    launches0 = C.cm_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        C.cm_profile_enable(True)
        ev_steps[0].record(stream)
        for k in range(args.steps):
            batch.step()
            ev_steps[k + 1].record(stream)
        torch.cuda.synchronize()
        C.cm_profile_enable(False)
    launches = C.cm_launch_count() - launches0
    step_ms = [ev_steps[k].elapsed_time(ev_steps[k + 1]) for k in range(args.steps)]
    total_ms = ev_steps[0].elapsed_time(ev_steps[-1])
    total_ms, job_events = reduce_over_ranks(total_ms, batch.events, dev)
    if world > 1:
        dist.barrier()
    clocks = clk.summary()
    prof = C.cm_profile_collect()
    ms_per_step = total_ms / args.steps
    value = job_events / (ms_per_step * 1e-3) / 1e6

    # ---- roofline of the dominant kernel ----
    peak, peak_kind = measured_peak()
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = None
    roof_iwe = None
    roof_l2 = None
    if dom:
        nl, ms = prof[dom]
        launches_per_step = nl / args.steps
        # the kernel's time: its share of the summed kernel time (CUDA events
        # around every launch), applied to the step's device time.  Launches of
        # concurrent chains overlap, so a launch's own event interval includes
        # the time it shares the GPU; the share does not.
        summed = sum(v[1] for v in prof.values())
        overlap = summed / args.steps / ms_per_step
        share = ms / summed
        per_launch_ms = share * ms_per_step / launches_per_step
        for model in ("strict", "iwe"):
            b = kernel_bytes(dom, batch.events, hw * len(wins), R, model) / launches_per_step
            ach = b / (per_launch_ms * 1e-3) / 1e9
            cnt = recorded_counters(dom)
            events_per_launch = batch.events / launches_per_step
            traffic = None if cnt is None or model != "strict" else cnt["dram_bytes_per_event"] * events_per_launch
            obj = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                   "traffic": traffic, "kernel": dom,
                   "launch_ms": per_launch_ms, "launch_ms_events": ms / nl, "share_of_kernel_time": share,
                   "bytes_per_launch": b, "launches_per_step": launches_per_step,
                   "step_bytes_strict": kernel_bytes_step(batch.events, hw * len(wins), R),
                   "step_frac_strict": kernel_bytes_step(batch.events, hw * len(wins), R) / (ms_per_step * 1e-3)
                   / 1e9 / peak,
                   "overlap": overlap, "peak_kind": f"{peak_kind} hbm_gbs"}
            if model == "strict":
                roof = obj
            else:
                roof_iwe = obj
        # request-bound model, for the whole step: the L2 requests of the two
        # event kernels (ncu counts per event x the step's events) over the
        # step's device time, against the random-request rates measured on this
        # GPU (a kernel's share of a step whose kernels overlap 5-6x is no time
        # of its own at which to rate its requests)
        cs, ca = recorded_counters("k_splat_batch"), recorded_counters("k_adjoint_batch")
        if cs is not None and ca is not None and l2 is not None:
            ev = batch.events
            rd = (cs["l2_read_requests_per_event"] + ca["l2_read_requests_per_event"]) * ev
            rq = (cs["l2_red_requests_per_event"] + ca["l2_red_requests_per_event"]) * ev
            t_min = rd / l2[1] + rq / l2[0]
            ach = (rd + rq) / (ms_per_step * 1e-3) / 1e9
            pk = (rd + rq) / t_min / 1e9
            roof_l2 = {"bound": "l2_requests", "achieved": ach, "peak": pk, "unit": "G requests/s",
                       "frac": ach / pk, "scope": "step: k_splat_batch + k_adjoint_batch requests per step",
                       "requests_per_step": rd + rq,
                       "read_requests_per_event": cs["l2_read_requests_per_event"] + ca["l2_read_requests_per_event"],
                       "red_requests_per_event": cs["l2_red_requests_per_event"] + ca["l2_red_requests_per_event"],
                       "measured_red_per_s": l2[0], "measured_load_per_s": l2[1],
                       "peak_kind": "measured by cm_measure_l2_rates on this GPU before the timed region"}

    # ---- plain per-window comparison (a stream sync after every window) ----
    plain = None
    if not args.no_plain:
        for i in range(min(3, len(wins))):
            batch.plain_window(i)
        lat = []
        t0 = time.perf_counter()
        for i in range(len(wins)):
            s = time.perf_counter()
            batch.plain_window(i)
            lat.append(1e3 * (time.perf_counter() - s))
        el = time.perf_counter() - t0
        plain = {"value": batch.events / el / 1e6, "unit": "Mev/s", "p50_ms": float(np.percentile(lat, 50)),
                 "p99_ms": float(np.percentile(lat, 99)), "windows": len(wins)}

    # ---- the splat strategies: single-window calls (atomic, sort) and the
    # batched plan (direct reductions, shared-memory tiles) on the bench's
    # windows and on motion-consistent windows (many events per pixel) ----
    splat_cmp = sched_cmp = None
    if not args.no_plain:
        splat_cmp = compare_splats(batch, min(4, len(wins)))
        c, g = schedule[0], schedule[1]
        splat_cmp["batched_iid"] = compare_batched_splats(
            batch, {"direct_bands": (c, g, 2), "direct_given_order": (c, g, 0), "smem_tiles": (c, g, 3)})
        splat_cmp["batched_iid"]["deterministic_sort"] = compare_deterministic(batch)
        batch.plan.set_schedule(*schedule)
        from paper_2412_06359_gb300 import synth as _synth
        mot = Batch(_synth.batch_windows_motion(8), dev)
        splat_cmp["batched_motion"] = compare_batched_splats(
            mot, {"direct_given_order": (2, 1, 0), "direct_bands": (2, 1, 2), "smem_tiles": (2, 1, 3)})
        splat_cmp["batched_motion"]["windows"] = 8
        splat_cmp["batched_motion"]["events"] = mot.events
        del mot
        # the graph of per-phase kernels against the persistent step (device work queue)
        sched_cmp = compare_batched_splats(batch, {
            "graph_6x2_bands": (6, 2, 2, 0), "graph_8x2_bands": (8, 2, 2, 0),
            "persistent_bands_stagger0": (1, 0, 2, 1), "persistent_bands_stagger1": (1, 0, 2, 2),
            "persistent_bands_stagger2": (1, 0, 2, 3), "persistent_bands_stagger7": (1, 0, 2, 8),
            "persistent_given_order_stagger1": (1, 0, 0, 2)})
        batch.plan.set_schedule(*schedule)

    # ---- the kernels beside the CM path (discrete flow, geometry loss, event frame) ----
    others = None
    if rank == 0 and not args.no_plain:
        others = measure_other_kernels(dev, peak)

    # ---- end to end through the public API with host buffers ----
    e2e = None
    if not args.no_e2e and not batch.flow_input:
        e2e = run_e2e(batch, args, stream, schedule)

    # ---- a short serving leg (32 streams, 0.5x and 1x the arrival rate, 3 runs each) ----
    serve = None
    if rank == 0 and world == 1 and not args.no_serve:
        serve = serve_leg([0.5, 0.9, 1.0], 2.0, 3, args.serve_lanes, args.serve_batch, args.serve_group)

    # ---- CPU oracle baseline (rank 0 at N = 1 only) ----
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n, sec, used = oracle_sample(wins, args.cpu_seconds)
        cpu = {"value": n / sec / 1e6, "unit": "Mev/s", "cores": 1, "kind": "oracle",
               "sample": f"first {used} windows of the batch ({n} events), loss + gradient, FP64, one thread"}
        par = oracle_all_cores([w.events.n for w in wins], args.events == "motion")
        if par:
            n, sec, nproc = par
            cpu_all = {"value": n / sec / 1e6, "unit": "Mev/s", "cores": nproc, "kind": "oracle",
                       "sample": f"all {len(wins)} windows of the batch ({n} events), loss + gradient, FP64, one "
                                 f"process per host core, windows dealt largest first to the least loaded"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mev/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(wins, args.events, batch.events),
            "plan": {"splat": "atomic", "backward": "stored warps" if args.store_warps else "recompute",
                     "path": "batched plan replayed from a CUDA graph",
                     "schedule": {"chains": schedule[0], "windows_per_kernel": schedule[1],
                                  "grouping": GROUPING[schedule[2]],
                                  "persistent": schedule[3] > 0,
                                  "stagger": schedule[3] - 1 if schedule[3] > 0 else None}},
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "plain": plain, "splat_compare": splat_cmp, "schedule_compare": sched_cmp, "roofline": roof,
            "roofline_iwe": roof_iwe,
            "roofline_l2": roof_l2, "other_kernels": others, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all, "e2e": e2e, "serve": serve,
            "clocks": clocks, "gpu_launches": int(launches),
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_other_kernels(device, peak: float, reps: int = 10):
    """The kernels beside the CM path on a 1280x720 sensor: the discrete flow
    (Eq. 2, 20 bins) and its adjoint, the geometry-consistency loss (Eq. 3)
    and its gradient, and the network's event frame of 2M events.  Device time
    per call from the library's CUDA events around its own kernels; between
    calls a 256 MB buffer is written so that no call finds its inputs in L2.
    Achieved bandwidth is over the algorithmic bytes against the measured HBM
    peak."""
    import torch
    from paper_2412_06359_gb300 import _capi as C
    from paper_2412_06359_gb300 import cm, synth
    W, H, nb = 1280, 720, 20
    hw = W * H
    cam = synth.camera_for(W, H)
    rng = synth.rng_for(4)
    rho = torch.from_numpy(synth.inv_depth_map(rng, W, H)).to(device)
    rho1 = rho * 1.02
    ego = torch.from_numpy(np.stack([synth.ego_motion(rng) for _ in range(nb)]).astype(np.float32)).to(device)
    dt, scale = 0.01 / nb, float(nb)
    g = torch.randn(nb, H, W, 2, device=device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    ev = cm.DeviceEvents.from_host(synth.uniform_events(rng, W, H, 2_000_000), device)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(device)
        C.cm_profile_reset()
        for _ in range(reps):
            flush.fill_(1)
            C.cm_profile_enable(True)
            fn()
            C.cm_profile_enable(False)
        torch.cuda.synchronize(device)
        prof = C.cm_profile_collect()
        return sum(v[1] for v in prof.values()) / reps

    def entry(ms, nbytes, unit_count, unit):
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"ms": ms, "bytes": nbytes, "gbs": gbs, "frac": gbs / peak, "per_s": unit_count / (ms * 1e-3),
                "unit": unit}

    e0 = ego[0].contiguous()
    scratch = torch.empty(C.cm_geo_scratch_query(cm.camera(cam)), dtype=torch.uint8, device=device)
    loss = torch.empty(1, device=device)
    ones = torch.ones(1, device=device)
    d0, d1, de = torch.empty_like(rho), torch.empty_like(rho), torch.empty(6, device=device)
    c = cm.camera(cam)

    def geo_f():
        C.cm_geo_forward(c, rho.data_ptr(), rho1.data_ptr(), e0.data_ptr(), 0.01, scratch.data_ptr(), scratch.numel(),
                         loss.data_ptr(), cm.stream_handle(device))

    def geo_b():
        C.cm_geo_backward(c, rho.data_ptr(), rho1.data_ptr(), e0.data_ptr(), 0.01, ones.data_ptr(), d0.data_ptr(),
                          d1.data_ptr(), de.data_ptr(), scratch.data_ptr(), scratch.numel(), cm.stream_handle(device))

    geo_f()
    out = {
        "sensor": "1280x720", "peak_gbs": peak,
        "flow_eq2_b20": entry(timed(lambda: cm.flow_eq2(cam, rho, ego, dt, scale)), 4.0 * hw + nb * 8.0 * hw, hw,
                              "pixels"),
        "flow_eq2_backward_b20": entry(timed(lambda: cm.flow_eq2_backward(cam, rho, ego, dt, scale, g)),
                                       8.0 * hw + nb * 8.0 * hw, hw, "pixels"),
        "geo_forward": entry(timed(geo_f), 8.0 * hw, hw, "pixels"),
        "geo_backward": entry(timed(geo_b), 16.0 * hw, hw, "pixels"),
        "event_frame_2M": entry(timed(lambda: cm.event_frame(cam, ev)), 5.0 * ev.n + 8.0 * hw, ev.n, "events"),
        "bytes_note": "algorithmic: inverse depth read and per-bin flows written (Eq. 2 flow); inverse depth and "
                      "per-bin dL/dflow read, dL/d inverse depth written (its adjoint); both inverse depths read "
                      "(geometry forward), and their gradients written (backward); 5 B per event read and the "
                      "2-channel frame written (event frame)",
    }
    del flush
    return out


def compare_splats(batch, nwin: int):
    """Loss + gradient of the first `nwin` windows through the single-window
    calls with the atomic and with the deterministic sort splat (a stream sync
    after each window), in Mev/s."""
    import torch
    cm = batch.cm
    out = {"windows": nwin, "path": "cm_loss_forward + cm_loss_backward per window"}
    for name, splat in (("atomic", cm.SPLAT_ATOMIC), ("sort", cm.SPLAT_SORT)):
        items = []
        for (w, _, ev, a, b, res, loss) in batch.items[:nwin]:
            cfg = cm.loss_cfg(w.nbins, w.ref_mode, splat)
            items.append((w, cm.Workspace(w.cam, cfg, w.events.n, 1, batch.dev), ev, a, b, res, loss))

        def one(it):
            batch.window_call(it)
            torch.cuda.current_stream().synchronize()

        for it in items:
            one(it)
        t0 = time.perf_counter()
        for _ in range(3):
            for it in items:
                one(it)
        el = (time.perf_counter() - t0) / 3
        out[name] = sum(it[0].events.n for it in items) / el / 1e6
        del items
    out["unit"] = "Mev/s"
    return out


def compare_batched_splats(batch, schedules, reps: int = 5):
    """The batched plan's splat strategies on the same windows: device time of
    `reps` replays (CUDA events) per schedule, in Mev/s.  schedules: name ->
    (chains, windows per kernel, grouping); grouping 3 is the shared-memory
    tile strategy, the others reduce straight into the images."""
    import torch
    out = {}
    for name, sched in schedules.items():
        batch.plan.set_schedule(*sched)
        batch.plan.run()
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            batch.plan.run()
        z.record()
        z.synchronize()
        out[name] = {"schedule": list(sched), "mev_s": batch.events * reps / (a.elapsed_time(z) * 1e-3) / 1e6}
    return out


def compare_deterministic(batch, reps: int = 3):
    """The batched plan in its deterministic mode (CM_SPLAT_SORT: the windows one
    after another through the sort path, the same bits on every run) on the
    same windows: device time of `reps` replays, in Mev/s."""
    import torch
    cm = batch.cm
    w0 = batch.wins[0]
    plan = cm.BatchPlan(batch.dev_wins, cm.loss_cfg(w0.nbins, w0.ref_mode, cm.SPLAT_SORT), batch.dev)
    plan.run()
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        plan.run()
    z.record()
    z.synchronize()
    out = {"schedule": list(plan.schedule()), "mev_s": batch.events * reps / (a.elapsed_time(z) * 1e-3) / 1e6}
    del plan
    torch.cuda.empty_cache()
    return out


def run_e2e(batch, args, stream, schedule):
    """Same metric through the public API with host buffers.  The inputs of all
    windows (events, inverse depth, ego-motion) sit back to back in one pinned
    host arena; two device arenas of the same layout each back a batch plan
    whose outputs live in one device arena (BatchPlan.output_arena).  Step k
    runs plan k % 2 on its inputs while a copy stream brings step k-1's outputs
    (both gradients of every window and the losses) back to pinned host memory
    and copies step k+1's inputs into the other arena, so the copies of every
    step stay in the timed region but overlap the compute of its neighbour."""
    import torch
    cm = batch.cm
    parts = []  # (window index, name, host array)
    for k, w in enumerate(batch.wins):
        for name, a in (("x", w.events.x), ("y", w.events.y), ("t", w.events.t), ("p", w.events.p),
                        ("rho", w.inv_depth), ("ego", w.ego)):
            parts.append((k, name, np.ascontiguousarray(a)))
    offs, total = [], 0
    for _, _, a in parts:
        offs.append(total)
        total += (a.nbytes + 255) // 256 * 256
    host_in = torch.empty(total, dtype=torch.uint8).pin_memory()
    hv = host_in.numpy()
    for (_, _, a), o in zip(parts, offs):
        hv[o:o + a.nbytes] = a.view(np.uint8).ravel()
    dtypes = {"x": torch.int16, "y": torch.int16, "t": torch.float32, "p": torch.int8, "rho": torch.float32,
              "ego": torch.float32}
    cfg = cm.loss_cfg(batch.wins[0].nbins, batch.wins[0].ref_mode, cm.SPLAT_ATOMIC)

    def plan_over(dev_in):
        views = {}
        for (k, name, a), o in zip(parts, offs):
            v = dev_in[o:o + a.nbytes].view(dtypes[name])
            views[(k, name)] = v.view(a.shape) if name == "rho" else v
        windows = []
        for k, w in enumerate(batch.wins):
            ev = cm.DeviceEvents(views[(k, "x")], views[(k, "y")], views[(k, "t")], views[(k, "p")], w.events.t0,
                                 w.events.t1)
            windows.append({"cam": w.cam, "ev": ev, "inv_depth": views[(k, "rho")], "ego": views[(k, "ego")],
                            "dt": w.dt})
        plan = cm.BatchPlan(windows, cfg, batch.dev)
        plan.set_schedule(*schedule)
        return plan

    dev_in = [torch.empty(total, dtype=torch.uint8, device=batch.dev) for _ in range(2)]
    plans = [plan_over(d) for d in dev_in]
    host_out = [torch.empty(plans[0].output_arena.numel(), dtype=torch.float32).pin_memory() for _ in range(2)]
    loss_host = [torch.empty(plans[0].loss.numel()).pin_memory() for _ in range(2)]
    h2d = host_in.numel()
    d2h = host_out[0].numel() * 4 + loss_host[0].numel() * 4
    copy = torch.cuda.Stream(device=batch.dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def run_steps(K, start=None, end=None):
        with torch.cuda.stream(copy):
            if start is not None:
                start.record(copy)
            dev_in[0].copy_(host_in, non_blocking=True)
            ready[0].record(copy)
        for k in range(K):
            b = k % 2
            stream.wait_event(ready[b])
            plans[b].run()
            done[b].record(stream)
            with torch.cuda.stream(copy):
                if k + 1 < K:
                    if k >= 1:
                        copy.wait_event(done[1 - b])  # step k-1 has released the other arena
                    dev_in[1 - b].copy_(host_in, non_blocking=True)
                    ready[1 - b].record(copy)
                copy.wait_event(done[b])
                host_out[b].copy_(plans[b].output_arena, non_blocking=True)
                loss_host[b].copy_(plans[b].loss, non_blocking=True)
        if end is not None:
            end.record(copy)
        torch.cuda.synchronize(batch.dev)

    run_steps(4)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    K = max(4, args.steps)
    run_steps(K, a, z)
    ms = a.elapsed_time(z) / K
    return {"value": batch.events / (ms * 1e-3) / 1e6, "unit": "Mev/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms,
            "pipeline": "1 H2D copy and 2 D2H copies per step on a copy stream, overlapping the neighbouring "
                        "steps' compute (two input arenas, two plans)"}


SERVE_STREAMS = 32


def serve_pools(pool: int):
    """Pre-generated requests of the serving workload: 32 streams (resolutions
    cycling 346x260 / 640x480 / 1280x720), `pool` windows per stream, event
    counts log-uniform in [10k, 2M], 10 bins, in pinned host memory."""
    import torch

    from paper_2412_06359_gb300 import synth
    from paper_2412_06359_gb300.serve import HostRequest

    def pinned(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    pools = []
    for s in range(SERVE_STREAMS):
        rng = synth.rng_for(5, s)
        W, H = synth.SERVE_RESOLUTIONS[s % len(synth.SERVE_RESOLUTIONS)]
        reqs = []
        for _ in range(pool):
            win = synth.depth_window(rng, W, H, synth.log_uniform_count(rng, 1e4, 2e6), nbins=10)
            r = HostRequest.from_window(s, win)
            for f in ("x", "y", "t", "p", "rho", "ego", "loss", "drho", "dego"):
                setattr(r, f, pinned(getattr(r, f)))
            reqs.append(r)
        pools.append(reqs)
    return pools


def serve_arrivals(scale: float, seconds: float, pool: int, seed: int = 77):
    """Poisson arrivals at 100 Hz x scale per stream over `seconds`: sorted
    (time, stream, pool index)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(SERVE_STREAMS):
        t = rng.exponential(1.0 / (100.0 * scale))
        k = 0
        while t < seconds:
            out.append((t, s, k % pool))
            k += 1
            t += rng.exponential(1.0 / (100.0 * scale))
    return sorted(out)


def serve_replay(srv, pools, arr):
    """Submit the arrivals at their times (host clock), wait for all; latency
    of a request = its completion - its submission (the server's clocks)."""
    from paper_2412_06359_gb300 import _capi as C
    # warm up: one request per stream (allocates its state, captures the graphs)
    for s in range(SERVE_STREAMS):
        srv.wait(srv.submit(pools[s][0]), 120)
    t0 = time.perf_counter()
    tickets = []
    for ta, s, k in arr:
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        while True:
            try:
                tickets.append((srv.submit(pools[s][k]), pools[s][k].x.shape[0]))
                break
            except C.CMError as e:
                if e.status != C.CM_EBUSY:
                    raise
                time.sleep(1e-4)
    res = [(srv.wait(t, 600), n) for t, n in tickets]
    lat = np.array([1e3 * (r.t_done - r.t_submit) for r, _ in res])
    first = min(r.t_submit for r, _ in res)
    last = max(r.t_done for r, _ in res)
    ev = sum(n for _, n in res)
    sizes = [r.batch_size for r, _ in res]
    slowest = int(np.argmax(lat))
    return {"requests": len(res), "events": int(ev), "throughput": ev / (last - first) / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat[slowest]), "slowest_submitted_at_s": float(res[slowest][0].t_submit - first),
            "mean_batch": float(np.mean(sizes)), "offered_mev_s": ev / arr[-1][0] / 1e6 if arr else 0.0,
            "stats": {k: int(getattr(srv.stats(), k)) for k in ("batches", "evictions", "memory_waits",
                                                                 "pool_peak")}}


def serve_leg(scales, seconds: float, reps: int, lanes: int, batch: int, group: int, pool: int = 2):
    """The serving workload at each rate scale, `reps` runs each (a fresh
    server per run): Mev/s served and p50 / p99 request latency per run, with
    the p99 spread over the runs.  The lanes group up to `group` events per
    batch by band; one more run at the last scale keeps the given order."""
    from paper_2412_06359_gb300.serve import Server
    pools = serve_pools(pool)
    out = {"workload": "serve32_mixed_res_poisson100hz", "seconds": seconds, "streams": SERVE_STREAMS,
           "lanes": lanes, "max_batch": batch, "hbm_budget_gb": 40, "group_events": group, "runs": reps,
           "unit": "Mev/s", "scales": {}}

    def one(arr, g):
        srv = Server(40 << 30, max_batch=batch, lanes=lanes, group_events=g)
        try:
            return serve_replay(srv, pools, arr)
        finally:
            srv.close()

    arr = None
    for scale in scales:
        arr = serve_arrivals(scale, seconds, pool)
        runs = [one(arr, group) for _ in range(reps)]
        p99 = [r["p99_ms"] for r in runs]
        out["scales"][str(scale)] = {
            "offered_mev_s": runs[0]["offered_mev_s"], "requests": runs[0]["requests"],
            "served_mev_s": [r["throughput"] for r in runs], "p50_ms": [r["p50_ms"] for r in runs],
            "p99_ms": p99, "p99_spread_ms": [min(p99), max(p99)], "mean_batch": [r["mean_batch"] for r in runs],
            "max_ms": [r["max_ms"] for r in runs], "slowest_submitted_at_s": [r["slowest_submitted_at_s"] for r in runs],
            "stats": [r["stats"] for r in runs]}
    if arr is not None and group > 0:
        r = one(arr, 0)
        out["given_order_last_scale"] = {"served_mev_s": r["throughput"], "p50_ms": r["p50_ms"],
                                         "p99_ms": r["p99_ms"]}
    return out


def run_serve(args):
    """Serving workload: 32 streams (resolutions cycling 346x260 / 640x480 /
    1280x720), Poisson arrivals at 100 Hz per stream scaled by --serve-scales,
    event counts log-uniform in [10k, 2M], 10 bins, loss + gradient per request,
    a 40 GB HBM budget.  Every stream cycles through --serve-pool pre-generated
    windows held in pinned host memory.  Prints one JSON line per scale, plus the
    plain path (one request at a time, no batching) on the same arrivals."""
    import torch

    from paper_2412_06359_gb300 import _capi as C
    from paper_2412_06359_gb300 import build
    from paper_2412_06359_gb300.serve import Server
    build.build()
    C.lib()
    torch.cuda.init()
    pools = serve_pools(args.serve_pool)
    budget = 40 << 30
    for scale in [float(x) for x in args.serve_scales.split(",")]:
        arr = serve_arrivals(scale, args.serve_seconds, args.serve_pool)
        srv = Server(budget, max_batch=args.serve_batch, lanes=args.serve_lanes, group_events=args.serve_group)
        batched = serve_replay(srv, pools, arr)
        srv.close()
        plain = None
        if not args.no_plain:
            srv = Server(budget, max_batch=1, lanes=1)
            plain = serve_replay(srv, pools, arr)
            srv.close()
        line = {"metric": "serving: CM loss+grad Mev/s and p50/p99 request latency", "unit": "Mev/s",
                "value": batched["throughput"], "p50_ms": batched["p50_ms"], "p99_ms": batched["p99_ms"],
                "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "serve32_mixed_res_poisson100hz", "rate_scale": scale,
                           "seconds": args.serve_seconds, "streams": SERVE_STREAMS,
                           "pool_per_stream": args.serve_pool, "max_batch": args.serve_batch,
                           "lanes": args.serve_lanes, "hbm_budget_gb": 40, "group_events": args.serve_group},
                "batched": batched, "plain": plain}
        print(json.dumps(line), flush=True)


def run_latency(args):
    """One JSON line: loss + gradient latency of one window of each parity
    workload, through the single-window calls (a stream sync after each call,
    as a per-window caller would) and through a one-window batched plan
    (autotuned, replayed from its CUDA graph, synced after each run); p50/p99
    over --reps calls after 10 warm-up calls, host clock."""
    import torch
    from paper_2412_06359_gb300 import _capi as C
    from paper_2412_06359_gb300 import build, synth
    build.build()
    C.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)

    def lat(fn):
        for _ in range(10):
            fn()
        t = []
        for _ in range(args.reps):
            s = time.perf_counter()
            fn()
            t.append(1e3 * (time.perf_counter() - s))
        return float(np.percentile(t, 50)), float(np.percentile(t, 99))

    out = {}
    for name, win in (("flow_128x128_b1_end", synth.flow_window()), ("depth_346x260_b10_all", synth.davis_window()),
                      ("depth_1280x720_b20_all", synth.hd_window())):
        b = Batch([win], dev)
        b.plan.autotune()

        def plan_run():
            b.plan.run()
            torch.cuda.current_stream(dev).synchronize()

        n = win.events.n
        p50, p99 = lat(lambda: b.plain_window(0))
        q50, q99 = lat(plan_run)
        out[name] = {"events": n, "plain": {"p50_ms": p50, "p99_ms": p99, "mev_s_at_p50": n / p50 / 1e3},
                     "plan": {"p50_ms": q50, "p99_ms": q99, "mev_s_at_p50": n / q50 / 1e3,
                              "schedule": list(b.plan.schedule())}}
        del b
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "single-window loss+grad latency", "unit": "ms", "reps": args.reps,
                      "higher_is_better": False, "data": "synthetic", "latency": out}), flush=True)


def run_other(args):
    """One JSON line: the kernels beside the CM path on a 1280x720 sensor."""
    import torch
    dev = torch.device("cuda", 0)
    peak, kind = measured_peak()
    out = measure_other_kernels(dev, peak)
    print(json.dumps({"other_kernels": out, "peak_kind": kind}), flush=True)


def main():
    args = parse()
    if args.serve:
        run_serve(args)
    elif args.other_kernels:
        run_other(args)
    elif args.latency:
        run_latency(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
