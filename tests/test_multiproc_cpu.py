"""The several-GPU path of bench.py, on CPU with gloo (world size 2): ranks
evaluate disjoint windows (replicas, weak scaling), the timing reduction takes
the maximum and the event count the sum, and the reference arm under torchrun
prints exactly one line (rank 0) while the other rank exits cleanly."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    first = bench.first_window_of(rank, 64)
    t, e = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), torch.device("cpu"))
    out[rank] = (first, t, e)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_sharding_and_timing_reduction():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    (f0, t0, e0), (f1, t1, e1) = out[0], out[1]
    assert (f0, f1) == (0, 64)               # disjoint windows
    assert t0 == t1 == 11.0                  # max over ranks
    assert e0 == e1 == 3000                  # sum over ranks


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--windows", "1"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mev/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
