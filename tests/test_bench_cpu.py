"""bench.py's host-side pieces: the byte model of the roofline fields and the
recorded ncu counters it reads (they must belong to the kernel sources as they
are, or roofline.traffic and roofline_l2 come out null)."""
import bench


def test_recorded_counters_belong_to_the_current_kernel_sources():
    for k in ("k_splat_batch", "k_adjoint_batch"):
        c = bench.recorded_counters(k)
        assert c is not None, (f"the recorded ncu counters do not match the kernel sources (hash "
                               f"{bench.kernel_source_hash()}): re-take them on a GPU")
        assert c["l2_read_requests_per_event"] > 0 and c["l2_red_requests_per_event"] > 0
        assert c["dram_bytes_per_event"] > 9.0  # at least the event's own bytes


def test_strict_byte_model():
    n, hw, R = 1000, 640 * 480, 11
    assert bench.kernel_bytes("k_splat_batch", n, hw, R, "strict") == 9.0 * n
    assert bench.kernel_bytes("k_adjoint_batch", n, hw, R, "strict") == 9.0 * n
    assert bench.kernel_bytes("k_prep_batch", n, hw, R, "strict") == 4.0 * hw
    assert bench.kernel_bytes("k_grad_batch", n, hw, R, "strict") == 4.0 * hw
    assert bench.kernel_bytes("k_loss_batch", n, hw, R, "strict") == 0.0
    # the materialised-image model adds the dense image traffic
    assert bench.kernel_bytes("k_loss_batch", n, hw, R, "iwe") == 16.0 * R * hw
    assert bench.kernel_bytes("k_splat_batch", n, hw, R, "iwe") == 9.0 * n + 16.0 * R * hw


def test_grouping_names_cover_every_schedule_mode():
    assert len(bench.GROUPING) == 4 and bench.GROUPING[2] == "32-row bands"


def test_oracle_on_every_core_covers_the_windows_once():
    # two windows of the batch workload on two spawned processes
    from paper_2412_06359_gb300 import synth
    sizes = [w.events.n for w in synth.batch_windows(2)]
    r = bench.oracle_all_cores(sizes, False, limit_s=120.0)
    assert r is not None
    ev, sec, nproc = r
    assert ev == sum(sizes) and sec > 0 and nproc == 2
