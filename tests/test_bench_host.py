"""Single-process host logic of bench.py on CPU: the figures it takes from the
committed profile summaries (only while the profiled sources are unchanged),
the executed lane-op rate, the algorithmic placement count behind the
roofline, and the percentile and win-count helpers of the surrogate leg."""


def test_traffic_figure_only_for_unchanged_kernel_sources(tmp_path, monkeypatch):
    """The benchmark reports a profile's DRAM bytes and counters only while
    the profiled kernel's sources are the ones the summary names."""
    import bench
    prof = tmp_path / "profiles"
    csrc = tmp_path / "paper_1511_07983_gb300" / "csrc"
    prof.mkdir()
    csrc.mkdir(parents=True)
    names = bench.KERNEL_SOURCES["lane_kernel"]
    for i, f in enumerate(names):
        (csrc / f).write_text(f"source {i}")
    import hashlib
    good = hashlib.sha256(b"".join(f"source {i}".encode() for i in range(len(names)))).hexdigest()
    (prof / "lane_kernel_w_dram.md").write_text(
        "x\n- bytes_per_launch: 1234\n- source sha256: " + good + "\n")
    (prof / "lane_kernel_w_counters.md").write_text(
        "- case: n11\n- issue_active_pct: 40.1\n- threads_per_inst: 7.77\n- source sha256: " + good + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("lane_kernel", "w") == 1234
    assert bench.measured_counters("lane_kernel", "w") == {"case": "n11", "issue_active_pct": 40.1,
                                                           "threads_per_inst": 7.77}
    assert bench.measured_traffic("lane_kernel", "other") is None
    assert bench.measured_traffic("fast_kernel", "w") is None
    (csrc / names[0]).write_text("changed")
    assert bench.measured_traffic("lane_kernel", "w") is None
    assert bench.measured_counters("lane_kernel", "w") is None


def test_executed_lane_ops_from_counters():
    import bench
    c = {"case": "n11", "warp_inst_per_order": 4000, "threads_per_inst": 8.0}
    r = bench.executed_lane_ops(c, orders=1_000_000, kernel_s=2.0, peak_gops=32.0)
    assert r["per_order"] == 32000.0
    assert r["achieved"] == 16.0 and r["frac"] == 0.5
    assert bench.executed_lane_ops(None, 1, 1.0, 1.0) is None
    assert bench.executed_lane_ops({"threads_per_inst": 8.0}, 1, 1.0, 1.0) is None


def test_algorithmic_placement_count_against_the_prefix_tree():
    # the roofline's work unit: every distinct prefix places its last kernel's blocks once
    import itertools
    import bench
    for n, blocks in ((1, [7]), (3, [1, 2, 3]), (5, [5, 1, 9, 2, 4])):
        kernels = [[0, 0, 0, b, 0, 0] for b in blocks]
        brute = sum(blocks[p[-1]] for d in range(1, n + 1) for p in itertools.permutations(range(n), d))
        assert bench.placements_per_exhaustive(kernels) == brute


def test_percentile_and_wins_helpers():
    import numpy as np
    import bench
    ref = np.array([5, 6, 7, 8])
    assert bench.percentile_of(6, ref) == 75.0 and bench.percentile_of(9, ref) == 0.0
    w = bench.wins([1, 5, 3], [2, 5, 2])
    assert (w["lower"], w["equal"], w["higher"]) == (1, 1, 1)
    assert abs(w["mean_gain"] - ((2 - 1) / 2 + 0 + (2 - 3) / 2) / 3) < 1e-12
