"""Multi-rank host logic of bench.py on CPU: world_size 2 over gloo (no GPU).
bench.py runs one independent replica per rank; only the barrier and the max
of the per-rank times cross ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    slowest = bench.max_over_ranks(1.5 + rank, dist)     # rank 1 is the slow one
    q.put((rank, slowest, bench.whole_job_rate(1000, 2, world, slowest), bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, env in out:
        assert slowest == 2.5
        assert rate == pytest.approx(1000 * 2 * 2 / 2.5)
        assert env == (rank, 2, rank)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""


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


def test_reference_arm_line_on_rank0(monkeypatch, capsys):
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                                     "--cpu-sample", "2000"])
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    assert line["metric"] == bench.METRIC and line["unit"] == "orders/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0


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
