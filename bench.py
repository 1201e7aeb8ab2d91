#!/usr/bin/env python
"""Benchmark: exact launch orders scored per second on the N=12 / 148-SM set.

One step = the whole hot path through the public C ABI (ko_rank_order):
Algorithm 1 order on the host, its makespan on the device, the makespan of all
12! = 479,001,600 orders (one-thread-per-order simulator; the run-length
and simple simulators re-run the work items it cannot hold),
min / max / better / equal / worse against the heuristic, and the 4096-bin
histogram.  Inputs are seeded synthetic kernel sets (no dataset exists).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` times K steps with the histogram kept in device memory (CUDA events on
the launching stream, barrier + synchronize on both sides, max over ranks).
`e2e` times the same call with host output buffers (device->host copies of the
histogram and results inside the timed region).  `--impl reference` times the
CPU oracle on this machine's cores on a bounded sample of the same workload.
Multi-GPU runs are independent replicas (one per rank): every rank scores the
whole space; only a barrier and the maximum of the per-rank times cross ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "single12"
NBINS = 4096
OPS_PER_PLACEMENT = 27   # fit test 8, usage 4, SumC/SumM 2, duration 7, release 6 (integer ops)
METRIC = "exact orders evaluated/s at N=12; best percentile: surrogate vs plain at equal time"


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--lanes", type=int, default=None)
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--n", type=int, default=None,
                    help="use only the first n kernels of the set (small profiling cases)")
    ap.add_argument("--cpu-sample", type=int, default=300000,
                    help="orders in the oracle's bounded CPU sample")
    ap.add_argument("--surrogate", type=int, default=1,
                    help="1: also run the surrogate-vs-plain comparison (outside the timed region)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick lanes / DFS depth with ko_autotune before warm-up")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(seconds: float, dist) -> float:
    """Slowest rank's time (a gloo all-reduce of one float; no data path)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(orders_per_replica: int, steps: int, world: int, seconds: float) -> float:
    """Orders all ranks scored divided by the slowest rank's time (replicas)."""
    return orders_per_replica * steps * world / seconds


def placements_per_exhaustive(kernels) -> int:
    """Block placements of an exhaustive lexicographic DFS with prefix sharing:
    every prefix of length d pays for its last kernel's blocks; each kernel is
    the last of (N-1)!/(N-d)! prefixes of length d."""
    n = len(kernels)
    total_blocks = int(sum(int(k[3]) for k in kernels))
    return sum(math.factorial(n - 1) // math.factorial(n - d) for d in range(1, n + 1)) * total_blocks


KERNEL_SOURCES = {"lane_kernel": ("ko_lane.cu", "ko_lane_sim.cuh", "ko_fast.cu", "ko_fast.h"),
                  "fast_kernel": ("ko_fast.cu", "ko_fast.h")}


def source_hash(kernel):
    """SHA-256 of the sources of a simulator kernel (the profile summaries
    record it; a changed kernel invalidates their counters)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1511_07983_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_fields(kernel, workload, kind):
    """`- key: value` lines of the committed ncu summary
    profiles/<kernel>_<workload>_<kind>.md, or None when there is none or the
    kernel's sources changed since its counters were taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}_{kind}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    mh = re.search(r"^- source sha256: ([0-9a-f]{64})$", text, re.M)
    if not mh or mh.group(1) != source_hash(kernel):
        return None
    out = {}
    for m in re.finditer(r"^- ([a-z_0-9]+): (.+)$", text, re.M):
        key, v = m.group(1), m.group(2).strip()
        if key == "source":
            continue
        try:
            out[key] = int(v) if re.fullmatch(r"-?\d+", v) else float(v)
        except ValueError:
            out[key] = v
    return out


def measured_traffic(kernel, workload):
    """DRAM bytes per full launch of the dominant kernel (read + write, from
    an ncu capture, scaled to the workload as its summary states), or None."""
    f = profile_fields(kernel, workload, "dram")
    return int(f["bytes_per_launch"]) if f and "bytes_per_launch" in f else None


def measured_counters(kernel, workload):
    """Issue-slot use, active threads per instruction and warp instructions
    per order of the dominant kernel from its committed ncu summary, or None."""
    f = profile_fields(kernel, workload, "counters")
    if not f:
        return None
    return {k: f[k] for k in ("case", "issue_active_pct", "threads_per_inst", "warp_inst_per_order") if k in f}


def executed_lane_ops(counters, orders, kernel_s, peak_gops):
    """Integer lane-ops the dominant kernel executes, from its ncu counters
    (warp instructions per order x active threads per instruction), as a rate
    over the measured kernel time and as a fraction of the measured integer
    peak; None without counters."""
    if not counters or "warp_inst_per_order" not in counters or "threads_per_inst" not in counters:
        return None
    per_order = counters["warp_inst_per_order"] * counters["threads_per_inst"]
    gops = per_order * orders / kernel_s / 1e9
    return {"per_order": per_order, "achieved": gops, "frac": gops / peak_gops,
            "from": f"ncu counters ({counters.get('case', '?')}): warp instructions per order x "
                    f"threads per instruction"}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(kset, sample: int, seed: int = 12):
    """Oracle (plain C, pthreads over index ranges) on this host's cores, on a
    seeded sample of Lehmer indices of the same set."""
    import oracle
    from paper_1511_07983_gb300 import synth
    cores = os.cpu_count() or 1
    ids = synth.random_indices(seed, math.factorial(kset.n), sample)
    oracle.lib()
    t0 = time.perf_counter()
    oracle.makespans_idx(kset.gpu, kset.kernels, idx=ids, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": "orders/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample} seeded uniform Lehmer indices of the {kset.n}-kernel set "
                      f"({dt:.1f} s of CPU work), rate extrapolated to the full space"}


def load_set(a):
    from paper_1511_07983_gb300 import synth
    kset = synth.gen_set(a.workload)
    if a.n is not None:
        kset = synth.KernelSet(gpu=kset.gpu, kernels=kset.kernels[:a.n].copy())
    return kset


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    kset = load_set(a)
    for _ in range(a.warmup):
        cpu_baseline(kset, max(1000, a.cpu_sample // 20), seed=1)
    times, vals = [], []
    for k in range(a.steps):
        cb = cpu_baseline(kset, a.cpu_sample, seed=100 + k)
        vals.append(cb["value"])
        times.append(a.cpu_sample / cb["value"])
    value = a.cpu_sample * a.steps / sum(times)
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "orders/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * sum(times) / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"{a.workload}: N={kset.n} launch orders, 148-SM simulated GPU, "
                                   f"blocks/kernel U[100,1000]; bounded sample of "
                                   f"{a.cpu_sample} orders per step on host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "orders/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(a):
    import numpy as np
    import torch

    from paper_1511_07983_gb300 import build, ko, synth

    rank, world, local = dist_env()
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")   # barrier and max of the times only; no data path

    def barrier():
        if dist:
            dist.barrier()

    kset = load_set(a)
    n_orders = math.factorial(kset.n)
    g = ko.Gpu.from_set(kset)
    tune = None
    if a.lanes or a.levels is not None:
        g.configure(lanes=a.lanes, levels=a.levels)
    elif a.autotune:
        t0 = time.perf_counter()
        choice = g.autotune(os.path.join(ROOT, "paper_1511_07983_gb300", "ko_tune_cache.json"))
        tune = {"lanes": choice["lanes"], "levels": choice["levels"], "lane_state": choice["lane_state"],
                "seconds": round(time.perf_counter() - t0, 2)}
    stream = torch.cuda.current_stream()
    d_hist = torch.zeros(NBINS, dtype=torch.int64, device="cuda")   # uint64 bits
    h_hist = np.zeros(NBINS, dtype=np.uint64)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step(host: bool):
        flush.fill_(1)
        r, _ = g.rank_order(None, nbins=NBINS, hist=h_hist if host else d_hist, stream=stream)
        return r

    for _ in range(a.warmup):
        r = step(False)
    torch.cuda.synchronize()

    # device-resident timing
    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ko.ko_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sim_ms, fallback = [], []
    e0.record(stream)
    for _ in range(a.steps):
        r = step(False)
        sim_ms.append(g.last_sim_ms())
        fallback.append(g.last_fallback_items())
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ko.ko_kernel_launches() - launches0
    barrier()
    elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist)

    # end-to-end through the same call with host buffers
    h2d0, d2h0 = g.transfer_bytes()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step(True)
    torch.cuda.synchronize()
    e2e_elapsed = max_over_ranks(time.perf_counter() - t0, dist)
    h2d1, d2h1 = g.transfer_bytes()

    if rank != 0:
        g.close()
        if dist:
            dist.destroy_process_group()
        return 0

    value = whole_job_rate(n_orders, a.steps, world, elapsed)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    issue_gops = sm_count * 4 * 32 * max_mhz * 1e6 / 1e9   # every issue slot a full-warp integer op
    # measured integer peak: add / xor / min chains on every SM (ko_hw_int_peak), clocks sampled
    iclk = Clocks(local)
    iclk.start()
    int_ops, int_ms = ko.ko_hw_int_peak(16384)
    iclk_stats = iclk.stop()
    peak_gops = int_ops / int_ms / 1e6
    placements = placements_per_exhaustive(kset.kernels.tolist())
    kernel_s = statistics.mean(sim_ms) / 1e3
    achieved = placements * OPS_PER_PLACEMENT / kernel_s / 1e9
    kernel = "lane_kernel" if ko.ko_get_option(g.h, ko.KO_OPT_LANES) == 1 else "fast_kernel"
    traffic = measured_traffic(kernel, a.workload)
    counters = measured_counters(kernel, a.workload)
    cb = cpu_baseline(kset, a.cpu_sample) if world == 1 else None
    sur = None
    if a.surrogate and world == 1:
        try:
            sur = surrogate_experiment()
        except Exception as exc:  # reported, never fatal to the bench line
            sur = {"error": f"{type(exc).__name__}: {exc}"}
    line = {
        "metric": METRIC, "value": value, "unit": "orders/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * elapsed / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"{a.workload}: all {n_orders} launch orders of N={kset.n} kernels "
                               f"on a {kset.gpu[0]}-SM simulated GPU (65536 regs, 228 KB smem, "
                               f"64 warps, 32 blocks/SM), blocks/kernel U[100,1000], 4096-bin "
                               f"histogram + heuristic rank",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "256 MB flush before every step; the 3.8 GB makespan buffer exceeds L2",
                   "lanes": ko.ko_get_option(g.h, ko.KO_OPT_LANES),
                   "levels": ko.ko_get_option(g.h, ko.KO_OPT_LEVELS),
                   "lane_state": ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE), "autotune": tune},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_gops, "unit": "Gop/s",
                     "frac": achieved / peak_gops, "traffic": traffic,
                     "kernel": kernel, "kernel_ms": kernel_s * 1e3,
                     "placements_per_launch": placements, "ops_per_placement": OPS_PER_PLACEMENT,
                     "peak_from": f"measured: ko_hw_int_peak, {int_ops} 32-bit add/xor/min lane-ops "
                                  f"in {int_ms:.3f} ms on {sm_count} SMs",
                     "peak_clocks": iclk_stats,
                     "issue_peak": issue_gops,
                     "issue_peak_from": f"{sm_count} SMs x 4 schedulers x 32 lanes x {max_mhz:.0f} MHz",
                     "ncu": counters,
                     "ncu_lane_ops": executed_lane_ops(counters, n_orders, kernel_s, peak_gops)},
        "cpu_baseline": cb,
        "e2e": {"value": whole_job_rate(n_orders, a.steps, world, e2e_elapsed), "unit": "orders/s",
                "h2d_bytes_per_step": (h2d1 - h2d0) // a.steps,
                "d2h_bytes_per_step": (d2h1 - d2h0) // a.steps},
        "gpu_launches": launches,
        "clocks": clk,
        "fallback_items_per_step": max(fallback) if fallback else 0,
        "surrogate": sur,
        "heuristic": {"makespan": r["makespan"], "percentile": r["percentile"],
                      "min": r["min"], "max": r["max"]},
    }
    print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.destroy_process_group()
    return 0


def percentile_of(best, ref):
    """Share (%) of the reference orders at least as slow as `best`."""
    import numpy as np
    return 100.0 * float(np.count_nonzero(ref >= best)) / ref.size


def train_surrogate(kind, seed=7, train_sets=1221, pairs=8192, steps=2500, batch=4096):
    """Train the MLP on exactly simulated uniform orders: kind "small" uses
    only enumerable sets (N 6..12, as the scope specifies), "mixed" half of
    them and half N 16..24 sets (disjoint seeds from the test sets), kind
    "untrained" returns the initial weights (the search's control)."""
    from paper_1511_07983_gb300 import ko, synth
    model = ko.Model(seed=seed)
    if kind == "untrained":
        return model, {"kind": kind}
    if kind == "small":
        sets = [synth.gen_set("train", 1000 + i) for i in range(train_sets)]
    else:
        half = train_sets // 2
        sets = [synth.gen_set("train", 1000 + i) for i in range(train_sets - half)]
        sets += [synth.gen_set("large", 1000 + i) for i in range(half)]
    gpus = [ko.Gpu.from_set(k) for k in sets]
    t0 = time.perf_counter()
    curve = model.train(gpus, pairs_per_set=pairs, steps=steps, batch=batch, lr=1e-3, seed=seed)
    train_s = time.perf_counter() - t0
    for g in gpus:
        g.close()
    return model, {"kind": kind, "train_sets": len(sets), "train_n": f"{min(k.n for k in sets)}..{max(k.n for k in sets)}",
                   "train_pairs": len(sets) * pairs, "train_steps": steps, "batch": batch,
                   "train_s": round(train_s, 2), "final_loss": float(curve[-50:].mean())}


def surrogate_experiment(seed=7, test_sets=32, n_cand=1 << 18, top_k=1024, rounds=6, beam=8, polish=64,
                         ref_orders=1 << 20):
    """The learned part on sets too large to enumerate (N 16..24), every
    reported makespan exact.  For each network -- trained on N <= 12 sets only
    (the specified transfer), trained with N <= 24 labels (the variant for a
    model that does not transfer), and untrained (control) -- on each of
    test_sets held-out sets:
      * screening at equal exact budgets: the best of the network's top_k out
        of n_cand random candidates vs the best of top_k uniform orders;
      * guided search (ko_surrogate_search: screening, then `rounds` rounds of
        network-ranked neighbours around a beam of the best exact orders) vs
        plain uniform random search given the same measured GPU time, without
        and with the exact steepest-descent polish (KO_MODEL_OPT_POLISH);
    wins are counted on exact makespans.  Exact local search from Algorithm
    1's order (no model, its own time) and ranks against ref_orders seeded
    uniform orders are reported beside them."""
    import numpy as np
    from paper_1511_07983_gb300 import ko, synth
    tests = [synth.gen_set("large", j) for j in range(test_sets)]
    rng = np.random.default_rng(seed)
    base = []
    for j, ks in enumerate(tests):
        with ko.Gpu.from_set(ks) as g:
            ref_rows = np.argsort(rng.random((ref_orders, ks.n)), axis=1).astype(np.int8)
            ref = g.eval_orders(orders=ref_rows)
            h_ms = int(g.eval_orders(orders=np.array([g.heuristic_order()], dtype=np.int8))[0])
            _, l_best, _, l_orders, l_ms = g.local_search(moves=True)
            _, r_best, _ = ko.ko_random_search(g, top_k, seed=seed + 200 + j)
            _, _, cal_ms = ko.ko_random_search(g, 1 << 16, seed=99 + j)
        base.append({"n": ks.n, "n_sm": ks.gpu[0], "ref": ref, "heuristic": h_ms, "local_search": int(l_best),
                     "local_search_ms": l_ms, "random_budget": int(r_best), "cal_ms": cal_ms})
    out = {"test_sets": test_sets, "candidates": n_cand, "top_k": top_k, "rounds": rounds, "beam": beam,
           "polish_steps": polish, "reference_orders": ref_orders,
           "heuristic_percentile_mean": float(np.mean([percentile_of(b["heuristic"], b["ref"]) for b in base])),
           "local_search_percentile_mean": float(np.mean([percentile_of(b["local_search"], b["ref"]) for b in base])),
           "local_search_ms_mean": float(np.mean([b["local_search_ms"] for b in base]))}
    for kind in ("small", "mixed", "untrained"):
        model, info = train_surrogate(kind, seed=seed)
        res = dict(info)
        if kind != "untrained":
            scr = []
            for j, ks in enumerate(tests):
                with ko.Gpu.from_set(ks) as g:
                    _, sb, _ = model.propose(g, n_cand=1 << 20, top_k=top_k, seed=seed + j)
                scr.append(int(sb))
            res["screening_vs_random_at_equal_exact_budget"] = wins(scr, [b["random_budget"] for b in base])
        for pol in (0, polish):
            model.set_polish(pol)
            guided, plain, pcts = [], [], []
            for j, ks in enumerate(tests):
                with ko.Gpu.from_set(ks) as g:
                    _, sb, s_ms = model.search(g, n_cand=n_cand, top_k=top_k, rounds=rounds, beam=beam, seed=seed + j)
                    n_plain = max(1, int((1 << 16) * s_ms / max(base[j]["cal_ms"], 1e-3)))
                    _, pb, _ = ko.ko_random_search(g, n_plain, seed=seed + 100 + j)
                guided.append(int(sb))
                plain.append(int(pb))
                pcts.append((percentile_of(sb, base[j]["ref"]), percentile_of(pb, base[j]["ref"])))
            key = "guided" if pol == 0 else "guided_polished"
            res[key + "_vs_plain_at_equal_gpu_time"] = wins(guided, plain)
            res[key + "_vs_local_search"] = wins(guided, [b["local_search"] for b in base])
            res[key + "_percentile_mean"] = float(np.mean([p[0] for p in pcts]))
            res[key + "_plain_percentile_mean"] = float(np.mean([p[1] for p in pcts]))
        model.close()
        out[kind] = res
    return out


def wins(a, b):
    """Exact-makespan comparison of two lists of best makespans (lower wins)."""
    return {"lower": sum(x < y for x, y in zip(a, b)), "equal": sum(x == y for x, y in zip(a, b)),
            "higher": sum(x > y for x, y in zip(a, b)),
            "mean_gain": sum((y - x) / y for x, y in zip(a, b)) / len(a)}


BATCH_WORKLOADS = {"single8": (1, NBINS), "sets10": (64, NBINS), "batched": (4096, 0)}


def run_batch(a):
    """Batched workloads: the 64 ten-kernel sets on a 15-SM GPU with 4096-bin
    histograms, the 4096 mixed sets (N 5..10 on 13/15/148-SM GPUs) with
    per-set min / max / rank, or the one eight-kernel set on a 13-SM GPU
    (40,320 orders, 4096-bin histogram; launch-latency-bound, run it with
    --steps 100); one step = one replay of the batch's captured graph (every
    order of every set), timed with CUDA events."""
    import torch

    from paper_1511_07983_gb300 import build, ko, synth
    build.build()
    torch.cuda.set_device(0)
    nsets, nbins = BATCH_WORKLOADS[a.workload]
    sets = [synth.gen_set(a.workload, i) for i in range(nsets)]
    gpus = [ko.Gpu.from_set(s) for s in sets]
    tune = None
    if a.lanes or a.levels is not None:
        for g in gpus:
            g.configure(lanes=a.lanes, levels=a.levels)
    elif a.autotune:
        t0 = time.perf_counter()
        cache = os.path.join(ROOT, "paper_1511_07983_gb300", "ko_tune_cache.json")
        if nsets == 1:
            gpus[0].autotune(cache)   # one set: timed on its own space, as the step runs it
        else:
            ko.ko_batch_autotune(gpus, cache)
        choices = sorted({(ko.ko_get_option(g.h, ko.KO_OPT_LANES), ko.ko_get_option(g.h, ko.KO_OPT_LEVELS),
                           ko.ko_get_option(g.h, ko.KO_OPT_STACK_GLOBAL), ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE))
                          for g in gpus})
        tune = {"seconds": round(time.perf_counter() - t0, 2),
                "choices (lanes, levels, global slab, lane state)": [list(c) for c in choices]}
    t0 = time.perf_counter()
    b = ko.Batch(gpus, nbins=nbins)
    build_s = time.perf_counter() - t0
    orders = b.orders()
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        b.run(stream=stream)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    launches0 = ko.ko_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        res, _ = b.run(stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1e3
    line = {"metric": "exact orders evaluated/s, batched", "value": orders * a.steps / elapsed,
            "unit": "orders/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * elapsed / a.steps, "higher_is_better": True, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": f"{a.workload}: {nsets} sets, {orders} orders per step, "
                                   f"{'4096-bin histograms' if nbins else 'per-set min/max/rank'}, "
                                   f"one captured graph", "autotune": tune,
                       "graph_build_s": round(build_s, 2)},
            "gpu_launches": ko.ko_kernel_launches() - launches0, "clocks": clk,
            "fallback_items": b.fallback_items(),
            "heuristic_percentile_mean": sum(r["percentile"] for r in res) / len(res)}
    print(json.dumps(line), flush=True)
    b.close()
    for g in gpus:
        g.close()
    return 0


def main():
    a = args_parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload in BATCH_WORKLOADS:
        return run_batch(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
