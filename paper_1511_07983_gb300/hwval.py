"""Does the dispatch model rank launch orders the way this GPU does?

Sec. 6 evaluates a launch order by running it on the hardware.  Here the same
is done for sets of synthetic busy kernels (FMA-chain kernels of chosen block
size, shared memory, grid and length, see ko_hw_create), every one of the N!
orders timed on this GPU, and the times compared with the makespans the
simulator gives for a descriptor of the same GPU:

* GPU: N_SM, registers, shared memory, warps and resident blocks per SM as the
  device reports them;
* kernel i: registers per block = warps x (registers per thread x 32 rounded
  up to 256, the per-warp allocation unit), shared memory per block = the
  reserved amount + the dynamic amount, warps = threads / 32, N_tblk = grid;
* the time of one block of kernel i running alone, in nanoseconds, is c_i for
  a compute kernel (m_i = c_i / 100) and m_i for a memory kernel (c_i =
  m_i / 100), so R_i is 100 or 1/100;
* Ccap and Mcap: either unbounded (durations are the alone times: the model is
  then pure packing under the four SM limits and head-of-line blocking) or
  calibrated from how much slower k co-resident blocks of the set's first
  compute (memory) kernel run than one (T(k) / T(1) = max(1, k c / Ccap)
  under the duration rule).

Sets are all compute kernels, or (--mixed) alternate compute and memory
kernels so that the compute/memory balance of Sec. 4 matters.

For each set the report gives Spearman's rank correlation between measured
time and simulated makespan over all orders, the measured spread (worst /
best), where the simulator's best order and Algorithm 1's order land among
the measured times, and, from per-block traces of two orders, how often the
hardware starts a block of a later-issued kernel before the earlier kernel's
last block (the model's first-in-first-out premise, Sec. 2).

    python -m paper_1511_07983_gb300.hwval [--sets 8] [--n 6] [--mixed] [--json out.json]
"""
from __future__ import annotations

import argparse
import itertools
import json
import math
import time

import numpy as np

from . import ko
from .synth import SplitMix64, _mix

REG_UNIT = 256  # registers are allocated per warp in units of 256
CAP_MAX = 1 << 30  # largest capacity the simulator takes; above 32 x the longest block it never binds


def rankdata(x) -> np.ndarray:
    """Ranks 1..n, ties given the mean of the ranks they span."""
    _, inv, cnt = np.unique(np.asarray(x), return_inverse=True, return_counts=True)
    last = np.cumsum(cnt).astype(np.float64)
    return ((last - cnt + 1.0 + last) / 2.0)[inv.reshape(-1)]


def spearman(a, b) -> float:
    """Pearson correlation of the two rank vectors."""
    ra, rb = rankdata(a), rankdata(b)
    ra -= ra.mean()
    rb -= rb.mean()
    den = math.sqrt(float((ra * ra).sum()) * float((rb * rb).sum()))
    return float((ra * rb).sum() / den) if den > 0 else float("nan")


def draw_set(seed: int, n: int, n_sm: int, max_smem: int, mixed: bool = False) -> list[tuple]:
    """n busy-kernel shapes (kind, threads, smem, blocks, target alone time in us).
    Without `mixed` every kernel is an FMA chain; with it the kinds alternate
    compute / memory from a seeded start, so both are present."""
    rng = SplitMix64(_mix((0x4D580000 if mixed else 0x48570000) + seed))
    first = rng.uniform_int(0, 1) if mixed else 0
    out = []
    for i in range(n):
        kind = (first + i) % 2 if mixed else ko.KO_HW_COMPUTE
        threads = rng.choice([64, 128, 256, 512])
        smem = rng.choice([0, 8 << 10, 24 << 10, 48 << 10, 96 << 10, 160 << 10])
        smem = min(smem, max_smem)
        blocks = rng.uniform_int(n_sm // 2, 4 * n_sm)
        us = rng.uniform_int(20, 200)
        out.append((kind, threads, smem, blocks, us))
    return out


def dispatch_order_stats(rec: np.ndarray, order) -> dict:
    """How far one traced run departs from the model's dispatch premise (Sec. 2:
    every block of an earlier-issued kernel is dispatched before any block of a
    later one).  rec: [blocks, 4] records (start ns, end ns, SM, kernel id).

    * overtaken: fraction of blocks, over kernels issued second and later,
      that started before the last block of the kernel issued just before;
    * inversions: fraction of block pairs from different kernels whose start
      times are in the opposite order of their kernels' issue positions;
    * first_start_us: each kernel's first block start after the run's first,
      in issue order."""
    t0 = rec[:, 0].astype(np.int64)
    kid = rec[:, 3].astype(np.int64)
    base = int(t0.min())
    starts = [np.sort(t0[kid == k]) for k in order]
    later = sum(len(x) for x in starts[1:])
    overtaken = sum(int((starts[j] < starts[j - 1][-1]).sum()) for j in range(1, len(order)))
    inv = pairs = 0
    for i in range(len(order)):
        for j in range(i + 1, len(order)):
            # pairs (a of position i, b of position j) with b starting strictly before a
            inv += int(np.searchsorted(starts[j], starts[i], side="left").sum())
            pairs += len(starts[i]) * len(starts[j])
    return {"overtaken": overtaken / later if later else 0.0, "inversions": inv / pairs if pairs else 0.0,
            "first_start_us": [round((int(x[0]) - base) / 1e3, 3) for x in starts]}


def model_kernel(threads, smem, blocks, c_ns, regs_per_thread, reserved, m_ns=1):
    warps = threads // 32
    reg_warp = -(-regs_per_thread * 32 // REG_UNIT) * REG_UNIT
    return (warps * reg_warp, smem + reserved, warps, blocks, max(1, int(c_ns)), max(1, int(m_ns)))


def blocks_that_fit(threads, smem, regs, lim) -> int:
    """Blocks of one shape an SM holds at once (the four limits)."""
    _, regs_sm, smem_sm, warps_sm, blk_sm, reserved, _ = lim
    w = threads // 32
    return max(1, min(blk_sm, warps_sm // w, smem_sm // (smem + reserved),
                      regs_sm // (w * (-(-regs * 32 // REG_UNIT) * REG_UNIT))))


def calibrate_iters(target_us: float, base_iters: int, base_ms: float) -> int:
    """Chain length for a target alone time, from a measured (iters, ms) pair."""
    return max(1, min(1 << 24, int(round(base_iters * (target_us * 1e-3) / base_ms))))


def _capacity(hw, k, alone_ns, fit, n_sm):
    """Slowdown sweep of kernel k with 1..fit blocks per SM; the capacity that
    the duration rule needs to reproduce the most loaded point (None if no
    point is slowed by more than 5 %)."""
    t1 = hw.time_grid(k, n_sm, reps=5)
    slow = [(j, hw.time_grid(k, j * n_sm, reps=5) / t1) for j in range(1, fit + 1)]
    k_max, sl = slow[-1]
    cap = min(CAP_MAX, max(1, int(alone_ns * k_max / sl))) if sl > 1.05 else None
    return cap, slow


def run_set(seed: int, n: int, reps: int = 3, mixed: bool = False) -> dict:
    lim = ko.ko_hw_device_limits()
    n_sm, regs_sm, smem_sm, warps_sm, blk_sm, reserved, _ = lim
    regs = {k: ko.ko_hw_regs(k) for k in (ko.KO_HW_COMPUTE, ko.KO_HW_MEMORY)}
    shapes = draw_set(seed, n, n_sm, smem_sm - reserved, mixed)
    # loop iterations per microsecond of each kind, from one block of 128 threads
    base_iters = {ko.KO_HW_COMPUTE: 1 << 16, ko.KO_HW_MEMORY: 1 << 12}
    with ko.Hw([(k, 128, 0, 1, it) for k, it in base_iters.items()]) as probe:
        base_ms = {k: probe.time_grid(i, 1, reps=5) for i, k in enumerate(base_iters)}
    kernels = [(kind, t, sm, b, calibrate_iters(us, base_iters[kind], base_ms[kind]))
               for kind, t, sm, b, us in shapes]
    with ko.Hw(kernels) as hw:
        alone_ns = [hw.time_grid(i, 1, reps=5) * 1e6 for i in range(n)]
        caps, sweeps = {}, {}
        for kind, name in ((ko.KO_HW_COMPUTE, "ccap"), (ko.KO_HW_MEMORY, "mcap")):
            ref = next((i for i, sh in enumerate(shapes) if sh[0] == kind), None)
            if ref is None:
                caps[name] = None
                continue
            _, t, sm, _, _ = shapes[ref]
            caps[name], sweeps[name] = _capacity(hw, ref, alone_ns[ref],
                                                 blocks_that_fit(t, sm, regs[kind], lim), n_sm)
        orders = np.array(list(itertools.permutations(range(n))), dtype=np.int8)
        t_start = time.time()
        measured = hw.time_orders(orders, reps=reps)
        wall = time.time() - t_start
        traced = {}
        for name, o in (("identity", list(range(n))), ("reversed", list(range(n))[::-1])):
            rec, _ = hw.trace_order(o)
            traced[name] = dispatch_order_stats(rec, o)
    # a compute kernel's alone time is its c (m = c / 100); a memory kernel's is its m (c = m / 100)
    mk = []
    for (kind, t, sm, b, _), a in zip(shapes, alone_ns):
        c, m = (a, a / 100.0) if kind == ko.KO_HW_COMPUTE else (a / 100.0, a)
        mk.append(model_kernel(t, sm, b, c, regs[kind], reserved, m))
    out = {"seed": seed, "n": n, "mixed": mixed, "shapes": shapes, "alone_ns": alone_ns,
           "regs_per_thread": regs, "slowdown": sweeps, "timing_wall_s": wall, "dispatch": traced,
           "measured_ms": {"min": float(measured.min()), "max": float(measured.max()),
                           "spread": float(measured.max() / measured.min())}}
    calibrated = None
    if caps.get("ccap") is not None or caps.get("mcap") is not None:
        calibrated = (caps.get("ccap") or CAP_MAX, caps.get("mcap") or CAP_MAX)
    for label, cc in (("unbounded", (CAP_MAX, CAP_MAX)), ("calibrated", calibrated)):
        if cc is None:
            out[label] = None
            continue
        with ko.Gpu(n_sm, regs_sm, smem_sm, warps_sm, blk_sm, c_cap=cc[0], m_cap=cc[1]) as g:
            for row in mk:
                g.add_kernel(*row)
            sim = np.asarray(g.eval_orders(orders=orders))
            alg1 = g.heuristic_order().tolist()
        best_sim = int(np.argmin(sim))
        alg1_row = [i for i, o in enumerate(orders.tolist()) if o == alg1][0]
        pct = lambda m: 100.0 * float((measured >= m).sum()) / len(measured)  # noqa: E731
        out[label] = {"c_cap": cc[0], "m_cap": cc[1], "spearman": spearman(measured, sim),
                      "sim_spread": float(sim.max() / sim.min()),
                      "measured_percentile_of_sim_best": pct(measured[best_sim]),
                      "measured_percentile_of_alg1": pct(measured[alg1_row]),
                      "sim_best_measured_over_best": float(measured[best_sim] / measured.min())}
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=8)
    ap.add_argument("--n", type=int, default=6)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mixed", action="store_true", help="alternate compute and memory kernels")
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    rows = []
    for seed in range(a.sets):
        r = run_set(seed, a.n, a.reps, a.mixed)
        rows.append(r)
        brief = {k: (None if r[k] is None else {kk: round(v, 4) if isinstance(v, float) else v
                                                 for kk, v in r[k].items()})
                 for k in ("unbounded", "calibrated")}
        print(json.dumps({"seed": seed, "spread": round(r["measured_ms"]["spread"], 4), **brief,
                          "dispatch": r["dispatch"]}), flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
