"""Launch-order strategies ranked against the whole permutation space.

For each set, every one of the N! orders is simulated (ko_eval_all) and each
strategy's order is placed in that ranking: its percentile
100 * #{orders with makespan >= M} / N! (the Table 3 percentile of Sec. 6),
its deviation (M - optimum) / optimum, and whether it is optimal.  The
strategies are Algorithm 1 under the two readings of its resource terms
(per-SM and per-block footprints, Sec. 5) and exact steepest-descent local
search (swaps, or swaps and moves) started from Algorithm 1's order or from
the order the kernels were added in.

With --variants K it also compares, on K ten-kernel sets, the default model
with its two variants (durations fixed at placement; processor sharing with
rates re-evaluated at every event): rank agreement over all orders and how
each model's best order and Algorithm 1's order rank under the other.

    python -m paper_1511_07983_gb300.study [--sets10 64] [--n11 16] [--variants 16] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ko, synth

STRATEGIES = ("alg1_per_sm", "alg1_per_block", "ls_swap_from_alg1", "ls_swap_move_from_alg1",
              "ls_swap_move_from_identity")


def rank_set(s) -> dict:
    """Percentile, deviation and search cost of every strategy on one set."""
    import torch
    n = s.n
    with ko.Gpu.from_set(s) as g:
        every = torch.empty(math.factorial(n), dtype=torch.int64, device="cuda")
        g.eval_all(every)
        torch.cuda.synchronize()
        best = int(every.min().item())
        orders, cost = {}, {}
        orders["alg1_per_sm"] = g.heuristic_order(ko.KO_HEUR_PER_SM)
        orders["alg1_per_block"] = g.heuristic_order(ko.KO_HEUR_PER_BLOCK)
        for name, start, moves in (("ls_swap_from_alg1", None, False), ("ls_swap_move_from_alg1", None, True),
                                   ("ls_swap_move_from_identity", list(range(n)), True)):
            o, _, steps, evals, ms = g.local_search(start=start, moves=moves)
            orders[name] = o
            cost[name] = {"steps": steps, "orders_simulated": evals, "gpu_ms": ms}
        rows = np.stack([np.asarray(orders[k], dtype=np.int8) for k in STRATEGIES])
        mk = g.eval_orders(orders=rows)
        out = {"n": n, "n_sm": int(s.gpu[0]), "optimum": best, "worst": int(every.max().item())}
        for k, m in zip(STRATEGIES, np.asarray(mk).tolist()):
            pct = 100.0 * int((every >= m).sum().item()) / every.numel()
            out[k] = {"makespan": int(m), "percentile": pct, "deviation": (m - best) / best,
                      "optimal": bool(m == best), **cost.get(k, {})}
        del every
    return out


def variants_set(s) -> dict:
    """One set under the default model (durations fixed after each burst) and
    its two variants -- durations fixed at placement, and processor sharing
    with rates re-evaluated at every event: for each variant, rank agreement
    with the default over all N! orders, the share of orders whose makespan
    changes, how each model's optimum ranks under the other, and Algorithm 1's
    percentile under both."""
    import itertools
    import torch
    from .hwval import spearman
    n = s.n
    with ko.Gpu.from_set(s) as g:
        every = torch.empty(math.factorial(n), dtype=torch.int64, device="cuda")
        g.eval_all(every)
        torch.cuda.synchronize()
        base = every.cpu().numpy()
        alg1 = g.heuristic_order()
    with ko.Gpu.from_set(s, sampling=ko.KO_SAMPLE_AT_PLACEMENT) as g:
        every = torch.empty(math.factorial(n), dtype=torch.int64, device="cuda")
        g.eval_all(every)
        torch.cuda.synchronize()
        placement = every.cpu().numpy()
    rows = torch.tensor(list(itertools.permutations(range(n))), dtype=torch.int8, device="cuda")
    with ko.Gpu.from_set(s) as g:
        ps = torch.empty(rows.shape[0], dtype=torch.float64, device="cuda")
        g.eval_orders_ps(rows, out=ps)
        torch.cuda.synchronize()
        ps = ps.cpu().numpy()
    del rows
    ia = int(sum(int(d) * math.factorial(n - 1 - j) for j, d in enumerate(_lehmer_digits(alg1))))
    pct = lambda v, m: 100.0 * float((v >= m).sum()) / len(v)  # noqa: E731
    out = {"n": n, "n_sm": int(s.gpu[0]), "alg1_percentile_burst_end": pct(base, base[ia])}
    for name, v in (("at_placement", placement), ("processor_sharing", ps)):
        out[name] = {"spearman": spearman(base, v), "changed_orders": float((base != v).mean()),
                     "burst_end_optimum_percentile": pct(v, v[int(np.argmin(base))]),
                     "optimum_percentile_burst_end": pct(base, base[int(np.argmin(v))]),
                     "alg1_percentile": pct(v, v[ia])}
    return out


def _lehmer_digits(order):
    """Lexicographic Lehmer digits of a permutation (index = sum d_j (n-1-j)!)."""
    rest = sorted(int(v) for v in order)
    out = []
    for v in order:
        d = rest.index(int(v))
        out.append(d)
        rest.pop(d)
    return out


def summarise(rows: list[dict]) -> dict:
    out = {}
    for k in STRATEGIES:
        v = [r[k] for r in rows]
        out[k] = {"mean_percentile": float(np.mean([x["percentile"] for x in v])),
                  "mean_deviation": float(np.mean([x["deviation"] for x in v])),
                  "optimal": int(sum(x["optimal"] for x in v)), "sets": len(v)}
        if "orders_simulated" in v[0]:
            out[k]["mean_orders_simulated"] = float(np.mean([x["orders_simulated"] for x in v]))
            out[k]["mean_gpu_ms"] = float(np.mean([x["gpu_ms"] for x in v]))
    return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets10", type=int, default=64, help="N=10 sets on the 15-SM GPU")
    ap.add_argument("--n11", type=int, default=16, help="N=11 sets on the 148-SM GPU")
    ap.add_argument("--variants", type=int, default=0,
                    help="also compare the model with its two variants on this many N=10 sets")
    ap.add_argument("--json", default=None)
    a = ap.parse_args(argv)
    groups = {"sets10 (N=10, 15 SMs)": [synth.gen_set("sets10", i) for i in range(a.sets10)],
              "N=11, 148 SMs": [synth.gen_set("single12", i, n=11) for i in range(a.n11)]}
    report = {}
    for name, sets in groups.items():
        if not sets:
            continue
        t0 = time.time()
        rows = [rank_set(s) for s in sets]
        report[name] = {"summary": summarise(rows), "wall_s": time.time() - t0, "sets": rows}
        print(json.dumps({name: report[name]["summary"]}, indent=1), flush=True)
    if a.variants:
        t0 = time.time()
        rows = [variants_set(synth.gen_set("sets10", i)) for i in range(a.variants)]
        summ = {"alg1_percentile_burst_end": float(np.mean([r["alg1_percentile_burst_end"] for r in rows]))}
        for name in ("at_placement", "processor_sharing"):
            summ[name] = {k: float(np.mean([r[name][k] for r in rows])) for k in rows[0][name]}
            summ[name]["min_spearman"] = float(min(r[name]["spearman"] for r in rows))
        report["model variants, sets10"] = {"summary": summ, "wall_s": time.time() - t0, "sets": rows}
        print(json.dumps({"model variants, sets10": summ}, indent=1), flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
