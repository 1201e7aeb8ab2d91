"""Writes tests/golden/batched_small_oracle.json: the oracle's exhaustive
statistics of every set with N <= 8 of the 4096-set batched workload (sets of
N 5..10 on 13-, 15- and 148-SM simulated GPUs).

For each such set: N, min, max, the makespan of Algorithm 1's order, the
better / equal / worse counts against it, and the SHA-256 of the 4096-bin
histogram (int64, bin = floor((M - min) * 4096 / (max - min + 1))).  Every
value comes from oracle/ alone (block-by-block simulation of all N! orders,
Algorithm 1, exact integer histogram); the batched GPU test compares the
library's one-launch batch against it.

    python tests/golden/make_batched_oracle.py [--threads T]
"""
import argparse
import hashlib
import json
import math
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1511_07983_gb300 import synth  # noqa: E402

NSETS = 4096
NBINS = 4096
OUT = os.path.join(ROOT, "tests", "golden", "batched_small_oracle.json")


def hist_sha(hist):
    import numpy as np
    return hashlib.sha256(np.asarray(hist, dtype=np.int64).tobytes()).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    rows = {}
    t0 = time.time()
    for i in range(NSETS):
        s = synth.gen_set("batched", i)
        if s.n > 8:
            continue
        ms = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(s.n), threads=a.threads)
        h = oracle.heuristic(s.gpu, s.kernels)
        mh = oracle.makespan(s.gpu, s.kernels, h)
        st = oracle.exhaustive_stats(s.gpu, s.kernels, mh, nbins=NBINS, makespans=ms)
        rows[str(i)] = [s.n, st["min"], st["max"], mh, st["n_better"], st["n_equal"], st["n_worse"],
                        hist_sha(st["hist"])]
    json.dump({"workload": "batched", "nsets": NSETS, "nbins": NBINS,
               "fields": ["n", "min", "max", "heuristic_makespan", "n_better", "n_equal", "n_worse",
                          "hist_sha256"],
               "sets": rows}, open(OUT, "w"), separators=(",", ":"))
    print(f"{len(rows)} sets in {time.time() - t0:.0f} s -> {OUT}")


if __name__ == "__main__":
    main()
