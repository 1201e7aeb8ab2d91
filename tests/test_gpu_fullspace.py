"""Full-space parity at the sizes the small oracle tests cannot reach.

* One N=10 set (15-SM GPU, the 64-set workload's first set): the oracle
  simulates all 3,628,800 orders on the host cores; the GPU's makespans are
  compared with them element by element, and its min / max, better / equal /
  worse counts and 4096-bin histogram with the oracle's own statistics --
  through one-set calls (every simulator) and as row 0 of the 64-set batch.
* The 4096-set mixed batch (N 5..10 on 13-, 15- and 148-SM GPUs) in one
  launch: every set with N <= 8 against the oracle's exhaustive statistics
  stored in tests/golden/batched_small_oracle.json (written by the committed
  script beside it, which calls only oracle/), and 256 seeded larger sets
  against properties the oracle fixes: Algorithm 1's makespan, bounds that
  contain seeded samples of exact makespans, counts and histograms that sum
  to N!."""
import hashlib
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NBINS = 4096


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


@pytest.fixture(scope="module")
def n10():
    """The oracle's whole space of the first 10-kernel set."""
    s = synth.gen_set("sets10", 0)
    ms = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(10))
    h = oracle.heuristic(s.gpu, s.kernels)
    mh = oracle.makespan(s.gpu, s.kernels, h)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, mh, nbins=NBINS, makespans=ms)
    return s, ms, h, st


def _stats_equal(r, st):
    assert (r["min"], r["max"], r["makespan"], r["n_total"]) == \
        (st["min"], st["max"], st["makespan"], st["n_total"])
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == \
        (st["n_better"], st["n_equal"], st["n_worse"])


# (1, 3): 151,200 items, the one-thread pass in full blocks (one per SM); (1, 5): 5,040 items,
# fewer than SMs x block threads, so it runs in the small blocks that spread them over the SMs
@pytest.mark.parametrize("lanes,levels", [(None, None), (16, 4), (32, 3), (1, 3), (1, 5)])
def test_n10_full_space(ko, n10, lanes, levels):
    import torch
    s, ms, h, st = n10
    with ko.Gpu.from_set(s) as g:
        if lanes is not None:
            g.configure(lanes=lanes, levels=levels)
        out = torch.full((ms.size,), -7, dtype=torch.int64, device="cuda")
        g.eval_all(out)
        r, hist = g.rank_order(h, nbins=NBINS)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
    assert np.array_equal(got, ms), int(np.argmax(got != ms))
    _stats_equal(r, st)
    assert np.array_equal(hist, st["hist"])


def test_n10_batch_row_full_space(ko, n10):
    s, ms, h, st = n10
    sets = [synth.gen_set("sets10", i) for i in range(64)]
    assert np.array_equal(sets[0].kernels, s.kernels)
    gpus = [ko.Gpu.from_set(x) for x in sets]
    b = ko.Batch(gpus, nbins=NBINS)
    res, hist = b.run()
    _stats_equal(res[0], st)
    assert np.array_equal(hist[0], st["hist"])
    for r, x, hrow in zip(res, sets, hist):     # every set: counts and histogram cover N!
        assert r["n_better"] + r["n_equal"] + r["n_worse"] == math.factorial(10)
        assert int(hrow.sum()) == math.factorial(10)
    b.close()
    for g in gpus:
        g.close()


def test_batched_4096_sets_one_launch(ko):
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "batched_small_oracle.json")))
    assert gold["nbins"] == NBINS and gold["nsets"] == 4096
    sets = [synth.gen_set("batched", i) for i in range(4096)]
    gpus = [ko.Gpu.from_set(x) for x in sets]
    b = ko.Batch(gpus, nbins=NBINS)
    res, hist = b.run()
    assert b.orders() == sum(math.factorial(x.n) for x in sets)
    checked = 0
    for key, row in gold["sets"].items():
        i = int(key)
        n, mn, mx, mh, nb, ne, nw, sha = row
        r = res[i]
        assert sets[i].n == n
        assert (r["min"], r["max"], r["makespan"], r["n_better"], r["n_equal"], r["n_worse"]) == \
            (mn, mx, mh, nb, ne, nw), i
        assert hashlib.sha256(hist[i].astype(np.int64).tobytes()).hexdigest() == sha, i
        checked += 1
    assert checked == sum(1 for x in sets if x.n <= 8)
    # seeded larger sets: what the oracle fixes without enumerating them
    large = [i for i, x in enumerate(sets) if x.n > 8]
    pick = synth.random_indices(4096, len(large), 256)
    for j in np.unique(pick.astype(np.int64)):
        i = large[int(j)]
        x, r = sets[i], res[i]
        total = math.factorial(x.n)
        assert r["n_total"] == total and r["n_better"] + r["n_equal"] + r["n_worse"] == total
        assert int(hist[i].sum()) == total
        assert r["makespan"] == oracle.makespan(x.gpu, x.kernels, oracle.heuristic(x.gpu, x.kernels))
        sample = oracle.makespans_idx(x.gpu, x.kernels, idx=synth.random_indices(i, total, 24))
        lb, ub = oracle.bounds(x.gpu, x.kernels)
        assert lb <= r["min"] <= sample.min() and sample.max() <= r["max"] <= ub, i
    b.close()
    for g in gpus:
        g.close()
