"""GPU parity of the batched launch: per-set statistics and histograms of many
sets in one captured graph equal the oracle's, and equal one-set calls."""
import math

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


def _oracle_stats(s, nbins):
    h = oracle.heuristic(s.gpu, s.kernels)
    mh = oracle.makespan(s.gpu, s.kernels, h)
    return oracle.exhaustive_stats(s.gpu, s.kernels, mh, nbins=nbins)


def test_batch_small_sets_match_oracle(ko):
    # uneven N, mixed simulated GPUs; every set small enough for the oracle
    sets = []
    for i in range(60):
        s = synth.gen_set("batched", i)
        if s.n <= 7:
            sets.append(s)
    sets = sets[:24]
    gpus = [ko.Gpu.from_set(s) for s in sets]
    b = ko.Batch(gpus, nbins=256)
    for rep in range(2):   # the graph replays with identical results
        res, hist = b.run()
        for s, r, h in zip(sets, res, hist):
            st = _oracle_stats(s, 256)
            assert (r["min"], r["max"], r["makespan"], r["n_total"]) == \
                (st["min"], st["max"], st["makespan"], st["n_total"])
            assert (r["n_better"], r["n_equal"], r["n_worse"]) == \
                (st["n_better"], st["n_equal"], st["n_worse"])
            assert np.array_equal(h, st["hist"])
    assert b.orders() == sum(math.factorial(s.n) for s in sets)


@pytest.mark.parametrize("lanes", [1, 16, 32])
def test_batch_of_shared_memory_node_states(ko, lanes):
    # every handle keeps its node states in shared memory: the graph's
    # reference-order pass (global slab) must still have its slab sized
    # before capture
    sets = [s for s in (synth.gen_set("batched", i) for i in range(40)) if s.n <= 7][:8]
    gpus = [ko.Gpu.from_set(s).configure(lanes=lanes, levels=2, stack_global=0) for s in sets]
    b = ko.Batch(gpus, nbins=64)
    res, hist = b.run()
    for s, r, h in zip(sets, res, hist):
        st = _oracle_stats(s, 64)
        assert (r["min"], r["max"], r["makespan"]) == (st["min"], st["max"], st["makespan"])
        assert (r["n_better"], r["n_equal"], r["n_worse"]) == (st["n_better"], st["n_equal"], st["n_worse"])
        assert np.array_equal(h, st["hist"])
    b.close()
    for g in gpus:
        g.close()


def test_batch_equals_single_set_calls(ko):
    sets = [synth.gen_set("batched", i) for i in range(30, 46)]
    gpus = [ko.Gpu.from_set(s) for s in sets]
    b = ko.Batch(gpus, nbins=0)
    res, _ = b.run()
    for s, r in zip(sets, res):
        with ko.Gpu.from_set(s) as g:
            one, _ = g.rank_order(None, nbins=0)
        for k in ("min", "max", "makespan", "n_better", "n_equal", "n_worse", "n_total"):
            assert r[k] == one[k], k


def test_batch_forced_handover(ko):
    sets = [synth.gen_set("batched", i) for i in range(60) if synth.gen_set("batched", i).n <= 6][:6]
    gpus = [ko.Gpu.from_set(s).configure(run_limit=2) for s in sets]
    b = ko.Batch(gpus, nbins=64)
    res, hist = b.run()
    for s, r, h in zip(sets, res, hist):
        st = _oracle_stats(s, 64)
        assert (r["min"], r["max"], r["n_equal"]) == (st["min"], st["max"], st["n_equal"])
        assert np.array_equal(h, st["hist"])


def test_batch_rejects_large_sets(ko):
    s = synth.random_set(1, 13)
    with pytest.raises(ko.KoError) as e:
        ko.Batch([ko.Gpu.from_set(s)])
    assert e.value.code == -3


def _check_full_batch(ko, sets, res, hist, nbins, cross):
    for i, (s, r) in enumerate(zip(sets, res)):
        total = math.factorial(s.n)
        assert r["n_total"] == total
        assert r["n_better"] + r["n_equal"] + r["n_worse"] == total and r["n_equal"] >= 1
        h = oracle.heuristic(s.gpu, s.kernels)
        assert r["makespan"] == oracle.makespan(s.gpu, s.kernels, h), i
        lb, ub = oracle.bounds(s.gpu, s.kernels)
        assert lb <= r["min"] <= r["makespan"] <= r["max"] <= ub
        if hist is not None:
            assert int(hist[i].sum()) == total and hist[i][0] >= 1
    for i in cross:   # single-set path on the same set (oracle-checked elsewhere)
        with ko.Gpu.from_set(sets[i]) as g:
            one, h1 = g.rank_order(None, nbins=nbins or 1)
        for k in ("min", "max", "makespan", "n_better", "n_equal", "n_worse"):
            assert res[i][k] == one[k], (i, k)
        if hist is not None:
            assert np.array_equal(hist[i], h1)


def test_sixty_four_n10_sets_with_histograms(ko):
    """All 64 N=10 sets (15-SM GPU), 232,243,200 orders, one captured graph."""
    sets = [synth.gen_set("sets10", i) for i in range(64)]
    b = ko.Batch([ko.Gpu.from_set(s) for s in sets], nbins=4096)
    res, hist = b.run()
    assert b.orders() == 64 * math.factorial(10)
    _check_full_batch(ko, sets, res, hist, 4096, cross=(0, 17, 63))


def test_mixed_batch_first_512_sets(ko):
    """First 512 of the 4096 mixed sets (N 5..10, 13/15/148 SMs)."""
    sets = [synth.gen_set("batched", i) for i in range(512)]
    b = ko.Batch([ko.Gpu.from_set(s) for s in sets], nbins=0)
    res, _ = b.run()
    _check_full_batch(ko, sets, res, None, 0, cross=(1, 200, 511))


def _class_key(s):
    S = s.gpu[0]
    c = 16 if S <= 16 else 32 if S <= 32 else 64 if S <= 64 else 128 if S <= 128 else 160 if S <= 160 else 1024
    return f"B_S{c}_N{s.n}"


def test_batch_autotune_per_class(ko, tmp_path):
    """ko_batch_autotune gives every set its class's choice, stores the timed
    classes in the cache, and the tuned batch (one launch per choice) returns
    what the default batch returns; small sets also match the oracle."""
    import json
    sets = [synth.gen_set("batched", i) for i in range(400)]
    gpus = [ko.Gpu.from_set(s) for s in sets]
    cache = str(tmp_path / "tune.json")
    ko.ko_batch_autotune(gpus, cache)
    data = json.load(open(cache))
    by_class = {}
    for s, g in zip(sets, gpus):
        c = (ko.ko_get_option(g.h, ko.KO_OPT_LANES), ko.ko_get_option(g.h, ko.KO_OPT_LEVELS),
             ko.ko_get_option(g.h, ko.KO_OPT_STACK_GLOBAL), ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE))
        assert c[0] in (1, 16, 32) and 1 <= c[1] <= min(s.n - 1, 5) and c[2] in (0, 1) and c[3] in (0, 1, 2)
        by_class.setdefault(_class_key(s), set()).add(c)
    assert all(len(v) == 1 for v in by_class.values())
    timed = {k for k in by_class if sum(math.factorial(s.n) for s in sets if _class_key(s) == k) >= 1 << 21}
    assert timed and timed <= set(data)
    for k in timed:
        assert (data[k]["lanes"], data[k]["levels"], data[k]["stack"], data[k]["shape"]) == next(iter(by_class[k]))
    b = ko.Batch(gpus, nbins=0)
    res, _ = b.run()
    plain = [ko.Gpu.from_set(s) for s in sets]
    b2 = ko.Batch(plain, nbins=0)
    res2, _ = b2.run()
    for r, r2 in zip(res, res2):
        for k in ("min", "max", "makespan", "n_better", "n_equal", "n_worse", "n_total"):
            assert r[k] == r2[k]
    for s, r in zip(sets, res):
        if s.n <= 6:
            st = _oracle_stats(s, 0)
            assert (r["min"], r["max"], r["n_better"], r["n_equal"], r["n_worse"]) == \
                (st["min"], st["max"], st["n_better"], st["n_equal"], st["n_worse"])
    # a second tuner call is served from the cache
    again = [ko.Gpu.from_set(s) for s in sets[:50]]
    ko.ko_batch_autotune(again, cache)
    for s, g in zip(sets[:50], again):
        assert (ko.ko_get_option(g.h, ko.KO_OPT_LANES), ko.ko_get_option(g.h, ko.KO_OPT_LEVELS),
                ko.ko_get_option(g.h, ko.KO_OPT_STACK_GLOBAL),
                ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE)) == next(iter(by_class[_class_key(s)]))
