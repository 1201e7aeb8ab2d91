"""GPU parity of the run-length, prefix-sharing simulator: every makespan must
equal the oracle's (and the simple device simulator's) for every tuning knob
setting, including forced hand-over of work items to the simple simulator."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


def _all(g, n):
    import torch
    out = torch.empty(math.factorial(n), dtype=torch.int64, device="cuda")
    g.eval_all(out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("lanes", [16, 32])
@pytest.mark.parametrize("levels", [0, 1, 3, 4, 6])
def test_single8_all_orders_every_config(ko, lanes, levels):
    s = synth.gen_set("single8")
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=40320)
    with ko.Gpu.from_set(s) as g:
        g.configure(lanes=lanes, levels=levels)
        assert np.array_equal(_all(g, 8), want)
        assert g.last_fallback_items() == 0


@pytest.mark.parametrize("seed", range(12))
def test_random_small_sets_exhaustive(ko, seed):
    # mixes of tiny and large N_SM, power-of-two and odd capacities, heavy smem
    n = 3 + seed % 6
    gpus = [(13, 65536, 49152, 64, 16), (148, 65536, 233472, 64, 32), (7, 32768, 49152, 48, 8),
            (40, 65536, 98304, 64, 32)]
    gpu = gpus[seed % len(gpus)]
    caps = (32768, 32768) if seed % 3 else (3000, 7001)
    s = synth.random_set(100 + seed, n, gpu=gpu, blk=(1, 5 * gpu[0]), c=(100, 30000),
                         c_cap=caps[0], m_cap=caps[1])
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(n))
    for lanes in (16, 32):
        with ko.Gpu.from_set(s) as g:
            g.configure(lanes=lanes)
            got = _all(g, n)
            assert np.array_equal(got, want), (lanes, int(np.argmax(got != want)))


@pytest.mark.parametrize("run_limit", [1, 2, 3])
def test_forced_handover_to_simple_simulator(ko, run_limit):
    s = synth.gen_set("sets10", 2, n=7)
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=5040)
    h = oracle.heuristic(s.gpu, s.kernels)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h),
                                 makespans=want)
    with ko.Gpu.from_set(s) as g:
        g.configure(run_limit=run_limit)
        assert np.array_equal(_all(g, 7), want)
        assert g.last_fallback_items() > 0
        r, hist = g.rank_order(h, nbins=4096)
    assert (r["min"], r["max"], r["n_better"], r["n_equal"], r["n_worse"]) == \
        (st["min"], st["max"], st["n_better"], st["n_equal"], st["n_worse"])
    assert np.array_equal(hist, st["hist"])


def test_every_item_handed_over_on_a_large_launch(ko):
    """More abandoned work items than any fixed list would hold: ten one-block
    kernels on a 2-SM GPU, one saved level (1,814,400 items of two orders) and
    one run per simulation allowed.  Every item's first kernel cuts the single
    run, so all items fail both run-length passes and reach the simple
    simulator; every makespan must still arrive, equal to the default
    configuration's (itself checked against the oracle on samples)."""
    import torch
    s = synth.random_set(41, 10, gpu=(2, 65536, 49152, 64, 4), blk=(1, 1))
    n_all = math.factorial(10)
    with ko.Gpu.from_set(s) as g:
        ref = torch.empty(n_all, dtype=torch.int64, device="cuda")
        g.eval_all(ref)
        torch.cuda.synchronize()
    ids = synth.random_indices(31, n_all, 500)
    assert np.array_equal(ref[torch.from_numpy(ids.astype(np.int64)).cuda()].cpu().numpy(),
                          oracle.makespans_idx(s.gpu, s.kernels, idx=ids))
    with ko.Gpu.from_set(s) as g:
        g.configure(run_limit=1, levels=1)
        out = torch.full((n_all,), -7, dtype=torch.int64, device="cuda")
        g.eval_all(out)
        torch.cuda.synchronize()
        assert g.last_fallback_items() == n_all // 2 > (1 << 20)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("lanes", [16, 32])
def test_single12_index_sample(ko, lanes):
    s = synth.gen_set("single12")
    ids = synth.random_indices(77, math.factorial(12), 3000)
    with ko.Gpu.from_set(s) as g:
        g.configure(lanes=lanes)
        got = g.eval_orders(idx=ids)
    assert np.array_equal(got, oracle.makespans_idx(s.gpu, s.kernels, idx=ids))


def test_single12_full_space_as_benchmarked(ko, tmp_path):
    """The exhaustive N=12 launch in the configuration the benchmark times (the
    tuned lanes and depth, all 479,001,600 orders): seeded samples of the stored
    makespans, work-item boundaries and the first and last orders equal the
    oracle's one by one; the fused reductions agree with the stored makespans."""
    import shutil

    import torch
    s = synth.gen_set("single12")
    n_all = math.factorial(12)
    cache = tmp_path / "tune.json"
    shutil.copy(os.path.join(ROOT, "paper_1511_07983_gb300", "ko_tune_cache.json"), cache)
    with ko.Gpu.from_set(s) as g:
        choice = g.autotune(str(cache))
        per_item = math.factorial(choice["levels"] + 1)   # orders below one item's fixed prefix
        out = torch.empty(n_all, dtype=torch.int64, device="cuda")
        g.eval_all(out)
        r, hist = g.rank_order(None, nbins=4096)
        torch.cuda.synchronize()
        mh = oracle.makespan(s.gpu, s.kernels, g.heuristic_order().tolist())

    items = synth.random_indices(1213, n_all // per_item, 40).astype(np.int64)
    ids = np.concatenate([synth.random_indices(1212, n_all, 2000).astype(np.int64),
                          items * per_item, items * per_item + per_item - 1,
                          [0, 1, per_item - 1, per_item, n_all - per_item, n_all - 2, n_all - 1]])
    got = out[torch.from_numpy(ids).cuda()].cpu().numpy()
    assert np.array_equal(got, oracle.makespans_idx(s.gpu, s.kernels, idx=ids.astype(np.uint64)))

    lb, ub = oracle.bounds(s.gpu, s.kernels)
    mn, mx = int(out.min()), int(out.max())
    assert lb <= mn <= mx <= ub
    assert r["makespan"] == mh and r["n_total"] == n_all
    assert (r["min"], r["max"]) == (mn, mx)
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == \
        (int((out < mh).sum()), int((out == mh).sum()), int((out > mh).sum()))
    bins = torch.div((out - mn) * 4096, mx - mn + 1, rounding_mode="floor")
    assert np.array_equal(hist.astype(np.int64), torch.bincount(bins, minlength=4096).cpu().numpy())


def test_simple_and_fast_agree_on_sets10(ko):
    s = synth.gen_set("sets10", 5)
    with ko.Gpu.from_set(s) as g:
        fast = _all(g, 10)
    with ko.Gpu.from_set(s) as g:
        g.configure(simple_only=True)
        simple = _all(g, 10)
    assert np.array_equal(fast, simple)
    ids = synth.random_indices(3, math.factorial(10), 3000).astype(np.int64)
    assert np.array_equal(fast[ids], oracle.makespans_idx(s.gpu, s.kernels, idx=ids.astype(np.uint64)))


@pytest.mark.parametrize("workload,count", [("batched", 40)])
def test_batched_sets_exhaustive_small(ko, workload, count):
    # every batched set with N <= 8 exhaustively against the oracle
    checked = 0
    for i in range(count):
        s = synth.gen_set(workload, i)
        if s.n > 8:
            continue
        want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(s.n))
        with ko.Gpu.from_set(s) as g:
            assert np.array_equal(_all(g, s.n), want), i
        checked += 1
    assert checked > 5


def test_autotune_choice_cache_and_exactness(ko, tmp_path):
    import json
    s = synth.gen_set("sets10", 7, n=8)
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=40320)
    cache = str(tmp_path / "tune.json")
    with ko.Gpu.from_set(s) as g:
        choice = g.autotune(cache)
        assert choice["lanes"] in (1, 16, 32) and 1 <= choice["levels"] <= 6
        assert choice["stack_global"] in (0, 1) and choice["lane_state"] in (0, 1, 2)
        assert np.array_equal(_all(g, 8), want)
    data = json.load(open(cache))
    assert data["S16_N8"]["lanes"] == choice["lanes"] and data["S16_N8"]["levels"] == choice["levels"]
    assert data["S16_N8"]["stack"] == choice["stack_global"] and data["S16_N8"]["shape"] == choice["lane_state"]
    with ko.Gpu.from_set(s) as g:   # second handle: served from the cache
        assert g.autotune(cache) == choice


@pytest.mark.parametrize("lanes", [16, 32])
@pytest.mark.parametrize("levels", [1, 3, 5])
def test_global_node_stack_is_exact(ko, lanes, levels):
    s = synth.gen_set("single8")
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=40320)
    with ko.Gpu.from_set(s) as g:
        g.configure(lanes=lanes, levels=levels, stack_global=True)
        assert np.array_equal(_all(g, 8), want)
        r, hist = g.rank_order(None, nbins=4096)
    h = oracle.heuristic(s.gpu, s.kernels)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h), makespans=want)
    assert (r["min"], r["max"], r["n_equal"]) == (st["min"], st["max"], st["n_equal"])
    assert np.array_equal(hist, st["hist"])


@pytest.mark.parametrize("case", ["sm1024", "one_block_per_sm", "no_smem", "huge_durations", "bk32_tiny_sm"])
def test_edge_gpus_match_oracle(ko, case):
    if case == "sm1024":        # many runs: hand-over to the wide pass and the simple simulator
        s = synth.random_set(41, 5, gpu=(1024, 65536, 233472, 64, 32), blk=(100, 3000), c=(1000, 50000))
    elif case == "one_block_per_sm":
        s = synth.random_set(42, 6, gpu=(7, 65536, 233472, 64, 1), blk=(1, 30))
    elif case == "no_smem":
        s = synth.random_set(43, 6, gpu=(13, 65536, 49152, 64, 16), blk=(5, 80))
        s.kernels[:, 1] = 0
    elif case == "huge_durations":  # durations reach 2^31: the run-length path does not apply
        s = synth.random_set(44, 5, gpu=(13, 65536, 49152, 64, 16), blk=(5, 60), c=(1 << 19, 1 << 20),
                             c_cap=1, m_cap=1)
    else:
        s = synth.random_set(45, 6, gpu=(2, 65536, 233472, 64, 32), blk=(1, 40))
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(s.n))
    with ko.Gpu.from_set(s) as g:
        got = _all(g, s.n)
        assert np.array_equal(got, want), case
        h = oracle.heuristic(s.gpu, s.kernels)
        r, hist = g.rank_order(h, nbins=128)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h), nbins=128,
                                 makespans=want)
    assert (r["min"], r["max"], r["n_better"], r["n_equal"], r["n_worse"]) == \
        (st["min"], st["max"], st["n_better"], st["n_equal"], st["n_worse"])
    assert np.array_equal(hist, st["hist"])
