"""Pins for the CPU oracle (no GPU).

Every expectation here comes from outside the oracle: hand traces of the
dispatch rule, values the paper prints (Table 3), library routines
(itertools.permutations is lexicographic), closed forms and invariants the
paper states (Sec. 2, Sec. 3).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    with open(os.path.join(GOLD, "hand_traces.json")) as f:
        return {c["name"]: c for c in json.load(f)["cases"]}


CASES = _cases()


# ------------------------------------------------------------------ Lehmer ---

def test_unrank_n3_table():
    table = [[0, 1, 2], [0, 2, 1], [1, 0, 2], [1, 2, 0], [2, 0, 1], [2, 1, 0]]
    assert [oracle.unrank(3, k) for k in range(6)] == table


@pytest.mark.parametrize("n", [1, 2, 4, 6, 8])
def test_unrank_is_lexicographic_bijection(n):
    # itertools.permutations of a sorted input yields lexicographic order
    ref = list(itertools.permutations(range(n)))
    got = [tuple(oracle.unrank(n, k)) for k in range(math.factorial(n))]
    assert got == ref
    for k in range(0, math.factorial(n), max(1, math.factorial(n) // 997)):
        assert oracle.rank(ref[k]) == k


@pytest.mark.parametrize("n", [9, 12, 16, 20])
def test_unrank_endpoints(n):
    assert oracle.unrank(n, 0) == list(range(n))
    assert oracle.unrank(n, math.factorial(n) - 1) == list(range(n))[::-1]
    rng = np.random.default_rng(n)
    for _ in range(50):
        perm = list(rng.permutation(n))
        assert oracle.unrank(n, oracle.rank(perm)) == perm


# ---------------------------------------------------------- hand traces ---

@pytest.mark.parametrize("name", ["W1", "T3", "T4", "W2", "P1", "P2"])
def test_hand_traced_makespans(name):
    c = CASES[name]
    for order, expect in c["makespans"]:
        assert oracle.makespan(c["gpu"], c["kernels"], order) == expect, (name, order)


def test_w1_exhaustive_stats():
    c = CASES["W1"]
    st = oracle.exhaustive_stats(c["gpu"], c["kernels"], 210, nbins=4096)
    assert (st["min"], st["max"], st["n_total"]) == (210, 300, 2)
    assert (st["n_better"], st["n_equal"], st["n_worse"]) == (0, 1, 1)
    h = st["hist"]
    assert h[0] == 1 and h[(300 - 210) * 4096 // 91] == 1 and h.sum() == 2
    out = oracle.rank_outputs(st)
    assert out["percentile"] == 100.0 and out["percentile_strict"] == 50.0
    assert out["speedup_over_worst"] == 300 / 210
    assert out["deviation_from_optimal"] == 0.0


def test_w1_bounds():
    c = CASES["W1"]
    assert oracle.bounds(c["gpu"], c["kernels"]) == (c["lb"], c["ub"])


# ------------------------------------------------------ closed forms ---

@pytest.mark.parametrize("b", [1, 5, 13, 14, 26, 39, 40])
def test_single_kernel_one_burst_closed_form(b):
    # One kernel, every block placed at t=0: SM s gets floor(b/S) + [s < b mod S]
    # blocks, so the busiest SM holds ceil(b/S) and the makespan is its duration.
    S, cap = 13, 4096
    gpu = (S, 65536, 49152, 64, 16, cap, cap)
    c, m = 3000, 700
    kern = [[2048, 0, 4, b, c, m]]
    j = -(-b // S)
    expect = max(-(-(c * max(j * c, cap)) // cap), -(-(m * max(j * m, cap)) // cap))
    assert oracle.makespan(gpu, kern, [0]) == expect


@pytest.mark.parametrize("rounds", [1, 2, 5])
def test_single_kernel_full_rounds(rounds):
    # Exactly `rounds` full waves of k blocks per SM: identical waves run back to back.
    S, cap, k = 7, 1000, 3
    gpu = (S, 3 * 1000, 10 ** 6, 64, 16, cap, cap)
    c, m = 900, 400
    kern = [[1000, 0, 2, rounds * S * k, c, m]]
    d = max(-(-(c * max(k * c, cap)) // cap), -(-(m * max(k * m, cap)) // cap))
    assert oracle.makespan(gpu, kern, [0]) == rounds * d


# ------------------------------------------------------ paper invariants ---

@pytest.mark.parametrize("seed", range(6))
def test_order_invariant_when_blocks_fit_one_per_sm(seed):
    # Sec. 2: total blocks <= N_SM -> no SM is shared, order does not matter.
    ks = synth.random_set(seed, 5, gpu=(40, 65536, 49152, 64, 16), blk=(1, 8)).kernels
    total = int(ks[:, 3].sum())
    gpu = (max(total, 1), 65536, 49152, 64, 16, 32768, 32768)
    ms = oracle.makespans_idx(gpu, ks, first=0, count=120)
    assert len(set(ms.tolist())) == 1
    d0 = [max(-(-(c * max(c, 32768)) // 32768), -(-(m * max(m, 32768)) // 32768))
          for c, m in ks[:, 4:6].tolist()]
    assert ms[0] == max(d0)


@pytest.mark.parametrize("seed", range(4))
def test_order_invariant_identical_kernels(seed):
    # Sec. 3: identical kernels that differ only in N_tblk -> order does not matter.
    ks = synth.random_set(seed, 6, blk=(1, 60)).kernels
    ks[:, [0, 1, 2, 4, 5]] = ks[0, [0, 1, 2, 4, 5]]
    gpu = (13, 65536, 49152, 64, 16, 32768, 32768)
    ms = oracle.makespans_idx(gpu, ks, first=0, count=720)
    assert len(set(ms.tolist())) == 1


@pytest.mark.parametrize("seed", range(8))
def test_bounds_bracket_every_order(seed):
    s = synth.random_set(seed, 6, blk=(4, 60), c=(100, 20000))
    lb, ub = oracle.bounds(s.gpu, s.kernels)
    ms = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=720)
    assert lb <= ms.min() and ms.max() <= ub


def test_determinism_and_threads():
    s = synth.gen_set("single8")
    a = oracle.makespans_idx(s.gpu, s.kernels, first=1000, count=500, threads=1)
    b = oracle.makespans_idx(s.gpu, s.kernels, first=1000, count=500, threads=7)
    assert np.array_equal(a, b)
    orders = np.array([oracle.unrank(8, 1000 + j) for j in range(0, 500, 50)], dtype=np.int32)
    assert np.array_equal(oracle.makespans_orders(s.gpu, s.kernels, orders), a[::50])


def test_exhaustive_counts_and_histogram_sum():
    s = synth.random_set(11, 6, blk=(4, 60))
    h = oracle.makespan(s.gpu, s.kernels, oracle.heuristic(s.gpu, s.kernels))
    st = oracle.exhaustive_stats(s.gpu, s.kernels, h)
    assert st["n_better"] + st["n_equal"] + st["n_worse"] == 720
    assert st["hist"].sum() == 720 and st["hist"][0] >= 1 and st["n_equal"] >= 1
    top = (st["max"] - st["min"]) * 4096 // (st["max"] - st["min"] + 1)
    assert st["hist"][top] >= 1 and st["hist"][top + 1:].sum() == 0


def test_unfittable_block_reports_error():
    gpu = (2, 100, 100, 100, 4, 10, 10)
    assert oracle.makespan(gpu, [[101, 0, 1, 1, 1, 1]], [0]) == -1


def test_empty_set():
    assert oracle.makespan((2, 100, 100, 100, 4, 10, 10), np.zeros((0, 6)), []) == 0


# ------------------------------------------------------------ Algorithm 1 ---

@pytest.mark.parametrize("name", ["W1", "W2", "W3", "W4", "W5"])
def test_heuristic_hand_traced(name):
    c = CASES[name]
    assert oracle.heuristic(c["gpu"], c["kernels"]) == c["heuristic"]
    if "rounds" in c:
        assert oracle.heuristic_rounds(c["gpu"], c["kernels"]) == c["rounds"]
    for i, j, v in c.get("scores", []):
        S = oracle.score_matrix(c["gpu"], c["kernels"])
        assert S[i, j] == pytest.approx(v, abs=1e-12) and S[j, i] == pytest.approx(v, abs=1e-12)


def test_w2_every_order_equal_percentile_100():
    c = CASES["W2"]
    st = oracle.exhaustive_stats(c["gpu"], c["kernels"], 160)
    assert st["min"] == st["max"] == 160
    assert oracle.rank_outputs(st)["percentile"] == 100.0


@pytest.mark.parametrize("seed", range(10))
def test_heuristic_returns_permutation(seed):
    s = synth.random_set(seed, 3 + seed % 10, blk=(1, 200))
    h = oracle.heuristic(s.gpu, s.kernels)
    assert sorted(h) == list(range(s.n))


# ------------------------------------------------------------- Table 3 ---

def test_table3_output_arithmetic():
    with open(os.path.join(GOLD, "table3.json")) as f:
        t3 = json.load(f)
    for name, opt, worst, alg, _pct, speed, dev in t3["rows"]:
        st = dict(min=opt, max=worst, makespan=alg, n_total=720, n_worse=0, n_equal=720)
        out = oracle.rank_outputs(st)
        assert round(out["speedup_over_worst"], 3) == pytest.approx(speed, abs=1e-9), name
        digits = 3 if dev < 0.1 else 2
        assert round(100 * out["deviation_from_optimal"], digits) == pytest.approx(dev, abs=1e-9), name
    assert math.factorial(8) == t3["orders"]["8 kernels"]


# ------------------------------------------- duration sampled at placement ---

def test_placement_sampling_hand_traced():
    c = CASES["W1"]
    orders = [o for o, _ in c["makespans_at_placement"]]
    want = [m for _, m in c["makespans_at_placement"]]
    assert oracle.makespans_sampled(c["gpu"], c["kernels"], orders, True).tolist() == want
    assert oracle.makespans_sampled(c["gpu"], c["kernels"], orders, False).tolist() == \
        [m for _, m in c["makespans"]]


def test_placement_sampling_equals_burst_end_with_one_block_per_sm():
    # one block slot per SM: the totals at placement are the totals after the burst
    for seed in range(8):
        s = synth.random_set(800 + seed, 5, gpu=(6, 65536, 49152, 64, 1), blk=(1, 20))
        every = [list(p) for p in itertools.permutations(range(5))]
        assert (oracle.makespans_sampled(s.gpu, s.kernels, every, True) ==
                oracle.makespans_sampled(s.gpu, s.kernels, every, False)).all()


def test_placement_sampling_equals_burst_end_when_capacity_never_binds():
    # Ccap >= Bk * max c and Mcap >= Bk * max m: every duration is the alone time
    for seed in range(8):
        s = synth.random_set(810 + seed, 5, gpu=(6, 65536, 49152, 64, 8), blk=(4, 40), c=(1, 5000),
                             c_cap=8 * 5000, m_cap=8 * 5000 * 10)
        every = [list(p) for p in itertools.permutations(range(5))]
        assert (oracle.makespans_sampled(s.gpu, s.kernels, every, True) ==
                oracle.makespans_sampled(s.gpu, s.kernels, every, False)).all()


def test_default_makespan_is_burst_end_sampling():
    s = synth.gen_set("single8", 0)
    idx = np.arange(0, 40320, 997, dtype=np.uint64)
    orders = np.array([oracle.unrank(8, int(i)) for i in idx], dtype=np.int32)
    assert (oracle.makespans_sampled(s.gpu, s.kernels, orders, False) ==
            oracle.makespans_idx(s.gpu, s.kernels, idx)).all()


# ------------------------------------------------------ processor sharing ---

@pytest.mark.parametrize("name", ["P1", "P2"])
def test_processor_sharing_hand_traced(name):
    c = CASES[name]
    orders = [o for o, _ in c["makespans_ps"]]
    got = oracle.makespans_ps(c["gpu"], c["kernels"], orders)
    for g, (_, want) in zip(got.tolist(), c["makespans_ps"]):
        assert g == pytest.approx(want, rel=1e-12)


def test_processor_sharing_equals_duration_rule_when_capacity_never_binds():
    for seed in range(8):
        s = synth.random_set(820 + seed, 5, gpu=(6, 65536, 49152, 64, 8), blk=(4, 40), c=(1, 5000),
                            c_cap=8 * 5000, m_cap=8 * 5000 * 10)
        every = [list(p) for p in itertools.permutations(range(5))]
        assert (oracle.makespans_ps(s.gpu, s.kernels, every) ==
                oracle.makespans_sampled(s.gpu, s.kernels, every, False).astype(np.float64)).all()


def test_processor_sharing_one_wave_closed_form():
    # 16 identical blocks, 4 per SM, all start at 0 and end together at c * SumC / Ccap
    gpu = (4, 65536, 49152, 64, 4, 1500, 1 << 30)
    kern = [[1024, 0, 2, 16, 1000, 1]]
    assert oracle.makespans_ps(gpu, kern, [[0]])[0] == pytest.approx(1000 * 4000 / 1500, rel=1e-15)
    # the duration rule rounds the same end up
    assert oracle.makespan(gpu, kern, [0]) == math.ceil(1000 * 4000 / 1500)
