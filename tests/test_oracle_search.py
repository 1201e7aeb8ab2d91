"""Pins for the oracle's Algorithm 1 footprint readings and its exact local
search (no GPU).

The expectations come from outside the functions under test: a hand trace
(tests/golden/hand_traces.json, case W5), the reduction of the two footprint
readings to one another when no kernel has more blocks than there are SMs,
the neighbourhood built independently here from itertools and list
operations, brute force over all N! orders for small N, and the fact that for
N = 3 the swap-and-move neighbourhood of an order is every other order.
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


def _case(name):
    with open(os.path.join(GOLD, "hand_traces.json")) as f:
        return {c["name"]: c for c in json.load(f)["cases"]}[name]


def _neighbours(p, moves):
    """All swap neighbours (pairs i < j in lexicographic order), then the move
    neighbours (from-major, destination ascending), built with list ops."""
    n = len(p)
    out = []
    for i, j in itertools.combinations(range(n), 2):
        q = list(p)
        q[i], q[j] = q[j], q[i]
        out.append(q)
    if moves:
        for a in range(n):
            for b in range(n):
                if a == b:
                    continue
                q = list(p)
                v = q.pop(a)
                q.insert(b, v)
                out.append(q)
    return out


def _small_sets():
    out = []
    for seed in range(6):
        out.append(synth.random_set(500 + seed, 5 + seed % 3, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64)))
    out.append(synth.gen_set("single8", 0))
    return out


# ------------------------------------------------------- footprint readings ---

def test_per_block_reading_hand_traced():
    c = _case("W5")
    assert oracle.heuristic_fp(c["gpu"], c["kernels"], per_block=False) == c["heuristic"]
    assert oracle.heuristic_fp(c["gpu"], c["kernels"], per_block=True) == c["heuristic_per_block"]


def test_readings_agree_when_no_kernel_exceeds_one_block_per_sm():
    # ceil(N_tblk / N_SM) = 1 for every kernel: both readings give the same footprints
    for seed in range(10):
        s = synth.random_set(600 + seed, 7, gpu=(64, 65536, 233472, 64, 32), blk=(1, 64))
        assert oracle.heuristic_fp(s.gpu, s.kernels, True) == oracle.heuristic_fp(s.gpu, s.kernels, False)
        assert oracle.heuristic_fp(s.gpu, s.kernels, False) == oracle.heuristic(s.gpu, s.kernels)


def test_per_block_reading_is_a_permutation():
    for s in _small_sets():
        o = oracle.heuristic_fp(s.gpu, s.kernels, True)
        assert sorted(o) == list(range(s.n))


# ------------------------------------------------------------ local search ---

@pytest.mark.parametrize("moves", [False, True])
def test_result_is_a_local_optimum(moves):
    for s in _small_sets():
        start = oracle.heuristic(s.gpu, s.kernels)
        order, ms, steps, evals = oracle.local_search(s.gpu, s.kernels, start, moves=moves)
        assert sorted(order) == list(range(s.n))
        assert ms == oracle.makespan(s.gpu, s.kernels, order)
        assert ms <= oracle.makespan(s.gpu, s.kernels, start)
        nb = np.array(_neighbours(order, moves), dtype=np.int32)
        assert oracle.makespans_orders(s.gpu, s.kernels, nb).min() >= ms
        # one full sweep per step plus the final sweep that found no improvement
        nq = math.comb(s.n, 2) + (s.n * (s.n - 1) if moves else 0)
        assert evals == 1 + (steps + 1) * nq


@pytest.mark.parametrize("moves", [False, True])
def test_each_step_takes_the_first_best_neighbour(moves):
    s = synth.random_set(510, 7, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    cur = oracle.heuristic(s.gpu, s.kernels)
    cur_ms = oracle.makespan(s.gpu, s.kernels, cur)
    for it in range(1, 30):
        nb = _neighbours(cur, moves)
        ms = oracle.makespans_orders(s.gpu, s.kernels, np.array(nb, dtype=np.int32))
        q = int(np.argmin(ms))  # first minimum
        order, got, steps, _ = oracle.local_search(s.gpu, s.kernels, oracle.heuristic(s.gpu, s.kernels),
                                                   moves=moves, max_iters=it)
        if ms[q] >= cur_ms:
            assert (order, got, steps) == (cur, cur_ms, it - 1)
            break
        cur, cur_ms = nb[q], int(ms[q])
        assert (order, got, steps) == (cur, cur_ms, it)


def test_three_kernels_reach_the_global_optimum():
    # for N = 3 the swaps and moves of an order cover all five other orders
    for seed in range(12):
        s = synth.random_set(520 + seed, 3, gpu=(4, 65536, 49152, 64, 8), blk=(4, 40))
        allms = {p: oracle.makespan(s.gpu, s.kernels, list(p)) for p in itertools.permutations(range(3))}
        best = min(allms.values())
        for p in allms:
            _, ms, _, _ = oracle.local_search(s.gpu, s.kernels, list(p), moves=True)
            assert ms == best


def test_two_kernels_swap_only():
    for seed in range(8):
        s = synth.random_set(540 + seed, 2, gpu=(4, 65536, 49152, 64, 8), blk=(4, 40))
        a = oracle.makespan(s.gpu, s.kernels, [0, 1])
        b = oracle.makespan(s.gpu, s.kernels, [1, 0])
        order, ms, steps, evals = oracle.local_search(s.gpu, s.kernels, [0, 1], moves=False)
        assert ms == min(a, b)
        assert order == ([1, 0] if b < a else [0, 1])
        assert steps == (1 if b < a else 0)


def test_single_kernel_and_zero_iterations():
    s = synth.random_set(550, 1, gpu=(4, 65536, 49152, 64, 8), blk=(4, 40))
    assert oracle.local_search(s.gpu, s.kernels, [0]) == ([0], oracle.makespan(s.gpu, s.kernels, [0]), 0, 1)
    s = synth.random_set(551, 6, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    st = [5, 4, 3, 2, 1, 0]
    assert oracle.local_search(s.gpu, s.kernels, st, max_iters=0) == (st, oracle.makespan(s.gpu, s.kernels, st), 0, 1)


def test_never_worse_than_exhaustive_optimum():
    s = synth.random_set(560, 7, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    every = oracle.makespans_idx(s.gpu, s.kernels, np.arange(math.factorial(7), dtype=np.uint64))
    _, ms, _, _ = oracle.local_search(s.gpu, s.kernels, oracle.heuristic(s.gpu, s.kernels), moves=True)
    assert every.min() <= ms <= every.max()
