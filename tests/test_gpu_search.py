"""GPU exact local search against the oracle's: the same walk (order, makespan,
steps and orders simulated) from the Algorithm 1 order and from other starts,
with and without move neighbours, on small and large simulated GPUs."""
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


def _check(ko, s, start, moves, max_iters=1 << 20):
    with ko.Gpu.from_set(s) as g:
        order, ms, steps, evals, t = g.local_search(start=start, moves=moves, max_iters=max_iters)
    st = start if start is not None else oracle.heuristic(s.gpu, s.kernels)
    want = oracle.local_search(s.gpu, s.kernels, st, moves=moves, max_iters=max_iters)
    assert (order.tolist(), ms, steps, evals) == want
    assert t >= 0.0
    return want


@pytest.mark.parametrize("moves", [False, True])
def test_from_heuristic_small_sets(ko, moves):
    for seed in range(6):
        s = synth.random_set(700 + seed, 6 + seed % 4, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
        _check(ko, s, None, moves)
    _check(ko, synth.gen_set("single8", 0), None, moves)


def test_from_other_starts(ko):
    s = synth.gen_set("sets10", 3)
    rng = np.random.default_rng(7)
    for _ in range(4):
        _check(ko, s, rng.permutation(s.n).tolist(), True)
    _check(ko, s, list(range(s.n))[::-1], False)


def test_large_gpu_twelve_kernels(ko):
    # the 148-SM, 12-kernel set, walked to its local optimum and cut short
    s = synth.gen_set("single12", 0)
    _check(ko, s, None, False)
    _check(ko, s, None, True)
    _check(ko, s, None, True, max_iters=2)


def test_twenty_kernels(ko):
    s = synth.random_set(720, 20, gpu=(15, 65536, 49152, 64, 16), blk=(15, 120))
    _check(ko, s, None, True)


def test_degenerate_sizes(ko):
    s1 = synth.random_set(730, 1, gpu=(4, 65536, 49152, 64, 8), blk=(4, 40))
    _check(ko, s1, None, True)
    s2 = synth.random_set(731, 2, gpu=(4, 65536, 49152, 64, 8), blk=(4, 40))
    _check(ko, s2, [1, 0], False)
    s3 = synth.random_set(732, 6, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    _check(ko, s3, [5, 4, 3, 2, 1, 0], True, max_iters=0)


def test_rejects_bad_start(ko):
    s = synth.random_set(733, 5, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    with ko.Gpu.from_set(s) as g:
        for bad in ([0, 0, 1, 2, 3], [0, 1, 2, 3, 5], [-1, 0, 1, 2, 3]):
            with pytest.raises(ko.KoError):
                g.local_search(start=bad)
        with pytest.raises(ko.KoError):
            g.local_search(max_iters=-1)


def test_study_ranks_are_consistent(ko):
    from paper_1511_07983_gb300 import study
    for s in (synth.gen_set("sets10", 0), synth.gen_set("single8", 0)):
        r = study.rank_set(s)
        every = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=__import__("math").factorial(s.n))
        assert r["optimum"] == every.min() and r["worst"] == every.max()
        for k in study.STRATEGIES:
            m = r[k]["makespan"]
            assert r[k]["percentile"] == pytest.approx(100.0 * (every >= m).sum() / every.size, abs=1e-12)
            assert r[k]["optimal"] == (m == every.min())
        # local search from Algorithm 1 never ends above its start
        assert r["ls_swap_from_alg1"]["makespan"] <= r["alg1_per_sm"]["makespan"]
        assert r["ls_swap_move_from_alg1"]["makespan"] <= r["alg1_per_sm"]["makespan"]


def test_large_gpu_twenty_four_kernels(ko):
    s = synth.gen_set("large", 2)          # N = 24 on one of the three GPUs
    _check(ko, s, None, False, max_iters=3)
