"""The one-thread simulator's state machine (ko_lane_sim.cuh, compiled for the
host by tests/lane_host_harness.cpp and driven as lane_kernel drives it)
against the hand-traced makespans and the oracle, on the CPU.

The device kernel runs the same header; these tests pin its dispatch, release,
duration and burst logic -- and the depth-first walk with saved and restored
node states -- without a GPU: hand traces of Sec. 2's dispatch rule, whole
spaces of small sets (N <= 8) and of subtrees of larger ones, and seeded
orders of the N = 12 benchmark set, all against oracle/ element by element."""
import json
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    import ctypes
    so = str(tmp_path_factory.mktemp("lane_host") / "liblanehost.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_1511_07983_gb300", "csrc"),
                    os.path.join(HERE, "lane_host_harness.cpp"), "-o", so], check=True)
    lib = ctypes.CDLL(so)
    p = ctypes.c_void_p
    lib.lane_host_orders.argtypes = [p, p, ctypes.c_int, p, ctypes.c_int64, p]
    lib.lane_host_subtree.argtypes = [p, p, ctypes.c_int, p, ctypes.c_int, p]

    def orders(s, rows):
        gpu = np.ascontiguousarray(s.gpu, dtype=np.int64)
        k = np.ascontiguousarray(s.kernels, dtype=np.int64)
        rows = np.ascontiguousarray(rows, dtype=np.int8)
        out = np.empty(rows.shape[0], dtype=np.int64)
        assert lib.lane_host_orders(gpu.ctypes.data, k.ctypes.data, s.n, rows.ctypes.data,
                                    rows.shape[0], out.ctypes.data) == 0
        return out

    def subtree(s, prefix):
        gpu = np.ascontiguousarray(s.gpu, dtype=np.int64)
        k = np.ascontiguousarray(s.kernels, dtype=np.int64)
        pre = np.ascontiguousarray(prefix, dtype=np.int8)
        out = np.empty(math.factorial(s.n - len(prefix)), dtype=np.int64)
        assert lib.lane_host_subtree(gpu.ctypes.data, k.ctypes.data, s.n, pre.ctypes.data, len(prefix),
                                     out.ctypes.data) == 0
        return out

    return orders, subtree


def _first_index(n, prefix):
    rest = [k for k in range(n) if k not in prefix]
    return oracle.rank(list(prefix) + rest)


def test_hand_traced_makespans(harness):
    orders, _ = harness
    cases = json.load(open(os.path.join(HERE, "golden", "hand_traces.json")))["cases"]
    checked = 0
    for c in cases:
        if "makespans" not in c:
            continue
        s = synth.KernelSet(gpu=tuple(c["gpu"]), kernels=np.array(c["kernels"], dtype=np.int64))
        for order, want in c["makespans"]:
            assert int(orders(s, np.array([order]))[0]) == want, (c["name"], order)
            checked += 1
    assert checked >= 5


def test_single8_full_space_both_walks(harness):
    orders, subtree = harness
    s = synth.gen_set("single8")
    n = s.n
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(n))
    got = subtree(s, [])
    assert np.array_equal(got, want)
    rows = np.array([oracle.unrank(n, k) for k in range(0, math.factorial(n), 97)], dtype=np.int8)
    assert np.array_equal(orders(s, rows), want[::97])


@pytest.mark.parametrize("seed", range(12))
def test_random_small_sets_full_space(harness, seed):
    # small GPUs, odd capacities (the divide path of the duration rule), tight limits
    _, subtree = harness
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    # every block of the generator (<= 32,256 registers, 24 KB, 16 warps) fits an empty SM
    gpu = (int(rng.integers(1, 7)), int(rng.choice([32768, 49152, 65536])), int(rng.choice([24576, 32768, 49152])),
           int(rng.choice([16, 32, 48, 64])), int(rng.integers(1, 17)), 1 << 15 if seed % 2 else 30000 + seed,
           1 << 15 if seed % 3 else 20000 + seed)
    s = synth.random_set(1000 + seed, n, gpu=gpu[:5], blk=(1, 24), c=(1, 5000), c_cap=gpu[5], m_cap=gpu[6])
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=math.factorial(n))
    got = subtree(s, [])
    ok = got >= 0
    assert ok.mean() > 0.9
    assert np.array_equal(got[ok], want[ok])


@pytest.mark.parametrize("set_idx,prefix", [(0, [3, 1, 4, 0]), (5, [9, 2]), (17, [0, 1, 2, 3, 4])])
def test_sets10_subtrees(harness, set_idx, prefix):
    _, subtree = harness
    s = synth.gen_set("sets10", set_idx)
    count = math.factorial(s.n - len(prefix))
    want = oracle.makespans_idx(s.gpu, s.kernels, first=_first_index(s.n, prefix), count=count)
    got = subtree(s, prefix)
    assert (got >= 0).all()
    assert np.array_equal(got, want)


def test_single12_seeded_orders_and_a_subtree(harness):
    # the benchmark set: seeded orders from scratch, and one 5-kernel subtree (120 orders) walked
    # with saved node states as a work item of the benchmark's launch is
    orders, subtree = harness
    s = synth.gen_set("single12")
    rows = synth.random_orders(12, s.n, 1500)
    got = orders(s, rows)
    want = oracle.makespans_orders(s.gpu, s.kernels, rows)
    ok = got >= 0
    assert ok.mean() > 0.97   # the rest overflow the 14-run / 56-slot state and are handed on
    assert np.array_equal(got[ok], want[ok])
    prefix = [int(v) for v in rows[7][:7]]
    got = subtree(s, prefix)
    want = oracle.makespans_idx(s.gpu, s.kernels, first=_first_index(s.n, prefix), count=120)
    ok = got >= 0
    assert np.array_equal(got[ok], want[ok])


def test_batched_workload_sets(harness):
    # the mixed batch's sets (N 5..10 on 13-, 15- and 148-SM GPUs): whole spaces up to N = 7,
    # a 120-order subtree above that
    _, subtree = harness
    seen = set()
    for i in range(40):
        s = synth.gen_set("batched", i)
        prefix = [] if s.n <= 7 else list(range(s.n - 5))
        count = math.factorial(s.n - len(prefix))
        want = oracle.makespans_idx(s.gpu, s.kernels, first=_first_index(s.n, prefix), count=count)
        got = subtree(s, prefix)
        ok = got >= 0
        assert ok.mean() > 0.9, i
        assert np.array_equal(got[ok], want[ok]), i
        seen.add(s.gpu[0])
    assert seen == {13, 15, 148}
