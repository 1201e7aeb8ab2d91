"""The seeded input generator against its published definition and the
workload recipes it states (simulated GPUs, kernel counts, per-kernel ranges).
These inputs feed both the oracle and the CUDA path, so a drift here would move
every test and benchmark at once."""
import numpy as np
import pytest

from paper_1511_07983_gb300 import synth

SMALL13 = (13, 65536, 48 * 1024, 64, 16)
SMALL15 = (15, 65536, 48 * 1024, 64, 16)
BIG148 = (148, 65536, 228 * 1024, 64, 32)

# workload -> (allowed GPUs with their (blocks lo, hi, c lo, hi), kernel-count range)
RECIPES = {
    "single8": ({SMALL13: (8, 64, 1000, 20000)}, (8, 8)),
    "sets10": ({SMALL15: (15, 120, 1000, 20000)}, (10, 10)),
    "single12": ({BIG148: (100, 1000, 1000, 50000)}, (12, 12)),
    "batched": ({SMALL13: (15, 120, 1000, 20000), SMALL15: (15, 120, 1000, 20000),
                 BIG148: (100, 1000, 1000, 50000)}, (5, 10)),
    "train": ({SMALL13: (15, 120, 1000, 20000), SMALL15: (15, 120, 1000, 20000),
               BIG148: (100, 1000, 1000, 50000)}, (6, 12)),
    "large": ({SMALL13: (15, 120, 1000, 20000), SMALL15: (15, 120, 1000, 20000),
               BIG148: (100, 1000, 1000, 50000)}, (16, 24)),
}


def test_splitmix64_published_vector():
    # first output of SplitMix64 from state 0 in the reference implementation
    assert synth.SplitMix64(0).next() == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("workload", sorted(RECIPES))
def test_sets_follow_the_stated_recipe(workload):
    gpus, (n_lo, n_hi) = RECIPES[workload]
    count = 1 if workload.startswith("single") else 64
    seen_gpus, seen_n = set(), set()
    for i in range(count):
        s = synth.gen_set(workload, i)
        gpu = tuple(int(v) for v in s.gpu[:5])
        assert gpu in gpus, (workload, i, gpu)
        assert tuple(s.gpu[5:]) == (synth.C_CAP, synth.M_CAP)
        assert n_lo <= s.n <= n_hi
        seen_gpus.add(gpu)
        seen_n.add(s.n)
        b_lo, b_hi, c_lo, c_hi = gpus[gpu]
        for regs, smem, warps, blocks, c, m in np.asarray(s.kernels).tolist():
            threads = warps * 32
            assert threads in (128, 256, 512)
            assert regs % threads == 0 and 16 <= regs // threads <= 63
            assert smem in range(0, 24 * 1024 + 1, 4096)
            assert b_lo <= blocks <= b_hi and c_lo <= c <= c_hi
            # m = max(1, round(c / R)) with R in [0.1, 10]
            assert max(1, round(c / 10)) <= m <= round(c * 10)
            # every block fits an empty SM of its GPU
            assert regs <= gpu[1] and smem <= gpu[2] and warps <= gpu[3]
    if count > 1:   # the drawn choices vary across a workload's sets
        assert len(seen_gpus) == len(gpus)
        assert len(seen_n) > 1 or n_lo == n_hi


def test_ratio_is_log_uniform_on_the_stated_range():
    r = []
    for i in range(200):
        k = np.asarray(synth.gen_set("train", i).kernels)
        r += (k[:, 4] / k[:, 5]).tolist()
    lr = np.log10(np.asarray(r))
    assert lr.min() > -1.05 and lr.max() < 1.05
    # log-uniform on [0.1, 10]: log10 R roughly uniform on [-1, 1]
    hist, _ = np.histogram(lr, bins=4, range=(-1, 1))
    assert hist.min() > 0.8 * len(lr) / 4


def test_streams_are_deterministic_and_distinct():
    a, b = synth.gen_set("sets10", 3), synth.gen_set("sets10", 3)
    assert a.gpu == b.gpu and np.array_equal(a.kernels, b.kernels)
    assert not np.array_equal(synth.gen_set("sets10", 4).kernels, a.kernels)
    assert not np.array_equal(synth.gen_set("batched", 3, n=10).kernels, a.kernels)
    ids = synth.random_indices(5, 3628800, 1000)
    assert ids.dtype == np.uint64 and int(ids.max()) < 3628800
    assert np.array_equal(ids, synth.random_indices(5, 3628800, 1000))
    rows = synth.random_orders(7, 9, 200)
    assert all(sorted(r) == list(range(9)) for r in rows.tolist())
