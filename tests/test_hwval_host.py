"""Host-side pieces of the hardware validation (no GPU): the rank correlation
against scipy's, tie handling, the model's per-block resource arithmetic and
the seeded kernel shapes."""
import numpy as np
import pytest

from paper_1511_07983_gb300 import hwval


def test_spearman_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.integers(0, 12, 200)          # many ties
        b = rng.normal(size=200) + 0.3 * a
        assert hwval.spearman(a, b) == pytest.approx(stats.spearmanr(a, b).statistic, abs=1e-12)


def test_rank_ties_take_mean_rank():
    assert hwval.rankdata([10, 20, 20, 5]).tolist() == [2.0, 3.5, 3.5, 1.0]
    assert hwval.spearman([1, 2, 3, 4], [10, 20, 30, 40]) == pytest.approx(1.0)
    assert hwval.spearman([1, 2, 3, 4], [4, 3, 2, 1]) == pytest.approx(-1.0)


def test_model_kernel_resources():
    # 256 threads = 8 warps; 19 registers/thread -> 608 per warp, rounded to 768
    assert hwval.model_kernel(256, 8192, 300, 12345.6, 19, 1024) == (8 * 768, 9216, 8, 300, 12345, 1)
    assert hwval.model_kernel(64, 0, 1, 0.2, 8, 1024) == (2 * 256, 1024, 2, 1, 1, 1)
    assert hwval.model_kernel(64, 0, 1, 7.9, 8, 1024, m_ns=790.2) == (512, 1024, 2, 1, 7, 790)


def test_shapes_are_seeded_and_in_range():
    a = hwval.draw_set(5, 6, 152, 200000)
    assert a == hwval.draw_set(5, 6, 152, 200000)
    assert a != hwval.draw_set(6, 6, 152, 200000)
    for kind, t, s, b, us in a:
        assert kind == 0
        assert t in (64, 128, 256, 512) and 0 <= s <= 200000 and 76 <= b <= 608 and 20 <= us <= 200
    m = hwval.draw_set(5, 6, 152, 200000, mixed=True)
    kinds = [x[0] for x in m]
    assert sorted(set(kinds)) == [0, 1] and all(kinds[i] != kinds[i + 1] for i in range(5))


def test_blocks_that_fit():
    lim = (152, 65536, 233472, 64, 32, 1024, 0)
    assert hwval.blocks_that_fit(128, 0, 16, lim) == 16          # warps: 64 / 4
    assert hwval.blocks_that_fit(64, 96 << 10, 16, lim) == 2      # shared memory
    assert hwval.blocks_that_fit(32, 0, 255, lim) == 8            # registers: 65536 / 8192
    assert hwval.blocks_that_fit(1024, 0, 64, lim) == 1


def test_iteration_calibration():
    assert hwval.calibrate_iters(100, 1 << 16, 0.2) == 32768
    assert hwval.calibrate_iters(1e9, 1 << 16, 0.2) == 1 << 24
    assert hwval.calibrate_iters(0, 1 << 16, 0.2) == 1


def test_dispatch_stats_on_synthetic_traces():
    # strict FIFO: kernel 1's blocks start after kernel 0's last start
    rec = np.array([[0, 9, 0, 0], [10, 19, 1, 0], [20, 29, 0, 1], [30, 39, 1, 1]], dtype=np.uint64)
    s = hwval.dispatch_order_stats(rec, [0, 1])
    assert s["overtaken"] == 0.0 and s["inversions"] == 0.0 and s["first_start_us"] == [0.0, 0.02]
    # issued as [1, 0]: both of kernel 0's blocks start... kernel 0 is second here
    s = hwval.dispatch_order_stats(rec, [1, 0])
    assert s["overtaken"] == 1.0 and s["inversions"] == 1.0
    # one of kernel 1's two blocks overtakes kernel 0's last block
    rec2 = np.array([[0, 9, 0, 0], [30, 39, 1, 0], [20, 29, 0, 1], [40, 49, 1, 1]], dtype=np.uint64)
    s = hwval.dispatch_order_stats(rec2, [0, 1])
    assert s["overtaken"] == 0.5 and s["inversions"] == 0.25
