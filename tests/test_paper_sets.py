"""Table 2's experiments as descriptor sets (no GPU): shapes as the paper
states them, every block fits an empty GTX580 SM, and the oracle's exhaustive
statistics are well formed."""
import math

import pytest

import oracle
from paper_1511_07983_gb300 import paper_sets


def test_six_experiments_with_paper_sizes():
    ex = paper_sets.experiments()
    assert list(ex) == ["EP-6-shm", "EP-6-grid", "BS-6-blk", "EpBs-6", "EpBs-6-shm", "EpBsEsSw-8"]
    assert [s.n for s in ex.values()] == [6, 6, 6, 6, 6, 8]   # 720 and 40,320 orders (Sec. 6)


@pytest.mark.parametrize("name", ["EP-6-shm", "EP-6-grid", "BS-6-blk", "EpBs-6", "EpBs-6-shm"])
def test_oracle_table3_columns(name):
    s = paper_sets.experiments()[name]
    h = oracle.heuristic(s.gpu, s.kernels)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h))
    assert st["n_total"] == math.factorial(s.n) and st["min"] > 0
    out = oracle.rank_outputs(st)
    assert 0 < out["percentile"] <= 100 and out["speedup_over_worst"] >= 1 and out["deviation_from_optimal"] >= 0
