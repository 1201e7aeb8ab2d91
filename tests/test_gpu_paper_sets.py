"""Table 2's experiments on the GPU: exhaustive statistics, histogram and the
heuristic's rank equal the oracle's for all six sets."""
import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import paper_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


@pytest.mark.parametrize("name", list(paper_sets.experiments()))
def test_table2_sets_match_oracle(ko, name):
    s = paper_sets.experiments()[name]
    h = oracle.heuristic(s.gpu, s.kernels)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h), nbins=4096)
    with ko.Gpu.from_set(s) as g:
        assert g.heuristic_order().tolist() == h
        r, hist = g.rank_order(None, nbins=4096)
    assert (r["min"], r["max"], r["makespan"]) == (st["min"], st["max"], st["makespan"])
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == (st["n_better"], st["n_equal"], st["n_worse"])
    assert np.array_equal(hist, st["hist"])
