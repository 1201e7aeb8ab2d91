"""GPU parity of the placement-time duration sampling (model variant) with the
oracle: explicit rows, the whole space and the ranked statistics, the W1 hand
trace, and the calls that require the default reading."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


def test_hand_trace(ko):
    c = {c["name"]: c for c in json.load(open(os.path.join(GOLD, "hand_traces.json")))["cases"]}["W1"]
    g = ko.Gpu(*c["gpu"][:5], c_cap=c["gpu"][5], m_cap=c["gpu"][6])
    ko.ko_set_sampling(g.h, ko.KO_SAMPLE_AT_PLACEMENT)
    for row in c["kernels"]:
        g.add_kernel(*row)
    rows = np.array([o for o, _ in c["makespans_at_placement"]], dtype=np.int8)
    assert np.asarray(g.eval_orders(orders=rows)).tolist() == [m for _, m in c["makespans_at_placement"]]


@pytest.mark.parametrize("case", ["single8", "sets10_sample", "single12_sample", "large_sample"])
def test_rows_match_oracle(ko, case):
    rng = np.random.default_rng(11)
    if case == "single8":
        s = synth.gen_set("single8", 0)
        rows = np.array([oracle.unrank(8, int(i)) for i in range(0, 40320, 7)], dtype=np.int8)
    else:
        s = synth.gen_set(case.split("_")[0], 1)
        rows = np.stack([rng.permutation(s.n) for _ in range(300)]).astype(np.int8)
    with ko.Gpu.from_set(s, sampling=ko.KO_SAMPLE_AT_PLACEMENT) as g:
        got = np.asarray(g.eval_orders(orders=rows))
    want = oracle.makespans_sampled(s.gpu, s.kernels, rows.astype(np.int32), True)
    assert (got == want).all()
    # the reading matters on these sets
    assert (want != oracle.makespans_sampled(s.gpu, s.kernels, rows.astype(np.int32), False)).any()


def test_whole_space_and_rank(ko):
    import torch
    s = synth.random_set(900, 7, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    every = np.array(list(__import__("itertools").permutations(range(7))), dtype=np.int32)
    want = oracle.makespans_sampled(s.gpu, s.kernels, every, True)
    with ko.Gpu.from_set(s, sampling=ko.KO_SAMPLE_AT_PLACEMENT) as g:
        out = torch.empty(math.factorial(7), dtype=torch.int64, device="cuda")
        g.eval_all(out)
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == want).all()
        h = g.heuristic_order()
        r, hist = g.rank_order(h, nbins=64)
    mh = int(oracle.makespans_sampled(s.gpu, s.kernels, np.array([h], dtype=np.int32), True)[0])
    assert (r["min"], r["max"], r["makespan"]) == (want.min(), want.max(), mh)
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == ((want < mh).sum(), (want == mh).sum(), (want > mh).sum())
    bins = (want - want.min()) * 64 // (want.max() - want.min() + 1)
    assert np.asarray(hist).tolist() == np.bincount(bins, minlength=64).tolist()


def test_calls_that_need_the_default_reading(ko):
    s = synth.random_set(901, 6, gpu=(13, 65536, 49152, 64, 16), blk=(8, 64))
    with ko.Gpu.from_set(s, sampling=ko.KO_SAMPLE_AT_PLACEMENT) as g:
        with pytest.raises(ko.KoError):
            g.local_search()
        with pytest.raises(ko.KoError):
            ko.ko_random_search(g, 1024)
        with pytest.raises(ko.KoError):
            ko.Batch([g], nbins=0)
        g.eval_orders(orders=np.arange(6, dtype=np.int8).reshape(1, 6))
        with pytest.raises(ko.KoError):
            ko.ko_set_sampling(g.h, ko.KO_SAMPLE_BURST_END)   # after the first evaluation


def test_variants_study_matches_oracle(ko):
    import itertools
    from paper_1511_07983_gb300 import hwval, study
    s = synth.gen_set("single8", 0)
    r = study.variants_set(s)
    every = np.array(list(itertools.permutations(range(8))), dtype=np.int32)   # lexicographic
    a = oracle.makespans_sampled(s.gpu, s.kernels, every, False)
    h = oracle.heuristic(s.gpu, s.kernels)
    ih = [i for i, p in enumerate(every.tolist()) if p == h][0]
    assert r["alg1_percentile_burst_end"] == pytest.approx(100.0 * (a >= a[ih]).sum() / a.size, abs=1e-12)
    for name, b in (("at_placement", oracle.makespans_sampled(s.gpu, s.kernels, every, True)),
                    ("processor_sharing", oracle.makespans_ps(s.gpu, s.kernels, every))):
        v = r[name]
        assert v["changed_orders"] == pytest.approx(float((a != b).mean()), abs=1e-15)
        assert v["spearman"] == pytest.approx(hwval.spearman(a, b), abs=1e-12)
        assert v["alg1_percentile"] == pytest.approx(100.0 * (b >= b[ih]).sum() / b.size, abs=1e-12)
        assert v["burst_end_optimum_percentile"] == pytest.approx(
            100.0 * (b >= b[int(np.argmin(a))]).sum() / b.size, abs=1e-12)
