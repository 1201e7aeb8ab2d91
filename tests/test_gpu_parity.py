"""GPU parity: every makespan, count and histogram bin from the CUDA path must
equal the oracle's exactly (integer work).  All calls go through the C ABI."""
import json
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


def _lehmer_sample(n, count, seed):
    total = math.factorial(n)
    idx = synth.random_indices(seed, total, count)
    return np.unique(np.concatenate([idx, np.array([0, total - 1], dtype=np.uint64)]))


def test_hand_traces(ko):
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "hand_traces.json")))["cases"]
    for c in cases:
        if "makespans" not in c:
            continue
        g = ko.Gpu(*c["gpu"][:5], c_cap=c["gpu"][5], m_cap=c["gpu"][6])
        for row in c["kernels"]:
            g.add_kernel(*row)
        orders = np.array([o for o, _ in c["makespans"]], dtype=np.int8)
        got = g.eval_orders(orders=orders)
        assert got.tolist() == [m for _, m in c["makespans"]], c["name"]


@pytest.mark.parametrize("workload,idx,count", [
    ("single8", 0, 3000), ("sets10", 0, 3000), ("sets10", 17, 3000), ("single12", 0, 1500),
    ("batched", 3, 2000), ("batched", 4, 2000), ("batched", 11, 2000)])
def test_eval_idx_matches_oracle(ko, workload, idx, count):
    s = synth.gen_set(workload, idx)
    ids = _lehmer_sample(s.n, count, 100 + idx)
    with ko.Gpu.from_set(s) as g:
        got = g.eval_orders(idx=ids)
    want = oracle.makespans_idx(s.gpu, s.kernels, idx=ids)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("workload,idx", [("large", 0), ("large", 1), ("large", 5), ("train", 2)])
def test_eval_explicit_orders_matches_oracle(ko, workload, idx):
    s = synth.gen_set(workload, idx)
    orders = synth.random_orders(7 + idx, s.n, 300).astype(np.int8)
    with ko.Gpu.from_set(s) as g:
        got = g.eval_orders(orders=orders)
    want = oracle.makespans_orders(s.gpu, s.kernels, orders.astype(np.int32))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", range(8))
def test_rank_order_small_sets_exhaustive(ko, seed):
    n = 3 + seed % 5
    s = synth.random_set(seed, n, blk=(1, 60), c=(50, 20000))
    h = oracle.heuristic(s.gpu, s.kernels)
    mh = oracle.makespan(s.gpu, s.kernels, h)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, mh, nbins=4096)
    with ko.Gpu.from_set(s) as g:
        r, hist = g.rank_order(None, nbins=4096)
    assert (r["min"], r["max"], r["makespan"]) == (st["min"], st["max"], mh)
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == (st["n_better"], st["n_equal"], st["n_worse"])
    assert r["n_total"] == math.factorial(n)
    assert np.array_equal(hist, st["hist"])
    ref = oracle.rank_outputs(st)
    for key in ("percentile", "percentile_strict", "speedup_over_worst", "deviation_from_optimal"):
        assert r[key] == pytest.approx(ref[key], rel=1e-15, abs=0)


def test_single8_full_space(ko):
    """All 40,320 orders of the N=8 / 13-SM set, element by element."""
    import torch
    s = synth.gen_set("single8")
    want = oracle.makespans_idx(s.gpu, s.kernels, first=0, count=40320)
    out = torch.empty(40320, dtype=torch.int64, device="cuda")
    with ko.Gpu.from_set(s) as g:
        g.eval_all(out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want)
        h = oracle.heuristic(s.gpu, s.kernels)
        r, hist = g.rank_order(h, nbins=4096)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h),
                                 makespans=want)
    assert (r["min"], r["max"], r["n_better"], r["n_equal"], r["n_worse"]) == \
        (st["min"], st["max"], st["n_better"], st["n_equal"], st["n_worse"])
    assert np.array_equal(hist, st["hist"])


def test_sets10_full_space_sampled(ko):
    """All 3,628,800 orders of an N=10 set on the GPU; oracle-checked on a
    sample of indices, histogram/counts checked for consistency and bounds."""
    import torch
    s = synth.gen_set("sets10", 0)
    total = math.factorial(10)
    out = torch.empty(total, dtype=torch.int64, device="cuda")
    with ko.Gpu.from_set(s) as g:
        g.eval_all(out)
        torch.cuda.synchronize()
        r, hist = g.rank_order(None, nbins=4096)
        lb, ub = g.bounds()
    ms = out.cpu().numpy()
    ids = _lehmer_sample(10, 4000, 5)
    assert np.array_equal(ms[ids.astype(np.int64)], oracle.makespans_idx(s.gpu, s.kernels, idx=ids))
    assert lb <= ms.min() and ms.max() <= ub
    mh = r["makespan"]
    assert (r["min"], r["max"]) == (int(ms.min()), int(ms.max()))
    assert (r["n_better"], r["n_equal"], r["n_worse"]) == \
        (int((ms < mh).sum()), int((ms == mh).sum()), int((ms > mh).sum()))
    assert np.array_equal(hist, oracle.histogram(ms, int(ms.min()), int(ms.max()), 4096))


def test_invariant_one_block_per_sm(ko):
    # Sec. 2: total blocks <= N_SM -> every order has the same makespan.
    ks = synth.random_set(3, 6, gpu=(40, 65536, 49152, 64, 16), blk=(1, 6)).kernels
    total = int(ks[:, 3].sum())
    s = synth.KernelSet(gpu=(total, 65536, 49152, 64, 16, 32768, 32768), kernels=ks)
    with ko.Gpu.from_set(s) as g:
        r, _ = g.rank_order(None, nbins=16)
    assert r["min"] == r["max"] == oracle.makespan(s.gpu, ks, list(range(6)))


def test_invariant_identical_kernels(ko):
    # Sec. 3: identical kernels differing only in N_tblk -> order does not matter.
    ks = synth.random_set(9, 7, blk=(1, 60)).kernels
    ks[:, [0, 1, 2, 4, 5]] = ks[0, [0, 1, 2, 4, 5]]
    s = synth.KernelSet(gpu=(13, 65536, 49152, 64, 16, 32768, 32768), kernels=ks)
    with ko.Gpu.from_set(s) as g:
        r, hist = g.rank_order(None, nbins=64)
    assert r["min"] == r["max"] and hist[0] == math.factorial(7)


def test_edge_cases(ko):
    import torch
    # single kernel
    s = synth.random_set(1, 1, blk=(50, 50))
    with ko.Gpu.from_set(s) as g:
        r, hist = g.rank_order(None, nbins=8)
        assert r["n_total"] == 1 and r["percentile"] == 100.0 and hist.sum() == 1
        assert g.eval_orders(idx=np.zeros(1, dtype=np.uint64))[0] == oracle.makespan(s.gpu, s.kernels, [0])
        # empty request
        assert g.eval_orders(idx=np.zeros(0, dtype=np.uint64)).shape == (0,)
    # invalid rows give -1, valid rows still evaluate
    s = synth.random_set(2, 4)
    with ko.Gpu.from_set(s) as g:
        rows = np.array([[0, 1, 2, 3], [0, 0, 2, 3], [0, 1, 2, 9], [3, 2, 1, 0]], dtype=np.int8)
        got = g.eval_orders(orders=rows)
        assert got[1] == -1 and got[2] == -1
        assert got[0] == oracle.makespan(s.gpu, s.kernels, [0, 1, 2, 3])
        assert got[3] == oracle.makespan(s.gpu, s.kernels, [3, 2, 1, 0])
        # device buffers in and out on the current torch stream
        d_rows = torch.from_numpy(rows).cuda()
        d_out = torch.empty(4, dtype=torch.int64, device="cuda")
        g.eval_orders(orders=d_rows, out=d_out)
        torch.cuda.synchronize()
        assert d_out.cpu().numpy().tolist() == got.tolist()
        # rank of an invalid order is rejected
        with pytest.raises(ko.KoError):
            g.rank_order([0, 0, 1, 2], nbins=8)
    # N = 13 is beyond the exhaustive limit
    s = synth.random_set(3, 13)
    with ko.Gpu.from_set(s) as g:
        with pytest.raises(ko.KoError) as e:
            g.rank_order(None, nbins=8)
        assert e.value.code == -3


def test_non_power_of_two_capacities(ko):
    s = synth.random_set(4, 6, blk=(5, 80), c_cap=3000, m_cap=7000)
    h = oracle.heuristic(s.gpu, s.kernels)
    st = oracle.exhaustive_stats(s.gpu, s.kernels, oracle.makespan(s.gpu, s.kernels, h), nbins=512)
    with ko.Gpu.from_set(s) as g:
        r, hist = g.rank_order(h, nbins=512)
    assert (r["min"], r["max"], r["n_equal"]) == (st["min"], st["max"], st["n_equal"])
    assert np.array_equal(hist, st["hist"])


def test_determinism(ko):
    s = synth.gen_set("sets10", 3)
    ids = _lehmer_sample(10, 5000, 1)
    with ko.Gpu.from_set(s) as g:
        a = g.eval_orders(idx=ids)
        b = g.eval_orders(idx=ids)
    assert np.array_equal(a, b)


def test_out_of_range_index_is_invalid(ko):
    s = synth.random_set(6, 5)
    ids = np.array([0, 119, 120, 10 ** 12, 5], dtype=np.uint64)
    with ko.Gpu.from_set(s) as g:
        got = g.eval_orders(idx=ids)
        g.configure(simple_only=True)
        got_simple = g.eval_orders(idx=ids)
    want = oracle.makespans_idx(s.gpu, s.kernels, idx=np.array([0, 119, 5], dtype=np.uint64))
    assert got[2] == -1 and got[3] == -1 and got_simple[2] == -1 and got_simple[3] == -1
    assert [got[0], got[1], got[4]] == want.tolist() == [got_simple[0], got_simple[1], got_simple[4]]
