"""GPU checks of the surrogate: encoder equal to the oracle's, forward and
gradients within BF16 tolerances of the oracle (FP64 accumulation, same
rounding points), Adam, training, and proposals confirmed by the exact oracle."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
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


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"],
                           p["w4"], p["b4"]]).astype(np.float32)


def _split(flat):
    out, off = {}, 0
    for k, shape in (("W1", (192, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
                     ("W3", (256, 256)), ("b3", (256,)), ("w4", (256,)), ("b4", (1,))):
        n = int(np.prod(shape))
        out[k] = flat[off:off + n].reshape(shape)
        off += n
    return out


def _params(seed):
    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed + 10)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(256) * 0.05).astype(np.float32)
    p["b4"] = np.array([0.2], dtype=np.float32)
    return p


def _features(seed, B):
    s = synth.gen_set("large", seed)
    lb, _ = oracle.bounds(s.gpu, s.kernels)
    x = mlp.encode(mlp.kernel_features(s.gpu, s.kernels), mlp.global_features(s.gpu, s.n, lb),
                   synth.random_orders(seed, s.n, B))
    return mlp.bf16(x)


def test_encoder_matches_oracle(ko):
    for i in range(6):
        s = synth.gen_set("large" if i % 2 else "train", i)
        orders = synth.random_orders(i, s.n, 50)
        lb, _ = oracle.bounds(s.gpu, s.kernels)
        want = mlp.bf16(mlp.encode(mlp.kernel_features(s.gpu, s.kernels),
                                   mlp.global_features(s.gpu, s.n, lb), orders))
        with ko.Gpu.from_set(s) as g:
            got = ko.ko_model_encode(g, orders)
        assert np.array_equal(got, want), i


def test_forward_matches_oracle(ko):
    p = _params(1)
    x = _features(2, 512)
    m = ko.Model()
    m.set_params(_flat(p))
    y = m.predict(x)
    want, _ = mlp.forward(p, x)
    err = np.abs(y - want)
    assert err.max() <= 2e-2 * max(1.0, np.abs(want).max()), err.max()
    assert np.quantile(err, 0.99) <= 1e-2 * max(1.0, np.abs(want).max())


def test_gradients_match_oracle(ko):
    p = _params(3)
    x = _features(4, 256)
    t = np.random.default_rng(5).standard_normal(256).astype(np.float32)
    m = ko.Model()
    m.set_params(_flat(p))
    g, loss = m.grad(x, t)
    y, cache = mlp.forward(p, x)
    want = mlp.backward(p, cache, y, t)
    assert loss == pytest.approx(mlp.loss(y, t), rel=1e-2)
    got = _split(g)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        rel = np.linalg.norm(got[k] - want[k]) / max(np.linalg.norm(want[k]), 1e-12)
        assert rel <= 2e-2, (k, rel)


def test_adam_step_matches_oracle_update(ko):
    p = _params(6)
    x = _features(7, 128)
    t = np.random.default_rng(8).standard_normal(128).astype(np.float32)
    m = ko.Model()
    m.set_params(_flat(p))
    g, _ = m.grad(x, t)
    m.train_step(x, t, lr=1e-3)
    after = _split(m.get_params())
    q = {k: v.copy() for k, v in p.items()}
    mlp.adam(q, _split(g.astype(np.float64)), {}, step=1, lr=1e-3)
    for k in q:
        assert np.allclose(after[k], q[k], atol=1e-6, rtol=1e-5), k


def test_training_lowers_loss_and_ranks_orders(ko):
    train_sets = [synth.gen_set("train", i) for i in range(24)]
    gpus = [ko.Gpu.from_set(s) for s in train_sets]
    m = ko.Model(seed=3)
    curve = m.train(gpus, pairs_per_set=4096, steps=300, batch=1024, lr=1e-3, seed=5)
    assert np.all(np.isfinite(curve))
    assert curve[-30:].mean() < 0.5 * curve[:10].mean()


def test_propose_and_random_search_are_exact(ko):
    s = synth.gen_set("large", 3)
    m = ko.Model(seed=1)
    with ko.Gpu.from_set(s) as g:
        order, ms, t_ms = m.propose(g, n_cand=70000, top_k=256, seed=9)
        assert sorted(order.tolist()) == list(range(s.n)) and t_ms > 0
        assert ms == oracle.makespan(s.gpu, s.kernels, order.tolist())
        ro, rms, _ = ko.ko_random_search(g, 5000, seed=4)
        assert sorted(ro.tolist()) == list(range(s.n))
        assert rms == oracle.makespan(s.gpu, s.kernels, ro.tolist())


def test_guided_search_is_exact_and_not_worse_than_screening(ko):
    s = synth.gen_set("large", 5)
    m = ko.Model(seed=2)
    with ko.Gpu.from_set(s) as g:
        _, screened, _ = m.search(g, n_cand=70000, top_k=256, rounds=0, beam=4, seed=3)
        order, ms, t_ms = m.search(g, n_cand=70000, top_k=256, rounds=3, beam=4, seed=3)
    assert sorted(order.tolist()) == list(range(s.n)) and t_ms > 0
    assert ms == oracle.makespan(s.gpu, s.kernels, order.tolist())
    assert ms <= screened      # the beam always keeps the screening's best


def test_tcgen05_forward_matches_mma_and_oracle(ko):
    p = _params(11)
    x = _features(12, 1024)
    m = ko.Model()
    m.set_params(_flat(p))
    m.set_tc(False)
    y_mma = m.predict(x)
    m.set_tc(True)
    y_tc = m.predict(x)
    assert np.allclose(y_tc, y_mma, rtol=1e-5, atol=1e-5)
    want, _ = mlp.forward(p, x)
    assert np.abs(y_tc - want).max() <= 2e-2 * max(1.0, np.abs(want).max())
    s = synth.gen_set("large", 4)
    with ko.Gpu.from_set(s) as g:
        order, ms, _ = m.search(g, n_cand=65536, top_k=128, rounds=2, beam=4, seed=1)
    assert ms == oracle.makespan(s.gpu, s.kernels, order.tolist())


def test_chunk_size_does_not_change_results(ko):
    s = synth.gen_set("large", 3)
    m = ko.Model(seed=9)
    out = []
    with ko.Gpu.from_set(s) as g:
        for rows in (65536, 1 << 18, 3 * 1024):
            m.set_chunk(rows)
            o1, ms1, _ = m.propose(g, n_cand=200000, top_k=256, seed=4)
            o2, ms2, _ = m.search(g, n_cand=100000, top_k=128, rounds=2, beam=4, seed=5)
            out.append((o1.tolist(), ms1, o2.tolist(), ms2))
        for bad in (1000, 0, 1 << 23):
            with pytest.raises(ko.KoError):
                m.set_chunk(bad)
    m.close()
    assert out[0] == out[1] == out[2]


@pytest.mark.parametrize("B", [256, 1024, 4096])
def test_tcgen05_training_gradients(ko, B):
    # weight gradients split over B / 256 K slices (W1's 192 rows padded to 256), input gradients
    # and the training forward with transposed copies, against the oracle and the mma.sync path
    p = _params(11)
    x = _features(12, B)
    t = np.random.default_rng(13).standard_normal(B).astype(np.float32)
    m = ko.Model()
    m.set_params(_flat(p))
    m.set_tc_train(True)
    g_tc, loss_tc = m.grad(x, t)
    g_tc2, _ = m.grad(x, t)
    m.set_tc_train(False)
    g_mma, loss_mma = m.grad(x, t)
    m.close()
    # the weight gradients' split-K slices are summed in a fixed order: bit-identical runs
    # (bias gradients are summed with atomics in the shared elementwise kernels)
    a, b = _split(g_tc), _split(g_tc2)
    for k in ("W1", "W2", "W3"):
        assert (a[k] == b[k]).all(), k
    assert loss_tc == pytest.approx(loss_mma, rel=1e-3)
    y, cache = mlp.forward(p, x)
    want = mlp.backward(p, cache, y, t)
    got, ref = _split(g_tc), _split(g_mma)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        nrm = max(np.linalg.norm(want[k]), 1e-12)
        assert np.linalg.norm(got[k] - want[k]) / nrm <= 2e-2, (k, "oracle")
        assert np.linalg.norm(got[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-12) <= 1e-2, (k, "mma")


def test_tcgen05_training_run(ko):
    sets = [synth.gen_set("train", 2000 + i) for i in range(8)]
    curves = []
    for tc in (True, False):
        gpus = [ko.Gpu.from_set(s) for s in sets]
        m = ko.Model(seed=3)
        m.set_tc_train(tc)
        curves.append(m.train(gpus, pairs_per_set=4096, steps=200, batch=4096, lr=1e-3, seed=5))
        m.close()
        for g in gpus:
            g.close()
    a, b = (float(np.mean(c[-20:])) for c in curves)
    assert a < float(np.mean(curves[0][:5]))      # it learns
    assert a == pytest.approx(b, rel=0.1)         # like the mma.sync path


def test_training_is_reproducible(ko):
    """Two trainings with the same seed give bit-identical weights and loss
    curves (the bias gradients are summed per block in a fixed order)."""
    sets = [synth.gen_set("train", 2000 + i) for i in range(24)]
    out = []
    for _ in range(2):
        gpus = [ko.Gpu.from_set(s) for s in sets]
        m = ko.Model(seed=3)
        curve = m.train(gpus, pairs_per_set=2048, steps=60, batch=1024, lr=1e-3, seed=5)
        out.append((curve.copy(), m.get_params().copy()))
        m.close()
        for g in gpus:
            g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_surrogate_trained_on_small_sets_beats_plain_search(ko):
    """The learned part's gain over the method without it, as specified: a
    network trained only on orders of enumerable sets (N 6..12, 10.0M pairs
    labelled exactly by the simulator) guides the search on 32 held-out sets
    with N 16..24; on a majority of them its best order (every candidate
    rescored exactly) has a lower exact makespan than plain uniform random
    search given the same measured GPU time.  Exact local search from
    Algorithm 1's order is run beside them and must stay exact."""
    train = [synth.gen_set("train", 1000 + i) for i in range(1221)]
    assert max(s.n for s in train) <= 12
    gpus = [ko.Gpu.from_set(s) for s in train]
    model = ko.Model(seed=7)
    model.train(gpus, pairs_per_set=8192, steps=2500, batch=4096, lr=1e-3, seed=7)
    for g in gpus:
        g.close()
    lower = higher = 0
    for j in range(32):
        s = synth.gen_set("large", j)
        assert 16 <= s.n <= 24
        with ko.Gpu.from_set(s) as g:
            order, best, s_ms = model.search(g, n_cand=1 << 20, top_k=1024, rounds=12, beam=8, seed=7 + j)
            assert sorted(order) == list(range(s.n))
            assert best == oracle.makespan(s.gpu, s.kernels, list(order))
            _, _, cal_ms = ko.ko_random_search(g, 1 << 16, seed=99 + j)
            n_plain = max(1, int((1 << 16) * s_ms / max(cal_ms, 1e-3)))
            p_order, p_best, _ = ko.ko_random_search(g, n_plain, seed=107 + j)
            assert p_best == oracle.makespan(s.gpu, s.kernels, list(p_order))
            l_order, l_best, *_ = g.local_search(moves=True)
            assert l_best == oracle.makespan(s.gpu, s.kernels, list(l_order))
        lower += best < p_best
        higher += best > p_best
    model.close()
    assert lower > 16 and lower > higher, (lower, higher)
