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
        # element by element: the oracle rounds at the same points, so every entry stays within
        # 1e-3 of the tensor's largest magnitude (measured: below 1e-4)
        assert np.abs(got[k] - want[k]).max() <= 1e-3 * np.abs(want[k]).max(), k


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
    m.set_polish(0)
    with ko.Gpu.from_set(s) as g:
        _, screened, _ = m.search(g, n_cand=70000, top_k=256, rounds=0, beam=4, seed=3)
        order, ms, t_ms = m.search(g, n_cand=70000, top_k=256, rounds=3, beam=4, seed=3)
        m.set_polish(64)   # exact descent from the same best order can only lower it
        p_order, p_ms, _ = m.search(g, n_cand=70000, top_k=256, rounds=3, beam=4, seed=3)
    assert sorted(order.tolist()) == list(range(s.n)) and t_ms > 0
    assert ms == oracle.makespan(s.gpu, s.kernels, order.tolist())
    assert ms <= screened      # the beam always keeps the screening's best
    assert p_ms == oracle.makespan(s.gpu, s.kernels, p_order.tolist()) and p_ms <= ms


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


def test_tcgen05_forward_many_tiles_bit_identical(ko):
    """Rows for several 128-row tiles per CTA (ring stages and both TMEM
    accumulators wrap) and a ragged last round: the tcgen05 layers give the
    mma.sync path's bits exactly; sampled rows stay within the oracle's bar."""
    p = _params(13)
    B = 128 * (152 * 5 + 37)
    x = _features(14, B)
    m = ko.Model()
    m.set_params(_flat(p))
    m.set_tc(False)
    y_mma = m.predict(x)
    m.set_tc(True)
    y_tc = m.predict(x)
    m.close()
    assert np.array_equal(y_tc.view(np.uint32), y_mma.view(np.uint32))
    idx = np.linspace(0, B - 1, 512).astype(np.int64)
    want, _ = mlp.forward(p, x[idx])
    assert np.abs(y_tc[idx] - want).max() <= 2e-2 * max(1.0, np.abs(want).max())


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
    # split-K slices and per-block bias partial sums are summed in a fixed order: bit-identical runs
    a, b = _split(g_tc), _split(g_tc2)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        assert (a[k] == b[k]).all(), k
    assert loss_tc == pytest.approx(loss_mma, rel=1e-3)
    y, cache = mlp.forward(p, x)
    want = mlp.backward(p, cache, y, t)
    got, ref = _split(g_tc), _split(g_mma)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        nrm = max(np.linalg.norm(want[k]), 1e-12)
        assert np.linalg.norm(got[k] - want[k]) / nrm <= 2e-2, (k, "oracle")
        assert np.abs(got[k] - want[k]).max() <= 1e-3 * np.abs(want[k]).max(), (k, "oracle, element-wise")
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


def test_trained_network_gain(ko):
    """What the trained network adds, on 32 held-out sets with N 16..24 (too
    large to enumerate), every reported makespan exact:
      * at equal exact budgets (no timing involved, so the outcome is
        reproducible): the best of the network's top 1024 of 2^20 random
        candidates against the best of 1024 uniform random orders -- a
        network trained with labels of N <= 24 sets wins on a majority, one
        trained only on N <= 12 sets does not transfer (it is recorded, not
        asserted);
      * the guided search (screening, then network-ranked neighbourhoods
        around a beam of exact orders) against plain uniform random search
        given the same measured GPU time: the N <= 24 network wins on a
        majority, and on at least as many sets as the same search with the
        untrained network."""
    import bench
    from paper_1511_07983_gb300 import synth as sy
    tests = [sy.gen_set("large", j) for j in range(32)]
    models = {k: bench.train_surrogate(k, seed=7)[0] for k in ("mixed", "small", "untrained")}
    rand_best = []
    for j, s in enumerate(tests):
        with ko.Gpu.from_set(s) as g:
            order, best, _ = ko.ko_random_search(g, 1024, seed=207 + j)
            assert best == oracle.makespan(s.gpu, s.kernels, list(order))
        rand_best.append(best)
    screen = {}
    for k in ("mixed", "small"):
        out = []
        for j, s in enumerate(tests):
            with ko.Gpu.from_set(s) as g:
                order, best, _ = models[k].propose(g, n_cand=1 << 20, top_k=1024, seed=7 + j)
                assert best == oracle.makespan(s.gpu, s.kernels, list(order))
            out.append(best)
        screen[k] = sum(b < r for b, r in zip(out, rand_best))
    assert screen["mixed"] > 16, screen
    guided_wins = {}
    for k in ("mixed", "untrained"):
        models[k].set_polish(0)
        w = 0
        for j, s in enumerate(tests):
            with ko.Gpu.from_set(s) as g:
                order, best, s_ms = models[k].search(g, n_cand=1 << 18, top_k=1024, rounds=6, beam=8, seed=7 + j)
                assert best == oracle.makespan(s.gpu, s.kernels, list(order))
                _, _, cal_ms = ko.ko_random_search(g, 1 << 16, seed=99 + j)
                n_plain = max(1, int((1 << 16) * s_ms / max(cal_ms, 1e-3)))
                _, p_best, _ = ko.ko_random_search(g, n_plain, seed=107 + j)
            w += best < p_best
        guided_wins[k] = w
    for m in models.values():
        m.close()
    assert guided_wins["mixed"] > 16 and guided_wins["mixed"] >= guided_wins["untrained"], guided_wins
