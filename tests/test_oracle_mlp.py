"""Pins for the surrogate MLP oracle (no GPU): bf16 bit patterns worked by hand,
finite differences, closed forms and the Adam bias correction."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_bit_patterns():
    # 1 + 2^-8 is exactly halfway between bf16 1.0 and 1.0078125: ties to even -> 1.0
    # 1 + 3*2^-8 is halfway between 1.0078125 (odd mantissa) and 1.015625 -> 1.015625
    # a hair above a tie rounds up; pi -> 3.140625; negatives are symmetric
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, np.pi,
                  -(1.0 + 3 * 2 ** -8), 0.0, 2.0 ** -130], dtype=np.float64)
    want = np.array([1.0, 1.0, 1.015625, 1.0078125, 3.140625, -1.015625, 0.0, 0.0],
                    dtype=np.float32)
    got = mlp.bf16(x.astype(np.float32))
    assert np.array_equal(got[:7], want[:7])
    assert got[7] == mlp.bf16(np.float32(2.0 ** -130))  # subnormal keeps its top bits
    assert (got.view(np.uint32) & 0xFFFF == 0).all()


def test_slot_map():
    for n in range(1, 25):
        slots = [mlp.slot_of(k, n) for k in range(n)]
        assert len(set(slots)) == n and all(0 <= s < 24 for s in slots)
        if n > 1:
            assert slots[0] == 0 and slots[-1] == 23
    assert [mlp.slot_of(k, 24) for k in range(24)] == list(range(24))
    assert [mlp.slot_of(k, 3) for k in range(3)] == [0, 12, 23]   # 11.5 rounds up


def test_encode_places_features():
    kf = np.arange(3 * 7, dtype=np.float32).reshape(3, 7)
    gf = np.arange(8, dtype=np.float32) + 100
    x = mlp.encode(kf, gf, np.array([[2, 0, 1]]))
    assert np.array_equal(x[0, 0:7], kf[2])
    assert np.array_equal(x[0, 12 * 7:13 * 7], kf[0])
    assert np.array_equal(x[0, 23 * 7:24 * 7], kf[1])
    assert np.array_equal(x[0, 168:176], gf) and not x[0, 176:].any()
    assert not x[0, 7:12 * 7].any()


def _small_params(seed):
    p = mlp.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        p[k] = (rng.standard_normal(p[k].shape) * 0.1).astype(np.float32)
    p["b4"] = np.array([0.3], dtype=np.float32)
    return p


def test_backward_matches_central_differences():
    p = _small_params(3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((6, mlp.IN_PAD)).astype(np.float32)
    t = rng.standard_normal(6)
    y, cache = mlp.forward(p, x, rounding=False)
    g = mlp.backward(p, cache, y, t, rounding=False)
    h = 1e-6
    for key in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            q = {k: v.astype(np.float64).copy() for k, v in p.items()}
            q[key].reshape(-1)[idx] += h
            lp = mlp.loss(mlp.forward(q, x, rounding=False)[0], t)
            q[key].reshape(-1)[idx] -= 2 * h
            lm = mlp.loss(mlp.forward(q, x, rounding=False)[0], t)
            num = (lp - lm) / (2 * h)
            ana = g[key].reshape(-1)[idx]
            assert abs(num - ana) <= 1e-5 * max(1.0, abs(num)), (key, idx, num, ana)


def test_closed_form_single_path():
    # only x0 -> h1[0] -> h2[0] -> h3[0] -> y is non-zero: y = b4 + w4 * w3 * w2 * w1 * x0
    p = {k: np.zeros_like(v) for k, v in mlp.init_params(0).items()}
    p["W1"][0, 0], p["W2"][0, 0], p["W3"][0, 0], p["w4"][0] = 2.0, 0.5, 3.0, 0.25
    p["b4"][0] = 1.0
    x = np.zeros((2, mlp.IN_PAD), dtype=np.float32)
    x[:, 0] = [1.0, -1.0]
    y, cache = mlp.forward(p, x)
    assert y.tolist() == [1.0 + 0.25 * 3.0 * 0.5 * 2.0, 1.0]   # ReLU cuts the negative path
    g = mlp.backward(p, cache, y, np.array([0.0, 0.0]))
    # dL/dy = 2 y / B; only the first row passes the ReLUs
    assert g["b4"][0] == pytest.approx((2 * 1.75 + 2 * 1.0) / 2)
    assert g["W1"][0, 0] == pytest.approx(1.75 * 0.25 * 3.0 * 0.5 * 1.0)


def test_adam_first_step_is_sign_step():
    p = {"w": np.array([1.0, -2.0, 0.5], dtype=np.float32)}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    st = {}
    mlp.adam(p, g, st, step=1, lr=0.01)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-7)
    mlp.adam(p, g, st, step=2, lr=0.01)
    assert np.allclose(p["w"], [1.0 - 0.02, -2.0 + 0.02, 0.5], atol=1e-6)


def test_forward_rounds_activations_to_bf16():
    p = _small_params(5)
    x = np.random.default_rng(6).standard_normal((4, mlp.IN_PAD)).astype(np.float32)
    _, cache = mlp.forward(p, x)
    for i in (1, 2, 3):
        a = cache[f"a{i}"].astype(np.float32)
        assert np.array_equal(a, mlp.bf16(a)) and (a >= 0).all()
