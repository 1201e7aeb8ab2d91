"""Surrogate MLP oracle -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The learned part of the build is not in the paper: a small MLP predicts
log2(makespan / lower bound) of a launch order from position-ordered kernel
descriptors so that orders can be proposed for sets too large to enumerate;
every proposal is rescored exactly by the simulator.  This module is the plain
numpy definition the device kernels are checked against:

* ``encode``     order -> 192 features (24 position slots x 7 + 8 globals),
* ``forward``    192 -> 256 -> 256 -> 256 -> 1 with ReLU; BF16 weights and
                 activations (round-to-nearest-even of the FP32 bit pattern),
                 accumulation in FP64 here (FP32 on the device),
* ``backward``   gradients of the mean squared error, BF16 operands at the
                 same points the device rounds them,
* ``adam``       Adam on FP32 master weights.

Pins (tests/test_oracle_mlp.py): central finite differences in FP64 with
rounding switched off, closed forms of a one-hidden-unit network, the bf16
rounding against hand-worked bit patterns, and the Adam bias correction.
"""
from __future__ import annotations

import math

import numpy as np

SLOTS = 24
SLOT_FEATURES = 7
GLOBALS = 8
IN_FEATURES = SLOTS * SLOT_FEATURES + GLOBALS   # 176
IN_PAD = 192
HIDDEN = 256


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) from the float32 bits."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (u & 0xFFFFFFFF).astype(np.uint32).view(np.float32).reshape(a.shape)


def _ident(x):
    return np.asarray(x, dtype=np.float64)


# ----------------------------------------------------------------- encoding ---

def kernel_features(gpu, kernels) -> np.ndarray:
    """Per-kernel slot features [N, 7] (float32): regs/R, smem/Sh, warps/W,
    ceil(blocks/S)/Bk, log2(c)/16, log2(m)/16, present flag."""
    S, R, Sh, W, Bk = (float(v) for v in gpu[:5])
    k = np.asarray(kernels, dtype=np.float64)
    f = np.zeros((k.shape[0], SLOT_FEATURES), dtype=np.float32)
    for i in range(k.shape[0]):
        r, s, w, b, c, m = k[i]
        f[i] = [np.float32(r / R), np.float32(s / Sh), np.float32(w / W),
                np.float32(math.ceil(b / S) / Bk), np.float32(math.log2(c) / 16.0),
                np.float32(math.log2(m) / 16.0), np.float32(1.0)]
    return f


def global_features(gpu, n: int, lb: int) -> np.ndarray:
    """[8] float32: N/24, S/148, log2 of the four limits / 24, log2(LB)/32, 1."""
    S, R, Sh, W, Bk = (float(v) for v in gpu[:5])
    return np.array([n / 24.0, S / 148.0, math.log2(R) / 24.0, math.log2(Sh) / 24.0,
                     math.log2(W) / 24.0, math.log2(Bk) / 24.0, math.log2(max(lb, 1)) / 32.0,
                     1.0], dtype=np.float32)


def slot_of(position: int, n: int) -> int:
    """Position k of an N-kernel order goes to slot round(23 k / (N-1))
    (integer arithmetic, halves rounded up; slot 0 when N = 1)."""
    if n <= 1:
        return 0
    return (2 * (SLOTS - 1) * position + (n - 1)) // (2 * (n - 1))


def encode(kfeat: np.ndarray, gfeat: np.ndarray, orders: np.ndarray) -> np.ndarray:
    """Orders [B, N] -> features [B, 192] (float32, zero padding)."""
    orders = np.asarray(orders)
    B, n = orders.shape
    x = np.zeros((B, IN_PAD), dtype=np.float32)
    for pos in range(n):
        sl = slot_of(pos, n)
        x[:, sl * SLOT_FEATURES:(sl + 1) * SLOT_FEATURES] = kfeat[orders[:, pos]]
    x[:, SLOTS * SLOT_FEATURES:IN_FEATURES] = gfeat
    return x


# ------------------------------------------------------------------ network ---

def init_params(seed: int) -> dict:
    """He-normal init (numpy Generator; tests pass the same arrays to the
    device, so the init itself needs no device counterpart)."""
    rng = np.random.default_rng(seed)
    p = {}
    dims = [(IN_PAD, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN)]
    for i, (a, b) in enumerate(dims, start=1):
        fan_in = IN_FEATURES if i == 1 else a
        p[f"W{i}"] = (rng.standard_normal((a, b)) * math.sqrt(2.0 / fan_in)).astype(np.float32)
        if i == 1:
            p["W1"][IN_FEATURES:] = 0.0
        p[f"b{i}"] = np.zeros(b, dtype=np.float32)
    p["w4"] = (rng.standard_normal(HIDDEN) * math.sqrt(1.0 / HIDDEN)).astype(np.float32)
    p["b4"] = np.zeros(1, dtype=np.float32)
    return p


def forward(p: dict, x: np.ndarray, rounding: bool = True):
    """Returns (y [B] float64, cache).  Layer l: Z = A_{l-1} W_l + b_l,
    A_l = round(relu(Z)); y = A_3 . w4 + b4."""
    r = bf16 if rounding else _ident
    a0 = np.asarray(r(x), dtype=np.float64)
    cache = {"a0": a0}
    a = a0
    for i in (1, 2, 3):
        w = np.asarray(r(p[f"W{i}"]), dtype=np.float64)
        z = a @ w + np.asarray(p[f"b{i}"], dtype=np.float64)
        a = np.asarray(r(np.maximum(z, 0.0)), dtype=np.float64)
        cache[f"z{i}"] = z
        cache[f"a{i}"] = a
    w4 = np.asarray(r(p["w4"]), dtype=np.float64)
    y = a @ w4 + float(p["b4"][0])
    return y, cache


def loss(y: np.ndarray, t: np.ndarray) -> float:
    """Mean squared error (1/B) sum (y - t)^2."""
    d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d))


def backward(p: dict, cache: dict, y: np.ndarray, t: np.ndarray, rounding: bool = True) -> dict:
    """Gradients of ``loss``.  The device rounds the upstream gradient of each
    hidden layer to bf16 before its two GEMMs (weight and input gradients);
    weights and activations are the bf16 values of the forward pass."""
    r = bf16 if rounding else _ident
    B = y.shape[0]
    dy = 2.0 * (np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)) / B
    g = {}
    a3 = cache["a3"]
    w4 = np.asarray(r(p["w4"]), dtype=np.float64)
    g["w4"] = a3.T @ dy
    g["b4"] = np.array([dy.sum()])
    da = np.outer(dy, w4)                           # dL/dA3
    for i in (3, 2, 1):
        dz = da * (cache[f"z{i}"] > 0.0)            # through ReLU
        dzr = np.asarray(r(dz), dtype=np.float64)
        a_prev = cache[f"a{i - 1}"]
        g[f"W{i}"] = a_prev.T @ dzr
        g[f"b{i}"] = dz.sum(axis=0)
        if i > 1:
            w = np.asarray(r(p[f"W{i}"]), dtype=np.float64)
            da = dzr @ w.T
    return g


def adam(p: dict, g: dict, state: dict, step: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8) -> None:
    """In-place Adam update of the float32 master weights (step counts from 1)."""
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k], dtype=np.float64))
        v = state.setdefault("v_" + k, np.zeros_like(p[k], dtype=np.float64))
        gk = np.asarray(g[k], dtype=np.float64).reshape(p[k].shape)
        m[...] = b1 * m + (1.0 - b1) * gk
        v[...] = b2 * v + (1.0 - b2) * gk * gk
        mhat = m / (1.0 - b1 ** step)
        vhat = v / (1.0 - b2 ** step)
        p[k] = (p[k] - lr * mhat / (np.sqrt(vhat) + eps)).astype(np.float32)
