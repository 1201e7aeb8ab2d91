"""CPU oracle for launch-order scoring -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never calls it and shares no
code with it; the only thing both sides consume is the seeded input generator.

The C file ``ko_oracle.c`` holds the simulator, Lehmer code, Algorithm 1 and the
bounds; this module compiles it with gcc, wraps it with ctypes and adds the
exhaustive statistics and the Table 3 outputs:

* ``exhaustive_stats`` -- min, max, better/equal/worse counts against the
  heuristic makespan and the 4096-bin histogram with
  bin = floor((M - min) * B / (max - min + 1)) over all N! orders.
* ``rank_outputs`` -- the Table 3 columns: percentile rank
  100 * (worse + equal) / N! (strict: 100 * worse / N!), speedup over worst
  max / M_h, deviation from optimal (M_h - min) / min.

Functions without an external pin are marked "parity unpinned" in their
docstring; every function here is pinned by a not-gpu test.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ko_oracle.c")
_BUILD = os.path.join(_HERE, "_build", platform.machine())
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Gpu(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("n_sm", "n_reg_sm", "n_shm_sm", "n_warp_sm", "n_blk_sm", "c_cap", "m_cap")]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                           "-ffp-contract=off", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            L.or_unrank.argtypes = [ctypes.c_int, ctypes.c_uint64, P(ctypes.c_int32)]
            L.or_rank.argtypes = [ctypes.c_int, P(ctypes.c_int32)]
            L.or_rank.restype = ctypes.c_uint64
            L.or_makespan.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32)]
            L.or_makespan.restype = ctypes.c_int64
            L.or_makespans_idx.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64),
                                           P(ctypes.c_uint64), ctypes.c_uint64, ctypes.c_int64,
                                           P(ctypes.c_int64), ctypes.c_int]
            L.or_makespans_orders.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64),
                                              P(ctypes.c_int32), ctypes.c_int64, P(ctypes.c_int64)]
            L.or_makespans_orders_sampled.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64),
                                                      P(ctypes.c_int32), ctypes.c_int64, ctypes.c_int,
                                                      P(ctypes.c_int64)]
            L.or_makespans_ps.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32),
                                          ctypes.c_int64, P(ctypes.c_double)]
            L.or_heuristic.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32)]
            L.or_heuristic.restype = ctypes.c_int
            L.or_heuristic_fp.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), ctypes.c_int,
                                          P(ctypes.c_int32)]
            L.or_heuristic_fp.restype = ctypes.c_int
            L.or_local_search.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_int32),
                                          ctypes.c_int, ctypes.c_int, P(ctypes.c_int32), P(ctypes.c_int64),
                                          P(ctypes.c_int64)]
            L.or_local_search.restype = ctypes.c_int
            L.or_score_matrix.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64), P(ctypes.c_double)]
            L.or_bounds.argtypes = [P(_Gpu), ctypes.c_int, P(ctypes.c_int64),
                                    P(ctypes.c_int64), P(ctypes.c_int64)]
            _lib = L
    return _lib


def _gpu(gpu) -> _Gpu:
    return _Gpu(*[int(v) for v in gpu])


def _kern(kernels) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(kernels, dtype=np.int64).reshape(-1, 6))


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def unrank(n: int, k: int) -> list[int]:
    """Lexicographic Lehmer unrank: index k of the n! orders -> permutation."""
    out = np.zeros(max(n, 1), dtype=np.int32)
    lib().or_unrank(n, int(k), _p(out, ctypes.c_int32))
    return [int(v) for v in out[:n]]


def rank(perm) -> int:
    p = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    return int(lib().or_rank(len(p), _p(p, ctypes.c_int32)))


def makespan(gpu, kernels, order) -> int:
    """Makespan of one launch order under the block-dispatch model."""
    k = _kern(kernels)
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    g = _gpu(gpu)
    return int(lib().or_makespan(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64),
                                 _p(o, ctypes.c_int32)))


def makespans_idx(gpu, kernels, idx=None, first: int = 0, count: int | None = None,
                  threads: int | None = None) -> np.ndarray:
    """Makespans of orders given by Lehmer index (array ``idx`` or the
    contiguous range ``first .. first+count-1``), threaded over ranges."""
    k = _kern(kernels)
    g = _gpu(gpu)
    threads = threads or os.cpu_count() or 1
    if idx is not None:
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64))
        count = idx.shape[0]
        ip = _p(idx, ctypes.c_uint64)
    else:
        ip = None
    out = np.empty(int(count), dtype=np.int64)
    if count:
        lib().or_makespans_idx(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64), ip,
                               int(first), int(count), _p(out, ctypes.c_int64), int(threads))
    return out


def makespans_orders(gpu, kernels, orders) -> np.ndarray:
    k = _kern(kernels)
    g = _gpu(gpu)
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
    cnt = o.shape[0] if o.ndim == 2 else 0
    out = np.empty(cnt, dtype=np.int64)
    if cnt:
        lib().or_makespans_orders(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64),
                                  _p(o, ctypes.c_int32), cnt, _p(out, ctypes.c_int64))
    return out


def makespans_sampled(gpu, kernels, orders, at_placement: bool) -> np.ndarray:
    """Makespans of explicit orders with durations fixed at the end of the
    burst (False, the default model) or at each block's placement (True)."""
    k = _kern(kernels)
    g = _gpu(gpu)
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
    if o.ndim == 1:
        o = o.reshape(1, -1)
    out = np.empty(o.shape[0], dtype=np.int64)
    if o.shape[0]:
        lib().or_makespans_orders_sampled(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64),
                                          _p(o, ctypes.c_int32), o.shape[0], int(bool(at_placement)),
                                          _p(out, ctypes.c_int64))
    return out


def makespans_ps(gpu, kernels, orders) -> np.ndarray:
    """Makespans (float64) of explicit orders under processor sharing with
    rates re-evaluated at every event (model variant)."""
    k = _kern(kernels)
    g = _gpu(gpu)
    o = np.ascontiguousarray(np.asarray(orders, dtype=np.int32))
    if o.ndim == 1:
        o = o.reshape(1, -1)
    out = np.empty(o.shape[0], dtype=np.float64)
    if o.shape[0]:
        lib().or_makespans_ps(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64), _p(o, ctypes.c_int32),
                              o.shape[0], _p(out, ctypes.c_double))
    return out


def heuristic(gpu, kernels) -> list[int]:
    """Algorithm 1 launch order."""
    k = _kern(kernels)
    g = _gpu(gpu)
    out = np.zeros(max(k.shape[0], 1), dtype=np.int32)
    lib().or_heuristic(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64), _p(out, ctypes.c_int32))
    return [int(v) for v in out[:k.shape[0]]]


def heuristic_fp(gpu, kernels, per_block: bool) -> list[int]:
    """Algorithm 1 with the per-SM (False) or per-block (True) footprint reading."""
    k = _kern(kernels)
    g = _gpu(gpu)
    out = np.zeros(max(k.shape[0], 1), dtype=np.int32)
    lib().or_heuristic_fp(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64), int(bool(per_block)),
                          _p(out, ctypes.c_int32))
    return [int(v) for v in out[:k.shape[0]]]


def local_search(gpu, kernels, start, moves: bool = True, max_iters: int = 1 << 20):
    """Steepest-descent hill climbing from `start` (swaps, plus moves if
    `moves`), every candidate scored exactly.  Returns (order, makespan,
    steps, orders scored)."""
    k = _kern(kernels)
    g = _gpu(gpu)
    n = k.shape[0]
    st = np.ascontiguousarray(np.asarray(start, dtype=np.int32).reshape(n))
    out = np.zeros(max(n, 1), dtype=np.int32)
    ms = ctypes.c_int64(0)
    ev = ctypes.c_int64(0)
    steps = lib().or_local_search(ctypes.byref(g), n, _p(k, ctypes.c_int64), _p(st, ctypes.c_int32),
                                  int(bool(moves)), int(max_iters), _p(out, ctypes.c_int32),
                                  ctypes.byref(ms), ctypes.byref(ev))
    return [int(v) for v in out[:n]], int(ms.value), int(steps), int(ev.value)


def heuristic_rounds(gpu, kernels) -> int:
    k = _kern(kernels)
    g = _gpu(gpu)
    out = np.zeros(max(k.shape[0], 1), dtype=np.int32)
    return int(lib().or_heuristic(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64),
                                  _p(out, ctypes.c_int32)))


def score_matrix(gpu, kernels) -> np.ndarray:
    k = _kern(kernels)
    g = _gpu(gpu)
    n = k.shape[0]
    out = np.zeros((n, n), dtype=np.float64)
    lib().or_score_matrix(ctypes.byref(g), n, _p(k, ctypes.c_int64), _p(out, ctypes.c_double))
    return out


def bounds(gpu, kernels) -> tuple[int, int]:
    k = _kern(kernels)
    g = _gpu(gpu)
    lb = ctypes.c_int64()
    ub = ctypes.c_int64()
    lib().or_bounds(ctypes.byref(g), k.shape[0], _p(k, ctypes.c_int64), ctypes.byref(lb),
                    ctypes.byref(ub))
    return int(lb.value), int(ub.value)


def histogram(ms: np.ndarray, lo: int, hi: int, nbins: int) -> np.ndarray:
    """bin = floor((M - lo) * nbins / (hi - lo + 1)), computed exactly in
    Python integers."""
    width = hi - lo + 1
    h = np.zeros(nbins, dtype=np.uint64)
    vals, counts = np.unique(ms, return_counts=True)
    for v, c in zip(vals.tolist(), counts.tolist()):
        h[(v - lo) * nbins // width] += c
    return h


def exhaustive_stats(gpu, kernels, heuristic_makespan: int, nbins: int = 4096,
                     threads: int | None = None, makespans: np.ndarray | None = None) -> dict:
    """All N! orders by Lehmer index: min, max, counts against the heuristic
    makespan, histogram."""
    n = _kern(kernels).shape[0]
    total = math.factorial(n)
    ms = makespans if makespans is not None else makespans_idx(gpu, kernels, first=0, count=total,
                                                                 threads=threads)
    lo, hi = int(ms.min()), int(ms.max())
    mh = int(heuristic_makespan)
    return dict(min=lo, max=hi, makespan=mh, n_total=total,
                n_better=int((ms < mh).sum()), n_equal=int((ms == mh).sum()),
                n_worse=int((ms > mh).sum()),
                hist=histogram(ms, lo, hi, nbins) if nbins else None)


def rank_outputs(st: dict) -> dict:
    """Table 3 columns from the exhaustive counts."""
    tot = st["n_total"]
    return dict(percentile=100.0 * (st["n_worse"] + st["n_equal"]) / tot,
                percentile_strict=100.0 * st["n_worse"] / tot,
                speedup_over_worst=st["max"] / st["makespan"],
                deviation_from_optimal=(st["makespan"] - st["min"]) / st["min"])
