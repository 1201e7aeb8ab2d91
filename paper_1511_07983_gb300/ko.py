"""ctypes binding of libko (include/ko.h): argument marshalling only.

Every simulation step runs in the library's CUDA kernels; this module only
converts numpy arrays / torch tensors to pointers and raises on error codes.
It loads ``_build/libko.so`` and fails loudly if the library was not built
(``python -m paper_1511_07983_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes
import math
import os
import platform

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", platform.machine(), "libko.so")

KO_OK = 0
STATUS = {0: "KO_OK", -1: "KO_ERR_ARG", -2: "KO_ERR_NOFIT", -3: "KO_ERR_TOO_LARGE",
          -4: "KO_ERR_OVERFLOW", -5: "KO_ERR_CUDA", -6: "KO_ERR_TIMEOUT", -7: "KO_ERR_STATE",
          -8: "KO_ERR_NOMEM"}


class KoError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class ko_rank(ctypes.Structure):
    _fields_ = [("min", ctypes.c_int64), ("max", ctypes.c_int64), ("makespan", ctypes.c_int64),
                ("n_total", ctypes.c_uint64), ("n_better", ctypes.c_uint64),
                ("n_equal", ctypes.c_uint64), ("n_worse", ctypes.c_uint64),
                ("percentile", ctypes.c_double), ("percentile_strict", ctypes.c_double),
                ("speedup_over_worst", ctypes.c_double), ("deviation_from_optimal", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None

_SIGNATURES = {
    "ko_create_gpu": (ctypes.c_void_p, [ctypes.c_int32] * 5),
    "ko_set_capacity": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]),
    "ko_add_kernel": (ctypes.c_int32, [ctypes.c_void_p] + [ctypes.c_int32] * 4 + [ctypes.c_int64] * 2),
    "ko_num_kernels": (ctypes.c_int32, [ctypes.c_void_p]),
    "ko_bounds": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int64)]),
    "ko_heuristic_order": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "ko_eval_orders": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "ko_rank_order": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ko_rank),
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "ko_eval_all": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ko_set_option": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "ko_last_fallback_items": (ctypes.c_int64, [ctypes.c_void_p]),
    "ko_get_option": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int32]),
    "ko_autotune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]),
    "ko_kernel_launches": (ctypes.c_int64, []),
    "ko_last_sim_ms": (ctypes.c_double, [ctypes.c_void_p]),
    "ko_transfer_bytes": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "ko_batch_create": (ctypes.c_void_p, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_int32]),
    "ko_batch_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ko_rank), ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "ko_batch_orders": (ctypes.c_int64, [ctypes.c_void_p]),
    "ko_batch_fallback_items": (ctypes.c_int64, [ctypes.c_void_p]),
    "ko_batch_destroy": (None, [ctypes.c_void_p]),
    "ko_model_create": (ctypes.c_void_p, [ctypes.c_uint64]),
    "ko_model_get_params": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "ko_model_set_params": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p]),
    "ko_model_predict": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "ko_model_grad": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "ko_model_train_step": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "ko_model_encode": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "ko_surrogate_train": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                            ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "ko_surrogate_propose": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_uint64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "ko_surrogate_search": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_void_p]),
    "ko_random_search": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_void_p]),
    "ko_heuristic_order_ex": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "ko_local_search": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "ko_batch_autotune": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_void_p]),
    "ko_hw_create": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "ko_hw_regs": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "ko_hw_int_peak": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_float)]),
    "ko_hw_device_limits": (ctypes.c_int32, [ctypes.c_void_p]),
    "ko_hw_time_orders": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.c_void_p]),
    "ko_hw_time_grid": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float)]),
    "ko_hw_trace_order": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_float)]),
    "ko_hw_trace_len": (ctypes.c_int64, [ctypes.c_void_p]),
    "ko_hw_destroy": (None, [ctypes.c_void_p]),
    "ko_set_sampling": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32]),
    "ko_eval_orders_ps": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "ko_model_set_option": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "ko_model_destroy": (None, [ctypes.c_void_p]),
    "ko_eval_orders_noalloc": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "ko_destroy_gpu": (None, [ctypes.c_void_p]),
    "ko_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "ko_last_error": (ctypes.c_int32, []),
}


def lib():
    """Load libko.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libko.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, what: str) -> int:
    if code < 0:
        raise KoError(code, what)
    return code


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer {type(a)}")


def _is_tensor(a) -> bool:
    return hasattr(a, "data_ptr") and not isinstance(a, np.ndarray)


def _check_tensor(a, np_dtype, what):
    import torch
    want = {np.dtype(np.int8): (torch.int8,), np.dtype(np.int32): (torch.int32,),
            np.dtype(np.int64): (torch.int64,), np.dtype(np.uint64): (torch.int64, torch.uint64),
            np.dtype(np.float32): (torch.float32,), np.dtype(np.float64): (torch.float64,)}[np.dtype(np_dtype)]
    if a.dtype not in want:
        raise TypeError(f"{what}: expected a {want[0]} tensor, got {a.dtype}")
    if not a.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")


def _in_buf(a, np_dtype, what):
    """An input buffer for the C ABI: host data becomes a C-contiguous numpy
    array of np_dtype; a torch tensor must already have that element type."""
    if _is_tensor(a):
        _check_tensor(a, np_dtype, what)
        return a
    return np.ascontiguousarray(np.asarray(a, dtype=np_dtype))


def _out_buf(a, np_dtype, what, min_len):
    """An output buffer for the C ABI: never converted (a copy would lose the
    results); element type, contiguity and length are checked."""
    if _is_tensor(a):
        _check_tensor(a, np_dtype, what)
        n = a.numel()
    elif isinstance(a, np.ndarray):
        if a.dtype != np.dtype(np_dtype):
            raise TypeError(f"{what}: expected a {np.dtype(np_dtype)} array, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: array must be C-contiguous")
        n = a.size
    else:
        raise TypeError(f"{what}: unsupported buffer {type(a)}")
    if n < min_len:
        raise ValueError(f"{what}: {n} elements, {min_len} needed")
    return a


def _rows(a, n, what):
    """Rows of n kernel ids (int8), shape [count, n]."""
    a = _in_buf(a, np.int8, what)
    if len(a.shape) != 2 or a.shape[1] != n:
        raise ValueError(f"{what}: expected shape [count, {n}], got {tuple(a.shape)}")
    return a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ----------------------------------------------------- C names, same arguments

def ko_create_gpu(n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm):
    h = lib().ko_create_gpu(n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm)
    if not h:
        raise KoError(lib().ko_last_error(), "ko_create_gpu")
    return h


def ko_set_capacity(g, c_cap, m_cap):
    return _check(lib().ko_set_capacity(g, c_cap, m_cap), "ko_set_capacity")


def ko_add_kernel(g, n_reg_i, n_shm_i, n_warp_i, n_tblk_i, c_i, m_i):
    return _check(lib().ko_add_kernel(g, n_reg_i, n_shm_i, n_warp_i, n_tblk_i, c_i, m_i),
                  "ko_add_kernel")


def ko_num_kernels(g):
    return _check(lib().ko_num_kernels(g), "ko_num_kernels")


def ko_bounds(g):
    lb, ub = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ko_bounds(g, ctypes.byref(lb), ctypes.byref(ub)), "ko_bounds")
    return lb.value, ub.value


def ko_heuristic_order(g):
    n = ko_num_kernels(g)
    out = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().ko_heuristic_order(g, _ptr(out)), "ko_heuristic_order")
    return out[:n]


KO_SAMPLE_BURST_END, KO_SAMPLE_AT_PLACEMENT = 0, 1


def ko_set_sampling(g, mode):
    return _check(lib().ko_set_sampling(g, mode), "ko_set_sampling")


def ko_eval_orders_ps(g, orders, out=None, stream=None):
    """Processor-sharing makespans (float64) of rows of kernel ids (int8);
    numpy (host) or torch CUDA tensors."""
    orders = _rows(orders, ko_num_kernels(g), "orders")
    n = int(orders.shape[0])
    out = np.empty(n, dtype=np.float64) if out is None else _out_buf(out, np.float64, "out", n)
    _check(lib().ko_eval_orders_ps(g, _ptr(orders), n, _ptr(out), _stream(stream)), "ko_eval_orders_ps")
    return out


KO_HEUR_PER_SM = 0
KO_HEUR_PER_BLOCK = 1


def ko_heuristic_order_ex(g, reading):
    n = ko_num_kernels(g)
    out = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().ko_heuristic_order_ex(g, reading, _ptr(out)), "ko_heuristic_order_ex")
    return out[:n]


def ko_eval_orders(g, idx=None, orders=None, out=None, stream=None):
    """Makespans of orders given as Lehmer indices (uint64) or rows of kernel
    ids (int8).  Inputs/outputs may be numpy (host) or torch CUDA tensors."""
    if idx is not None:
        idx = _in_buf(idx, np.uint64, "idx")
        if len(idx.shape) != 1:
            raise ValueError(f"idx: expected one dimension, got shape {tuple(idx.shape)}")
    if orders is not None:
        orders = _rows(orders, ko_num_kernels(g), "orders")
    src = idx if idx is not None else orders
    count = int(src.shape[0]) if src is not None else 0
    out = np.empty(count, dtype=np.int64) if out is None else _out_buf(out, np.int64, "out", count)
    _check(lib().ko_eval_orders(g, _ptr(idx), _ptr(orders), count, _ptr(out), _stream(stream)),
           "ko_eval_orders")
    return out


def ko_rank_order(g, order=None, nbins=4096, hist=None, stream=None):
    """Exhaustive scoring; returns (ko_rank dict, histogram or None)."""
    r = ko_rank()
    o = None
    if order is not None:
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        if o.shape != (ko_num_kernels(g),):
            raise ValueError(f"order: expected {ko_num_kernels(g)} kernel ids, got shape {o.shape}")
    if hist is None and nbins:
        hist = np.zeros(nbins, dtype=np.uint64)
    elif hist is not None:
        hist = _out_buf(hist, np.uint64, "hist", int(nbins))
    _check(lib().ko_rank_order(g, _ptr(o), ctypes.byref(r), _ptr(hist), int(nbins) if hist is not None else 0,
                               _stream(stream)), "ko_rank_order")
    return r.as_dict(), hist


def ko_eval_all(g, out, stream=None):
    """All N! makespans into `out`, a CUDA int64 tensor of at least N! elements."""
    if not _is_tensor(out):
        raise TypeError("out: expected a CUDA int64 tensor")
    _out_buf(out, np.int64, "out", math.factorial(ko_num_kernels(g)))
    return _check(lib().ko_eval_all(g, _ptr(out), _stream(stream)), "ko_eval_all")


KO_OPT_LANES, KO_OPT_LEVELS, KO_OPT_SIMPLE_ONLY, KO_OPT_RUN_LIMIT, KO_OPT_STACK_GLOBAL = 1, 2, 3, 4, 5
KO_OPT_LANE_STATE = 6


def ko_set_option(g, key, value):
    return _check(lib().ko_set_option(g, key, value), "ko_set_option")


def ko_get_option(g, key):
    return _check(lib().ko_get_option(g, key), "ko_get_option")


def ko_autotune(g, cache_path=None, stream=None):
    p = cache_path.encode() if cache_path else None
    return _check(lib().ko_autotune(g, p, _stream(stream)), "ko_autotune")


def ko_last_fallback_items(g):
    return lib().ko_last_fallback_items(g)


def ko_kernel_launches():
    return lib().ko_kernel_launches()


def ko_last_sim_ms(g):
    return lib().ko_last_sim_ms(g)


def ko_transfer_bytes(g):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ko_transfer_bytes(g, ctypes.byref(a), ctypes.byref(b)), "ko_transfer_bytes")
    return a.value, b.value


def ko_destroy_gpu(g):
    lib().ko_destroy_gpu(g)


def ko_status_str(code):
    return lib().ko_status_str(code).decode()


def ko_last_error():
    return lib().ko_last_error()


def ko_batch_create(handles, nbins=0):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    b = lib().ko_batch_create(arr, len(handles), nbins)
    if not b:
        raise KoError(lib().ko_last_error(), "ko_batch_create")
    return b


def ko_batch_run(b, nsets, hist=None, stream=None, nbins=0):
    """Runs the batch; `hist`, if given, holds nsets x nbins uint64 (the bins
    the batch was created with)."""
    if hist is not None:
        hist = _out_buf(hist, np.uint64, "hist", nsets * nbins)
    out = (ko_rank * nsets)()
    _check(lib().ko_batch_run(b, out, _ptr(hist), _stream(stream)), "ko_batch_run")
    return [r.as_dict() for r in out]


def ko_batch_orders(b):
    return lib().ko_batch_orders(b)


def ko_batch_fallback_items(b):
    return lib().ko_batch_fallback_items(b)


def ko_batch_destroy(b):
    lib().ko_batch_destroy(b)


def ko_batch_autotune(gpus, cache_path=None, stream=None):
    """Per-(N_SM class, N) simulator choice for a batch of handles; sets each
    handle's lanes / levels / node-state placement."""
    arr = (ctypes.c_void_p * len(gpus))(*[g.h for g in gpus])
    path = cache_path.encode() if cache_path else None
    _check(lib().ko_batch_autotune(arr, len(gpus), path, _stream(stream)), "ko_batch_autotune")


class Batch:
    """Owning wrapper of a ko_batch (many sets, one captured graph)."""

    def __init__(self, gpus, nbins=0):
        self.nsets = len(gpus)
        self.nbins = nbins
        self.b = ko_batch_create([g.h for g in gpus], nbins)

    def run(self, hist=None, stream=None):
        if hist is None and self.nbins:
            hist = np.zeros((self.nsets, self.nbins), dtype=np.uint64)
        return ko_batch_run(self.b, self.nsets, hist=hist, stream=stream, nbins=self.nbins), hist

    def orders(self):
        return ko_batch_orders(self.b)

    def fallback_items(self):
        return ko_batch_fallback_items(self.b)

    def close(self):
        if self.b:
            ko_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


KO_MODEL_PARAMS = 181249
KO_MODEL_FEATURES = 192   # encoded width of one order (24 slots x 7 + 8 globals, padded)


def _features(x):
    """Host encoded orders, float32 [B, KO_MODEL_FEATURES]."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    if x.ndim != 2 or x.shape[1] != KO_MODEL_FEATURES:
        raise ValueError(f"x: expected shape [B, {KO_MODEL_FEATURES}], got {x.shape}")
    return x


def _targets(t, x):
    """Host targets, float32 [B] for features x [B, ...]."""
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
    if t.shape != (x.shape[0],):
        raise ValueError(f"t: expected shape ({x.shape[0]},), got {t.shape}")
    return t


class Model:
    """Owning wrapper of a ko_model (surrogate MLP)."""

    def __init__(self, seed=0):
        self.m = lib().ko_model_create(seed)
        if not self.m:
            raise KoError(lib().ko_last_error(), "ko_model_create")

    def set_tc(self, on: bool):
        """Inference layers on tcgen05 (True) or warp-level mma.sync (False)."""
        _check(lib().ko_model_set_option(self.m, 1, int(bool(on))), "ko_model_set_option")

    def set_tc_train(self, on: bool):
        """Training GEMMs on tcgen05 (True) or warp-level mma.sync (False)."""
        _check(lib().ko_model_set_option(self.m, 3, int(bool(on))), "ko_model_set_option")

    def set_polish(self, steps: int):
        """Exact descent steps after a guided search (KO_MODEL_OPT_POLISH; 0 = none)."""
        _check(lib().ko_model_set_option(self.m, 4, int(steps)), "ko_model_set_option")

    def set_chunk(self, rows: int):
        """Candidate rows per forward pass of propose/search (multiple of 1024)."""
        _check(lib().ko_model_set_option(self.m, 2, int(rows)), "ko_model_set_option")

    def get_params(self):
        out = np.empty(KO_MODEL_PARAMS, dtype=np.float32)
        _check(lib().ko_model_get_params(self.m, _ptr(out)), "ko_model_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        if flat.size != KO_MODEL_PARAMS:
            raise ValueError(f"params: {flat.size} values, {KO_MODEL_PARAMS} expected")
        _check(lib().ko_model_set_params(self.m, _ptr(flat)), "ko_model_set_params")

    def predict(self, x, stream=None):
        x = _features(x)
        y = np.empty(x.shape[0], dtype=np.float32)
        _check(lib().ko_model_predict(self.m, _ptr(x), x.shape[0], _ptr(y), _stream(stream)), "ko_model_predict")
        return y

    def grad(self, x, t, stream=None):
        x, t = _features(x), _targets(t, x)
        g = np.empty(KO_MODEL_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().ko_model_grad(self.m, _ptr(x), _ptr(t), x.shape[0], _ptr(g), ctypes.byref(loss),
                                   _stream(stream)), "ko_model_grad")
        return g, loss.value

    def train_step(self, x, t, lr, stream=None):
        x, t = _features(x), _targets(t, x)
        loss = ctypes.c_float()
        _check(lib().ko_model_train_step(self.m, _ptr(x), _ptr(t), x.shape[0], lr, ctypes.byref(loss),
                                         _stream(stream)), "ko_model_train_step")
        return loss.value

    def train(self, gpus, pairs_per_set, steps, batch=8192, lr=1e-3, seed=0, stream=None):
        arr = (ctypes.c_void_p * len(gpus))(*[g.h for g in gpus])
        curve = np.zeros(steps, dtype=np.float32)
        _check(lib().ko_surrogate_train(self.m, arr, len(gpus), pairs_per_set, steps, batch, lr, seed,
                                        _ptr(curve), _stream(stream)), "ko_surrogate_train")
        return curve

    def propose(self, g, n_cand, top_k=1024, seed=0, stream=None):
        order = np.zeros(max(g.n, 1), dtype=np.int32)
        ms = ctypes.c_int64()
        t = ctypes.c_double()
        _check(lib().ko_surrogate_propose(self.m, g.h, n_cand, top_k, seed, _ptr(order), ctypes.byref(ms),
                                          ctypes.byref(t), _stream(stream)), "ko_surrogate_propose")
        return order[:g.n], ms.value, t.value

    def search(self, g, n_cand=1 << 20, top_k=1024, rounds=8, beam=8, seed=0, stream=None):
        order = np.zeros(max(g.n, 1), dtype=np.int32)
        ms = ctypes.c_int64()
        t = ctypes.c_double()
        _check(lib().ko_surrogate_search(self.m, g.h, n_cand, top_k, rounds, beam, seed, _ptr(order),
                                         ctypes.byref(ms), ctypes.byref(t), _stream(stream)), "ko_surrogate_search")
        return order[:g.n], ms.value, t.value

    def close(self):
        if self.m:
            lib().ko_model_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ko_model_encode(g, orders, stream=None):
    orders = _rows(np.asarray(orders), g.n, "orders")
    x = np.empty((orders.shape[0], KO_MODEL_FEATURES), dtype=np.float32)
    _check(lib().ko_model_encode(g.h, _ptr(orders), orders.shape[0], _ptr(x), _stream(stream)), "ko_model_encode")
    return x


def ko_random_search(g, n_orders, seed=0, stream=None):
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    ms = ctypes.c_int64()
    t = ctypes.c_double()
    _check(lib().ko_random_search(g.h, n_orders, seed, _ptr(order), ctypes.byref(ms), ctypes.byref(t),
                                  _stream(stream)), "ko_random_search")
    return order[:g.n], ms.value, t.value


def ko_local_search(g, start=None, moves=True, max_iters=1 << 20, stream=None):
    """Exact steepest-descent hill climbing; returns (order, makespan, steps,
    orders simulated, elapsed ms)."""
    n = g.n
    st = None
    if start is not None:
        st = np.ascontiguousarray(np.asarray(start, dtype=np.int32).reshape(n))
    order = np.zeros(max(n, 1), dtype=np.int32)
    ms, steps, evals, t = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_double()
    _check(lib().ko_local_search(g.h, _ptr(st) if st is not None else None, int(bool(moves)), max_iters,
                                 _ptr(order), ctypes.byref(ms), ctypes.byref(steps), ctypes.byref(evals),
                                 ctypes.byref(t), _stream(stream)), "ko_local_search")
    return order[:n], ms.value, steps.value, evals.value, t.value


KO_HW_COMPUTE, KO_HW_MEMORY = 0, 1


class HwKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("threads", ctypes.c_int32), ("smem", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("iters", ctypes.c_int32)]


def ko_hw_device_limits():
    """(N_SM, regs/SM, smem/SM, warps/SM, blocks/SM, reserved smem/block, SM kHz)."""
    out = np.zeros(7, dtype=np.int32)
    _check(lib().ko_hw_device_limits(_ptr(out)), "ko_hw_device_limits")
    return tuple(int(v) for v in out)


def ko_hw_int_peak(turns=2048):
    """(lane operations per launch, fastest launch time in ms) of the integer
    issue-rate microbenchmark on the current device."""
    ops = ctypes.c_int64()
    ms = ctypes.c_float()
    _check(lib().ko_hw_int_peak(int(turns), ctypes.byref(ops), ctypes.byref(ms)), "ko_hw_int_peak")
    return int(ops.value), float(ms.value)


def ko_hw_regs(kind):
    r = ctypes.c_int32()
    _check(lib().ko_hw_regs(kind, ctypes.byref(r)), "ko_hw_regs")
    return r.value


class Hw:
    """Busy kernels on the current GPU, timed alone or in launch orders."""

    def __init__(self, kernels):
        """kernels: sequence of (kind, threads, smem, blocks, iters)."""
        arr = (HwKernel * len(kernels))(*[HwKernel(*map(int, k)) for k in kernels])
        self.n = len(kernels)
        self.h = lib().ko_hw_create(arr, self.n)
        if not self.h:
            raise KoError(lib().ko_last_error(), "ko_hw_create")

    def time_orders(self, orders, reps=3):
        o = np.ascontiguousarray(np.asarray(orders, dtype=np.int8).reshape(-1, self.n))
        out = np.zeros(o.shape[0], dtype=np.float32)
        _check(lib().ko_hw_time_orders(self.h, _ptr(o), o.shape[0], reps, _ptr(out)), "ko_hw_time_orders")
        return out

    def trace_order(self, order):
        """Per-block records [blocks, 4] (start ns, end ns, SM, kernel) of one
        run of `order`, and the run's event time in ms."""
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int8).reshape(self.n))
        rec = np.zeros(lib().ko_hw_trace_len(self.h), dtype=np.uint64)
        t = ctypes.c_float()
        _check(lib().ko_hw_trace_order(self.h, _ptr(o), _ptr(rec), ctypes.byref(t)), "ko_hw_trace_order")
        return rec.reshape(-1, 4), t.value

    def time_grid(self, k, blocks, reps=5):
        t = ctypes.c_float()
        _check(lib().ko_hw_time_grid(self.h, k, blocks, reps, ctypes.byref(t)), "ko_hw_time_grid")
        return t.value

    def close(self):
        if self.h:
            lib().ko_hw_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ convenience

class Gpu:
    """Owning wrapper of a ko_gpu handle."""

    def __init__(self, n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm, c_cap=None, m_cap=None):
        self.h = ko_create_gpu(n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm)
        if c_cap is not None:
            ko_set_capacity(self.h, c_cap, m_cap)

    @classmethod
    def from_set(cls, kset, sampling=KO_SAMPLE_BURST_END):
        """Handle for a synth.KernelSet (gpu 7-tuple + int64 [N, 6] kernels)."""
        g = cls(*kset.gpu[:5], c_cap=kset.gpu[5], m_cap=kset.gpu[6])
        if sampling != KO_SAMPLE_BURST_END:
            ko_set_sampling(g.h, sampling)
        for row in np.asarray(kset.kernels).tolist():
            g.add_kernel(*row)
        return g

    def add_kernel(self, n_reg, n_shm, n_warp, n_tblk, c, m):
        return ko_add_kernel(self.h, n_reg, n_shm, n_warp, n_tblk, c, m)

    @property
    def n(self):
        return ko_num_kernels(self.h)

    def bounds(self):
        return ko_bounds(self.h)

    def heuristic_order(self, reading=KO_HEUR_PER_SM):
        if reading == KO_HEUR_PER_SM:
            return ko_heuristic_order(self.h)
        return ko_heuristic_order_ex(self.h, reading)

    def eval_orders_ps(self, orders, out=None, stream=None):
        return ko_eval_orders_ps(self.h, orders, out=out, stream=stream)

    def local_search(self, start=None, moves=True, max_iters=1 << 20, stream=None):
        return ko_local_search(self, start=start, moves=moves, max_iters=max_iters, stream=stream)

    def eval_orders(self, idx=None, orders=None, out=None, stream=None):
        return ko_eval_orders(self.h, idx=idx, orders=orders, out=out, stream=stream)

    def rank_order(self, order=None, nbins=4096, hist=None, stream=None):
        return ko_rank_order(self.h, order=order, nbins=nbins, hist=hist, stream=stream)

    def eval_all(self, out, stream=None):
        return ko_eval_all(self.h, out, stream=stream)

    def set_option(self, key, value):
        return ko_set_option(self.h, key, value)

    def configure(self, lanes=None, levels=None, simple_only=None, run_limit=None, stack_global=None,
                  lane_state=None):
        if lanes is not None:
            self.set_option(KO_OPT_LANES, lanes)
        if levels is not None:
            self.set_option(KO_OPT_LEVELS, levels)
        if simple_only is not None:
            self.set_option(KO_OPT_SIMPLE_ONLY, int(bool(simple_only)))
        if run_limit is not None:
            self.set_option(KO_OPT_RUN_LIMIT, run_limit)
        if stack_global is not None:
            self.set_option(KO_OPT_STACK_GLOBAL, int(bool(stack_global)))
        if lane_state is not None:
            self.set_option(KO_OPT_LANE_STATE, lane_state)
        return self

    def last_fallback_items(self):
        return ko_last_fallback_items(self.h)

    def autotune(self, cache_path=None, stream=None):
        ko_autotune(self.h, cache_path, stream)
        return {"lanes": ko_get_option(self.h, KO_OPT_LANES),
                "levels": ko_get_option(self.h, KO_OPT_LEVELS),
                "stack_global": ko_get_option(self.h, KO_OPT_STACK_GLOBAL),
                "lane_state": ko_get_option(self.h, KO_OPT_LANE_STATE)}

    def last_sim_ms(self):
        return ko_last_sim_ms(self.h)

    def transfer_bytes(self):
        return ko_transfer_bytes(self.h)

    def n_orders(self):
        return math.factorial(self.n)

    def close(self):
        if self.h:
            ko_destroy_gpu(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
