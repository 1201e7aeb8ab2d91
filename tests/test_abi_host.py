"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/*.h, validates arguments, and its host-side Algorithm 1 and
bounds agree exactly with the oracle's."""
import glob
import os
import re

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ko():
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    kmod.lib()
    return kmod


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(ko_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["ko_create_gpu", "ko_add_kernel", "ko_eval_orders", "ko_rank_order",
                     "ko_heuristic_order"]:
        assert required in names


def _declared_returns():
    """name -> (return type, number of parameters) of every function in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for ret, name, args in re.findall(r"^([A-Za-z_][\w \*]*?)\b(ko_\w+)\s*\(([^)]*)\)", text, flags=re.M):
            args = args.strip()
            out[name] = (" ".join(ret.split()), 0 if args in ("", "void") else args.count(",") + 1)
    return out


def test_binding_declares_every_function_with_its_return_type():
    """Every function of include/ko.h has a ctypes signature in the binding
    whose return type and parameter count match the header's (a missing one
    would default to a 32-bit int and truncate 64-bit results or pointers)."""
    import ctypes

    from paper_1511_07983_gb300 import ko as kmod
    want = {"ko_status": ctypes.c_int32, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
            "double": ctypes.c_double, "void": None, "const char *": ctypes.c_char_p}
    declared = _declared_returns()
    assert set(declared) == set(kmod._SIGNATURES)
    for name, (ret, nargs) in declared.items():
        got, argtypes = kmod._SIGNATURES[name]
        assert len(argtypes) == nargs, (name, nargs, len(argtypes))
        if ret.endswith("*") and ret != "const char *":
            assert got is ctypes.c_void_p, (name, ret)   # opaque handles
        else:
            assert got is want[ret], (name, ret, got)


def test_library_exports_every_declared_symbol(ko):
    L = ko.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_argument_validation(ko):
    with pytest.raises(ko.KoError) as e:
        ko.ko_create_gpu(0, 65536, 49152, 64, 16)
    assert e.value.code == -1
    with pytest.raises(ko.KoError):
        ko.ko_create_gpu(13, 65536, 49152, 64, 33)       # > 32 blocks per SM
    g = ko.Gpu(2, 100, 100, 100, 4)
    with pytest.raises(ko.KoError) as e:
        g.add_kernel(101, 0, 1, 1, 1, 1)                 # block larger than an SM
    assert e.value.code == -2
    with pytest.raises(ko.KoError) as e:
        g.add_kernel(10, 0, 1, 0, 1, 1)                  # zero blocks
    assert e.value.code == -1
    with pytest.raises(ko.KoError):
        g.add_kernel(10, 0, 1, 1, 1, 1 << 25)             # cycles beyond 2^24
    assert g.add_kernel(10, 0, 1, 1, 5, 5) == 0
    assert g.n == 1
    assert ko.ko_status_str(-3) == "KO_ERR_TOO_LARGE"
    with pytest.raises(ko.KoError):
        ko.ko_set_capacity(g.h, 0, 1)
    with pytest.raises(ko.KoError):
        ko.ko_set_sampling(g.h, 2)
    ko.ko_set_sampling(g.h, ko.KO_SAMPLE_AT_PLACEMENT)
    # tuning knobs: the one-thread simulator's three state sizes, nothing else
    assert ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE) == 0
    for v in (0, 1, 2):
        ko.ko_set_option(g.h, ko.KO_OPT_LANE_STATE, v)
        assert ko.ko_get_option(g.h, ko.KO_OPT_LANE_STATE) == v
    for bad in (-1, 3):
        with pytest.raises(ko.KoError):
            ko.ko_set_option(g.h, ko.KO_OPT_LANE_STATE, bad)
    with pytest.raises(ko.KoError):
        ko.ko_set_option(g.h, ko.KO_OPT_LANES, 8)
    ko.ko_set_sampling(g.h, ko.KO_SAMPLE_BURST_END)


def _sets():
    out = [synth.gen_set("single8"), synth.gen_set("single12")]
    out += [synth.gen_set("sets10", i) for i in range(8)]
    out += [synth.gen_set("batched", i) for i in range(40)]
    out += [synth.gen_set("large", i) for i in range(20)]
    out += [synth.random_set(s, 2 + s % 20, blk=(1, 300)) for s in range(60)]
    return out


def test_binding_rejects_buffers_that_do_not_fit(ko):
    """The C ABI takes pointers and counts only, so the binding checks what it
    hands over: rows of N kernel ids, one-dimensional index lists, outputs of
    the right element type and length.  A mismatch raises before any call."""
    import torch
    s = synth.gen_set("single8", 0)
    n = s.n
    with ko.Gpu.from_set(s) as g:
        rows = np.zeros((2, n), dtype=np.int8)
        ids = np.zeros(3, dtype=np.uint64)
        for bad in (np.zeros((2, n - 1), dtype=np.int8), np.zeros(n, dtype=np.int8),
                    np.zeros((2, n + 1), dtype=np.int8)):
            with pytest.raises(ValueError):
                g.eval_orders(orders=bad)
            with pytest.raises(ValueError):
                g.eval_orders_ps(bad)
            with pytest.raises(ValueError):
                ko.ko_model_encode(g, bad)
        with pytest.raises(TypeError):
            g.eval_orders(orders=torch.zeros((2, n), dtype=torch.int64))
        with pytest.raises(ValueError):
            g.eval_orders(idx=np.zeros((3, 1), dtype=np.uint64))
        with pytest.raises(ValueError):
            g.eval_orders(idx=ids, out=np.empty(2, dtype=np.int64))
        with pytest.raises(TypeError):
            g.eval_orders(idx=ids, out=np.empty(3, dtype=np.float64))
        with pytest.raises(TypeError):
            g.eval_orders(orders=rows, out=torch.empty(2, dtype=torch.float32))
        with pytest.raises(TypeError):
            g.eval_orders_ps(rows, out=np.empty(2, dtype=np.int64))
        with pytest.raises(ValueError):
            g.eval_orders_ps(rows, out=np.empty(1, dtype=np.float64))
        with pytest.raises(ValueError):
            g.rank_order(list(range(n - 1)), nbins=8)
        with pytest.raises(ValueError):
            g.rank_order(None, nbins=8, hist=np.zeros(7, dtype=np.uint64))
        with pytest.raises(TypeError):
            g.rank_order(None, nbins=8, hist=np.zeros(8, dtype=np.float64))
        with pytest.raises(TypeError):
            g.eval_all(np.empty(40320, dtype=np.int64))
        with pytest.raises(ValueError):
            g.eval_all(torch.empty(40319, dtype=torch.int64))
        with pytest.raises(TypeError):
            g.eval_all(torch.empty(40320, dtype=torch.float64))
    with pytest.raises(ValueError):
        ko._features(np.zeros((4, ko.KO_MODEL_FEATURES - 1), dtype=np.float32))
    with pytest.raises(ValueError):
        ko._targets(np.zeros(3, dtype=np.float32), np.zeros((4, ko.KO_MODEL_FEATURES)))
    with pytest.raises(ValueError):
        ko._out_buf(np.zeros((2, 3), dtype=np.uint64), np.uint64, "hist", 2 * 4)


def test_heuristic_matches_oracle(ko):
    for s in _sets():
        with ko.Gpu.from_set(s) as g:
            assert g.heuristic_order().tolist() == oracle.heuristic(s.gpu, s.kernels)


def test_heuristic_hand_traces(ko):
    import json
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "hand_traces.json")))["cases"]
    for c in cases:
        if "heuristic" not in c:
            continue
        g = ko.Gpu(*c["gpu"][:5], c_cap=c["gpu"][5], m_cap=c["gpu"][6])
        for row in c["kernels"]:
            g.add_kernel(*row)
        assert g.heuristic_order().tolist() == c["heuristic"], c["name"]


def test_heuristic_per_block_reading_matches_oracle(ko):
    for s in _sets():
        with ko.Gpu.from_set(s) as g:
            assert g.heuristic_order(ko.KO_HEUR_PER_BLOCK).tolist() == oracle.heuristic_fp(s.gpu, s.kernels, True)
            assert g.heuristic_order(ko.KO_HEUR_PER_SM).tolist() == oracle.heuristic(s.gpu, s.kernels)
    import json
    cases = json.load(open(os.path.join(ROOT, "tests", "golden", "hand_traces.json")))["cases"]
    c = [c for c in cases if c["name"] == "W5"][0]
    g = ko.Gpu(*c["gpu"][:5], c_cap=c["gpu"][5], m_cap=c["gpu"][6])
    for row in c["kernels"]:
        g.add_kernel(*row)
    assert g.heuristic_order(ko.KO_HEUR_PER_BLOCK).tolist() == c["heuristic_per_block"]
    with pytest.raises(ko.KoError):
        ko.ko_heuristic_order_ex(g.h, 2)


def test_bounds_match_oracle(ko):
    for s in _sets():
        with ko.Gpu.from_set(s) as g:
            assert g.bounds() == oracle.bounds(s.gpu, s.kernels)


def test_upper_bound_at_the_admission_limit(ko):
    """Sets are admitted while the serial upper bound stays below 2^62: one
    kernel of 2^17 - 1 blocks with c = m = 2^20 on a 32-slot SM with unit
    capacities has UB = (2^17 - 1) * 2^20 * 32 * 2^20 = 2^62 - 2^45, which
    the library reports exactly as the oracle does; one more block of the same
    kind makes UB = 2^62, which the oracle computes exactly and the library
    refuses (KO_ERR_OVERFLOW).  Above int64 the oracle saturates."""
    gpu = (4, 65536, 49152, 64, 32, 1, 1)
    big = [1, 0, 1, (1 << 17) - 1, 1 << 20, 1 << 20]
    g = ko.Gpu(*gpu[:5], c_cap=1, m_cap=1)
    g.add_kernel(*big)
    lb, ub = g.bounds()
    assert ub == (1 << 62) - (1 << 45)
    assert (lb, ub) == oracle.bounds(gpu, [big])
    one = [1, 0, 1, 1, 1 << 20, 1 << 20]
    assert oracle.bounds(gpu, [big, one])[1] == 1 << 62
    with pytest.raises(ko.KoError) as e:
        g.add_kernel(*one)
    assert "OVERFLOW" in str(e.value)
    assert g.bounds() == (lb, ub)   # the refused kernel left the set unchanged
    huge = [1, 0, 1, 1 << 20, 1 << 24, 1 << 24]
    assert oracle.bounds(gpu, [huge])[1] == (1 << 63) - 1


def test_non_power_of_two_capacity_heuristic(ko):
    s = synth.random_set(5, 9, blk=(1, 100), c_cap=3000, m_cap=7000)
    with ko.Gpu.from_set(s) as g:
        assert g.heuristic_order().tolist() == oracle.heuristic(s.gpu, s.kernels)
