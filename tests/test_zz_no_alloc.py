"""Allocation-free entry point (ko_eval_orders_noalloc), called through the C
ABI.  It serves callers that cannot allocate device memory (a framework that
owns the whole device heap, or code that must not risk the device-wide
synchronisation of cudaMalloc / cudaFree); its scratch is a fixed device array
inside the library.  Its makespans must equal ko_eval_orders' for the same
rows, on two calls in a row (the shared array carries nothing between calls).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

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


def _noalloc(ko, g, rows_dev, out_dev):
    import torch
    code = ko.lib().ko_eval_orders_noalloc(g.h, ctypes.c_void_p(rows_dev.data_ptr()), rows_dev.shape[0],
                                           ctypes.c_void_p(out_dev.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return code


@pytest.mark.parametrize("workload,idx", [("single8", 0), ("single12", 0), ("large", 2)])
def test_noalloc_matches_eval_orders_twice(ko, workload, idx):
    import torch
    s = synth.gen_set(workload, idx)
    with ko.Gpu.from_set(s) as g:
        for call, seed in enumerate((11, 12)):   # two calls in a row, different rows
            rows = synth.random_orders(seed, s.n, 600).astype(np.int8)
            rows[5] = rows[5][::-1]
            rows[7, 0] = rows[7, 1]            # not a permutation -> -1 on both paths
            want = g.eval_orders(orders=rows)
            d_rows = torch.from_numpy(rows).cuda()
            d_out = torch.full((rows.shape[0],), -7, dtype=torch.int64, device="cuda")
            assert _noalloc(ko, g, d_rows, d_out) == 0, call
            got = d_out.cpu().numpy()
            assert np.array_equal(got, want), (call, int(np.argmax(got != want)))
            assert got[7] == -1


def test_noalloc_rejects_host_buffers_and_oversized_sets(ko):
    s = synth.random_set(2, 4)
    with ko.Gpu.from_set(s) as g:
        rows = np.zeros((2, 4), dtype=np.int8)
        out = np.zeros(2, dtype=np.int64)
        code = ko.lib().ko_eval_orders_noalloc(g.h, rows.ctypes.data, 2, out.ctypes.data, None)
        assert code == -1
    big = synth.random_set(3, 3, gpu=(1000, 65536, 49152, 64, 32))
    with ko.Gpu.from_set(big) as g:
        import torch
        d_rows = torch.zeros((1, 3), dtype=torch.int8, device="cuda")
        d_out = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _noalloc(ko, g, d_rows, d_out) == -3
