"""Busy kernels on the GPU: device limits, calibration grids, order timing
and argument checks, plus one small end-to-end validation run."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


def test_device_limits(ko):
    import torch
    n_sm, regs, smem, warps, blks, reserved, khz = ko.ko_hw_device_limits()
    assert n_sm == torch.cuda.get_device_properties(0).multi_processor_count
    assert regs >= 32768 and smem >= 49152 and warps >= 32 and blks >= 8 and 0 <= reserved <= 4096
    assert ko.ko_hw_regs(ko.KO_HW_COMPUTE) > 0 and ko.ko_hw_regs(ko.KO_HW_MEMORY) > 0


def test_longer_chain_takes_longer(ko):
    with ko.Hw([(ko.KO_HW_COMPUTE, 128, 0, 1, 1 << 14), (ko.KO_HW_COMPUTE, 128, 0, 1, 1 << 15),
                (ko.KO_HW_MEMORY, 256, 0, 152, 64)]) as hw:
        a, b = hw.time_grid(0, 1), hw.time_grid(1, 1)
        assert 1.5 < b / a < 2.5
        assert hw.time_grid(2, 152) > 0


def test_orders_are_timed(ko):
    with ko.Hw([(ko.KO_HW_COMPUTE, 128, 48 << 10, 300, 1 << 13), (ko.KO_HW_COMPUTE, 256, 0, 200, 1 << 12),
                (ko.KO_HW_MEMORY, 128, 0, 400, 32)]) as hw:
        t = hw.time_orders([[0, 1, 2], [2, 1, 0], [1, 0, 2]], reps=2)
        assert t.shape == (3,) and (t > 0).all() and (t < 1000).all()
        for bad in ([[0, 0, 1]], [[0, 1, 3]], [[-1, 0, 1]]):
            with pytest.raises(ko.KoError):
                hw.time_orders(bad)
        with pytest.raises(ko.KoError):
            hw.time_grid(3, 10)


def test_invalid_kernel_descriptions(ko):
    for bad in ([(2, 128, 0, 1, 1)], [(0, 100, 0, 1, 1)], [(0, 128, -1, 1, 1)], [(0, 128, 0, 0, 1)],
                [(0, 128, 1 << 30, 1, 1)], [(0, 2048, 0, 1, 1)]):
        with pytest.raises(ko.KoError):
            ko.Hw(bad)
    with pytest.raises(ko.KoError):
        ko.Hw([(0, 128, 0, 1, 1)] * 9)


def test_small_validation_run(ko):
    from paper_1511_07983_gb300 import hwval
    r = hwval.run_set(0, 3, reps=1)
    assert r["n"] == 3 and r["measured_ms"]["min"] > 0
    for k in ("unbounded", "calibrated"):
        if r[k] is not None:
            assert -1.0 <= r[k]["spearman"] <= 1.0 or math.isnan(r[k]["spearman"])
            assert 0 < r[k]["measured_percentile_of_sim_best"] <= 100


def test_trace_records(ko):
    n_sm = ko.ko_hw_device_limits()[0]
    ks = [(ko.KO_HW_COMPUTE, 128, 0, 300, 1 << 12), (ko.KO_HW_COMPUTE, 256, 16 << 10, 50, 1 << 12),
          (ko.KO_HW_MEMORY, 128, 0, 200, 16)]
    with ko.Hw(ks) as hw:
        rec, ms = hw.trace_order([2, 0, 1])
        assert rec.shape == (550, 4) and ms > 0
        assert (rec[:, 0] > 0).all() and (rec[:, 1] >= rec[:, 0]).all()
        assert (rec[:, 2] < n_sm).all()
        assert rec[:, 3].tolist() == [0] * 300 + [1] * 50 + [2] * 200
        # every block ran inside the timed interval (global timer in ns, events in ms)
        span_ms = (int(rec[:, 1].max()) - int(rec[:, 0].min())) / 1e6
        assert 0 < span_ms <= ms * 1.05 + 0.05
        with pytest.raises(ko.KoError):
            hw.trace_order([0, 0, 1])
