"""GPU parity of the processor-sharing model variant with the oracle: the
same doubles, bit for bit, on hand traces, random rows of small and large
sets, invalid rows, and host and device buffers."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1511_07983_gb300 import synth

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ko():
    import torch
    assert torch.cuda.is_available()
    from paper_1511_07983_gb300 import build, ko as kmod
    build.build()
    torch.cuda.init()
    return kmod


@pytest.mark.parametrize("name", ["P1", "P2"])
def test_hand_traces(ko, name):
    c = {c["name"]: c for c in json.load(open(os.path.join(GOLD, "hand_traces.json")))["cases"]}[name]
    g = ko.Gpu(*c["gpu"][:5], c_cap=c["gpu"][5], m_cap=c["gpu"][6])
    for row in c["kernels"]:
        g.add_kernel(*row)
    rows = np.array([o for o, _ in c["makespans_ps"]], dtype=np.int8)
    got = g.eval_orders_ps(rows)
    assert got.tolist() == pytest.approx([m for _, m in c["makespans_ps"]], rel=1e-12)
    assert (got == oracle.makespans_ps(c["gpu"], c["kernels"], rows.astype(np.int32))).all()


@pytest.mark.parametrize("case", ["single8", "sets10", "single12", "large", "tight"])
def test_rows_match_oracle_bitwise(ko, case):
    rng = np.random.default_rng(5)
    if case == "tight":   # small capacities: every block slowed, many re-timings
        s = synth.random_set(950, 7, gpu=(5, 65536, 49152, 64, 8), blk=(4, 30), c=(1000, 20000),
                             c_cap=3000, m_cap=3000)
    else:
        s = synth.gen_set(case, 2)
    rows = np.stack([rng.permutation(s.n) for _ in range(256)]).astype(np.int8)
    with ko.Gpu.from_set(s) as g:
        got = g.eval_orders_ps(rows)
    want = oracle.makespans_ps(s.gpu, s.kernels, rows.astype(np.int32))
    assert got.view(np.uint64).tolist() == want.view(np.uint64).tolist()


def test_device_buffers_and_invalid_rows(ko):
    import torch
    s = synth.gen_set("single8", 0)
    rows = np.array([[0, 1, 2, 3, 4, 5, 6, 7], [0, 0, 1, 2, 3, 4, 5, 6], [7, 6, 5, 4, 3, 2, 1, 9]], dtype=np.int8)
    with ko.Gpu.from_set(s) as g:
        host = g.eval_orders_ps(rows)
        d_rows = torch.from_numpy(rows).cuda()
        d_out = torch.empty(3, dtype=torch.float64, device="cuda")
        g.eval_orders_ps(d_rows, out=d_out)
        torch.cuda.synchronize()
    assert host[1] == -1.0 and host[2] == -1.0
    assert host[0] == oracle.makespans_ps(s.gpu, s.kernels, rows[:1].astype(np.int32))[0]
    assert d_out.cpu().numpy().tolist() == host.tolist()


def test_degenerate_sets(ko):
    # one kernel, one block; a single kernel filling every SM in one wave; 1024 SMs
    cases = [((4, 65536, 49152, 64, 8, 100, 100), [[1024, 0, 2, 1, 50, 7]]),
             ((4, 65536, 49152, 64, 4, 1500, 1 << 30), [[1024, 0, 2, 16, 1000, 1]]),
             ((1024, 65536, 233472, 64, 32, 32768, 32768), [[4096, 8192, 4, 900, 3000, 700],
                                                            [2048, 0, 2, 3000, 1200, 4000]])]
    for gpu, kern in cases:
        g = ko.Gpu(*gpu[:5], c_cap=gpu[5], m_cap=gpu[6])
        for row in kern:
            g.add_kernel(*row)
        rows = np.array([list(p) for p in __import__("itertools").permutations(range(len(kern)))], dtype=np.int8)
        got = g.eval_orders_ps(rows)
        want = oracle.makespans_ps(gpu, kern, rows.astype(np.int32))
        assert got.view(np.uint64).tolist() == want.view(np.uint64).tolist()
    assert want.min() > 0
