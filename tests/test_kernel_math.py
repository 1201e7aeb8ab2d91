"""The two closed forms the run-length simulator rests on, checked on the CPU
against brute force (the CUDA kernel's own results are checked against the
oracle in the GPU tests):

* bulk round-robin: placing `left` blocks of the head kernel by first fit, one
  block at a time from the round-robin pointer, equals a water-fill -- with
  L the smallest sweep count whose capacity F(L) = sum_s min(cap_s, L) covers
  `left`, every SM takes min(cap_s, L - 1) blocks plus one for the first `rem`
  SMs cyclically from the pointer that have cap_s >= L, and the pointer ends
  after the last of them (when everything fits, after the SM with the largest
  capacity that comes last cyclically);
* the order in which a warp's two segments take the prefixes of a chunk: a
  bijection on any item range that pairs item j with j ^ 1 as two prefixes
  differing only in the order of their last two kernels.
"""
import itertools
import math
import random

import pytest


def first_fit(caps, p, left):
    """Block-by-block dispatch of Sec. 2: each block goes to the first SM at or
    after the pointer with room, and the pointer moves past it; a block that
    fits nowhere ends the burst."""
    S = len(caps)
    room = list(caps)
    got = [0] * S
    while left > 0:
        for off in range(S):
            s = (p + off) % S
            if room[s] > 0:
                break
        else:
            break
        room[s] -= 1
        got[s] += 1
        p = (s + 1) % S
        left -= 1
    return got, p, left


def water_fill(caps, p, left):
    """The closed form the kernel evaluates per run of identical SMs."""
    S = len(caps)
    total = sum(caps)
    if total == 0:
        return [0] * S, p, left
    cyc = [(p + off) % S for off in range(S)]
    if total <= left:
        top = max(caps)
        last = [s for s in cyc if caps[s] == top][-1]
        return list(caps), (last + 1) % S, left - total
    L = next(L for L in range(1, max(caps) + 1) if sum(min(c, L) for c in caps) >= left)
    got = [min(c, L - 1) for c in caps]
    rem = left - sum(got)
    takers = [s for s in cyc if caps[s] >= L][:rem]
    for s in takers:
        got[s] += 1
    return got, (takers[-1] + 1) % S, 0


@pytest.mark.parametrize("seed", range(40))
def test_water_fill_equals_first_fit(seed):
    rng = random.Random(seed)
    for _ in range(300):
        S = rng.randint(1, 24)
        # runs of identical SMs, as the simulator sees them
        caps = []
        while len(caps) < S:
            caps += [rng.choice((0, 0, 1, 2, 3, 5, 8, 16, 32))] * rng.randint(1, 6)
        caps = caps[:S]
        p = rng.randrange(S)
        left = rng.randint(1, sum(caps) + 20)
        assert water_fill(caps, p, left) == first_fit(caps, p, left), (caps, p, left)


def pair_swap_order(j, m, lo, hi):
    """Item order of the kernel's paired segments (groups of m (m - 1) prefixes
    sharing all but their last two kernels, pairs of ranks {x < y} in
    lexicographic order, member 0 = (x, y), member 1 = (y, x))."""
    M = m * (m - 1)
    g0 = j - j % M
    if g0 < lo or g0 + M > hi:
        return j
    v = j - g0
    x = next(x for x in range(m) if v // 2 < sum(m - 1 - t for t in range(x + 1)))
    y = x + 1 + v // 2 - sum(m - 1 - t for t in range(x))
    a, b = (y, x) if v & 1 else (x, y)
    return g0 + a * (m - 1) + (b - 1 if b > a else b)


def prefix(n, d0, j):
    rest = list(range(n))
    out = []
    for i in range(d0):
        r = math.perm(n - 1 - i, d0 - 1 - i)
        out.append(rest.pop(j // r))
        j %= r
    return out


@pytest.mark.parametrize("n,d0", [(4, 2), (6, 3), (7, 5), (8, 6), (5, 5)])
def test_pair_order_is_a_bijection_of_swap_partners(n, d0):
    m = n - d0 + 2
    total = math.perm(n, d0)
    # the prefixes in lexicographic order are itertools' order
    assert [prefix(n, d0, j) for j in range(total)] == \
        [list(t) for t in itertools.permutations(range(n), d0)]
    for lo, hi in [(0, total), (1, total - 3), (m * (m - 1), min(total, 5 * m * (m - 1) + 7))]:
        img = [pair_swap_order(j, m, lo, hi) for j in range(lo, hi)]
        assert sorted(img) == list(range(lo, hi))
        M = m * (m - 1)
        for j in range(lo, hi - 1, 1):
            g0 = j - j % M
            if j % 2 == 0 and g0 >= lo and g0 + M <= hi:
                a, b = prefix(n, d0, img[j - lo]), prefix(n, d0, img[j + 1 - lo])
                assert a[:-2] == b[:-2] and a[-2:] == b[-2:][::-1]


def test_header_limits_fit_the_packed_fields():
    """The run-length simulator packs state into fixed bit fields; the ABI's
    limits must keep every packed value in range."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "ko.h")).read()
    lim = {}
    for name, num, shift in re.findall(r"#define (KO_MAX_\w+) (?:(\d+)|\(1 << (\d+)\))", text):
        lim[name] = int(num) if num else 1 << int(shift)
    max_kernels, max_sm, max_blk, max_cycles = (lim["KO_MAX_KERNELS"], lim["KO_MAX_SM"],
                                                lim["KO_MAX_BLK_SM"], lim["KO_MAX_CYCLES"])
    assert max_kernels <= 32                  # kernel id: 5 bits of a group word
    assert max_blk <= 63                      # blocks per SM of a group: 6 bits
    assert max_sm < 1 << 16                   # run range: begin | count << 16
    assert max_cycles < 1 << 25 and max_blk < 1 << 7   # warps used | blocks used << 25
    assert max_blk * max_cycles < 1 << 31     # SumC, SumM of one SM in a 32-bit int
    assert max_cycles * max(max_blk * max_cycles, 1 << 30) + (1 << 30) < 1 << 64  # duration product


def test_float_reciprocal_quotient_with_one_correction_is_exact():
    """The per-SM capacity uses floor(x / d) for 0 <= x <= 2^24, d >= 1,
    clamped at 32: min(x, 32 d) times the float reciprocal of d (IEEE
    round-to-nearest conversion, reciprocal and product, truncation), then one
    exact integer correction either way.  Checked where it is hardest, on both
    sides of every integer quotient 0..32, for every d up to 2^12 and random
    larger d."""
    import numpy as np

    def quot32(x, d):
        xc = np.minimum(x, d << 5)
        rcp = (np.float32(1.0) / d.astype(np.float32)).astype(np.float32)
        q = np.trunc(xc.astype(np.float32) * rcp).astype(np.int64)
        q = q + ((q + 1) * d <= xc)
        q = q - (q * d > xc)
        return q

    rng = np.random.default_rng(5)
    ds = np.concatenate([np.arange(1, 1 << 12), rng.integers(1 << 12, 1 << 24, 20000)]).astype(np.int64)
    k = np.arange(0, 34, dtype=np.int64)
    for off in (-1, 0, 1):
        d = np.repeat(ds, k.size)
        x = np.clip(np.tile(k, ds.size) * d + off, 0, 1 << 24)
        assert np.array_equal(quot32(x, d), np.minimum(x // d, 32))
    x = rng.integers(0, (1 << 24) + 1, 200000)
    d = rng.integers(1, 1 << 24, 200000)
    assert np.array_equal(quot32(x, d), np.minimum(x // d, 32))
