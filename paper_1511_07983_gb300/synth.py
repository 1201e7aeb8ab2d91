"""Seeded synthetic kernel-set generator.

This module only draws inputs: simulated-GPU limits (Table 1, first three rows)
and per-kernel descriptors (Table 1, last three rows).  It holds none of the
method's arithmetic (no dispatch, no durations, no scores), so both the CUDA
path and the CPU oracle can be fed from it without sharing any computation.

The paper profiles real kernels (Sec. "Experimental Results"); those kernels and
their GPU are not available, so every set here is synthetic.  Workload recipes:

* ``single8``   one set, N=8, 13-SM GPU (65536 regs, 48 KB smem, 64 warps,
                16 blocks/SM), blocks/kernel U[8,64], c U[1000,20000].
* ``sets10``    64 sets, N=10, 15-SM GPU with the same limits, blocks U[15,120].
* ``batched``   4096 sets, N U[5,10], GPU drawn from {13, 15, 148} SMs.
* ``single12``  one set, N=12, 148-SM GPU (65536 regs, 228 KB smem, 64 warps,
                32 blocks/SM), blocks U[100,1000], c U[1000,50000].
* ``train``     surrogate training sets, N U[6,12], GPU from {13, 15, 148}.
* ``large``     surrogate test sets, N U[16,24], GPU from {13, 15, 148}.

Per kernel: threads/block in {128,256,512}; regs/thread U[16,63];
smem/block in {0, 4, 8, ..., 24} KB; R_i = c_i/m_i log-uniform on [0.1, 10],
i.e. R_i = 10**(2u-1); m_i = max(1, round(c_i / R_i)).  Per-block quantities are
stored (registers = regs/thread x threads, warps = threads/32).

Random numbers come from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), one
stream per (workload id, set index).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

#: default compute / memory capacities per SM (cycles of demand per cycle);
#: Ccap/Mcap = 1 puts R_B at the geometric centre of R_i in [0.1, 10].
C_CAP = 32768
M_CAP = 32768

WORKLOAD_IDS = {"single8": 1, "sets10": 2, "batched": 3, "single12": 4,
                "train": 5, "large": 6}

# (n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm)
GPU_SMALL13 = (13, 65536, 49152, 64, 16)
GPU_SMALL15 = (15, 65536, 49152, 64, 16)
GPU_BIG148 = (148, 65536, 233472, 64, 32)


def _mix(z: int) -> int:
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & MASK64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """SplitMix64 stream: state += golden gamma, output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return _mix(self.state)

    def uniform_int(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] as lo + x mod (hi - lo + 1)."""
        return lo + self.next() % (hi - lo + 1)

    def uniform01(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))

    def choice(self, seq):
        return seq[self.next() % len(seq)]


def stream(workload: str | int, set_idx: int) -> SplitMix64:
    wid = WORKLOAD_IDS[workload] if isinstance(workload, str) else int(workload)
    return SplitMix64(_mix((20151123 ^ (wid << 32) ^ set_idx) & MASK64))


@dataclass
class KernelSet:
    """One synthetic problem: a simulated GPU and N kernel descriptors.

    ``gpu`` = (n_sm, n_reg_sm, n_shm_sm, n_warp_sm, n_blk_sm, c_cap, m_cap).
    ``kernels`` is int64 [N, 6] with columns (n_reg_i, n_shm_i, n_warp_i,
    n_tblk_i, c_i, m_i), all per block except n_tblk_i.
    """
    gpu: tuple
    kernels: np.ndarray

    @property
    def n(self) -> int:
        return int(self.kernels.shape[0])


def draw_kernel(rng: SplitMix64, blk_lo: int, blk_hi: int, c_lo: int, c_hi: int):
    threads = rng.choice((128, 256, 512))
    regs_per_thread = rng.uniform_int(16, 63)
    smem = rng.choice((0, 4096, 8192, 12288, 16384, 20480, 24576))
    n_tblk = rng.uniform_int(blk_lo, blk_hi)
    c = rng.uniform_int(c_lo, c_hi)
    ratio = 10.0 ** (2.0 * rng.uniform01() - 1.0)
    m = max(1, int(round(c / ratio)))
    return (regs_per_thread * threads, smem, threads // 32, n_tblk, c, m)


def _gpu_for(rng: SplitMix64):
    choice = rng.next() % 3
    if choice == 0:
        return GPU_SMALL13, (15, 120, 1000, 20000)
    if choice == 1:
        return GPU_SMALL15, (15, 120, 1000, 20000)
    return GPU_BIG148, (100, 1000, 1000, 50000)


def gen_set(workload: str, set_idx: int = 0, n: int | None = None) -> KernelSet:
    """Draw set ``set_idx`` of ``workload`` (see module docstring)."""
    rng = stream(workload, set_idx)
    if workload == "single8":
        gpu, ranges, nk = GPU_SMALL13, (8, 64, 1000, 20000), 8
    elif workload == "sets10":
        gpu, ranges, nk = GPU_SMALL15, (15, 120, 1000, 20000), 10
    elif workload == "single12":
        gpu, ranges, nk = GPU_BIG148, (100, 1000, 1000, 50000), 12
    elif workload == "batched":
        nk = rng.uniform_int(5, 10)
        gpu, ranges = _gpu_for(rng)
    elif workload == "train":
        nk = rng.uniform_int(6, 12)
        gpu, ranges = _gpu_for(rng)
    elif workload == "large":
        nk = rng.uniform_int(16, 24)
        gpu, ranges = _gpu_for(rng)
    else:
        raise ValueError(f"unknown workload {workload!r}")
    if n is not None:
        nk = int(n)
    ks = np.array([draw_kernel(rng, *ranges) for _ in range(nk)], dtype=np.int64)
    return KernelSet(gpu=tuple(gpu) + (C_CAP, M_CAP), kernels=ks.reshape(nk, 6))


def random_set(seed: int, n: int, gpu=GPU_SMALL13, blk=(1, 40), c=(1, 5000),
               c_cap: int = C_CAP, m_cap: int = M_CAP) -> KernelSet:
    """Free-form seeded set for property and edge-case tests."""
    rng = SplitMix64(_mix(seed & MASK64))
    ks = [draw_kernel(rng, blk[0], blk[1], c[0], c[1]) for _ in range(n)]
    return KernelSet(gpu=tuple(gpu) + (c_cap, m_cap),
                     kernels=np.array(ks, dtype=np.int64).reshape(n, 6))


def random_orders(seed: int, n: int, count: int) -> np.ndarray:
    """``count`` seeded uniform permutations of range(n) (Fisher-Yates), int32."""
    rng = SplitMix64(_mix((seed * 0x2545F4914F6CDD1D) & MASK64))
    out = np.empty((count, n), dtype=np.int32)
    for r in range(count):
        p = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.next() % (i + 1)
            p[i], p[j] = p[j], p[i]
        out[r] = p
    return out


def random_indices(seed: int, total: int, count: int) -> np.ndarray:
    """``count`` seeded uniform integers in [0, total), uint64."""
    rng = SplitMix64(_mix((seed * 0x9E3779B97F4A7C15 + 7) & MASK64))
    return np.array([rng.next() % total for _ in range(count)], dtype=np.uint64)


def factorial(n: int) -> int:
    return math.factorial(n)
