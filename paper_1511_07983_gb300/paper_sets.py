"""The six experiments of Table 2 as descriptor sets on a GTX580-like GPU.

Sec. 6 runs every permutation of six (or eight) real kernels on a GTX580
(16 SMs, R_B = 4.11, 32K registers, 48 warps, 48 KB shared memory, 8 blocks
per SM) and reports Table 3.  The kernels themselves (NPB EP, BlackScholes,
VMD Electrostatics, Smith-Waterman) are not available, so these sets carry only
what Table 2 states -- R_i, shared memory per block, block and grid sizes --
plus stated assumptions for what it does not: cycles per block, registers per
thread, and the two ES / SW kernels of EpBsEsSw-8.  The simulator's Table 3
columns for them are therefore qualitative (simulated cycles, not ms).

Readings of Table 2 (inputs only; no method arithmetic here):
* EP: 128 threads (4 warps) per block, 20 registers per thread, R = 3.11;
  EP-6-shm uses 16 blocks of 8K..48K shared memory; EP-6-grid varies the grid
  16..96 blocks (warp footprints 4..24 per SM on 16 SMs).
* BS: R = 11.1, 32 blocks of 64..1024 threads (BS-6-blk), 24 registers per
  thread; the table's warp list 4, 8, 12, 16, 32, 64 does not match those block
  sizes and is not used.
* EpBs-6 / EpBs-6-shm: three EP kernels with a 4-warp footprint (64 blocks)
  and three BS kernels with a 12-warp footprint (64 blocks of 96 threads);
  EpBs-6-shm gives each family 16K, 24K and 48K of shared memory.
* EpBsEsSw-8: two kernels of each family; ES (R = 25, 256 threads, 2K smem,
  96 blocks) and SW (R = 0.8, 64 threads, 12K smem, 48 blocks) are assumed.
* Every block needs c = 20,000 compute cycles alone and m = round(c / R)
  memory cycles; R_B = 4.11 is Ccap / Mcap = 4110 / 1000.
"""
from __future__ import annotations

import numpy as np

from .synth import KernelSet

GTX580 = (16, 32768, 49152, 48, 8, 4110, 1000)
C_BLOCK = 20000


def _k(threads, regs_per_thread, smem, blocks, ratio, c=C_BLOCK):
    return (threads * regs_per_thread, smem, (threads + 31) // 32, blocks, c, max(1, round(c / ratio)))


def _ep(blocks=16, smem=0):
    return _k(128, 20, smem, blocks, 3.11)


def _bs(threads=96, blocks=64, smem=0):
    return _k(threads, 24, smem, blocks, 11.1)


def experiments() -> dict[str, KernelSet]:
    kb = 1024
    sets = {
        "EP-6-shm": [_ep(16, s * kb) for s in (8, 16, 24, 32, 40, 48)],
        "EP-6-grid": [_ep(g, 0) for g in (16, 32, 48, 64, 80, 96)],
        "BS-6-blk": [_bs(t, 32, 0) for t in (64, 128, 256, 512, 768, 1024)],
        "EpBs-6": [_ep(64, 0)] * 3 + [_bs(96, 64, 0)] * 3,
        "EpBs-6-shm": [_ep(64, s * kb) for s in (16, 24, 48)] + [_bs(96, 64, s * kb) for s in (16, 24, 48)],
        "EpBsEsSw-8": [_ep(64, 8 * kb), _ep(32, 24 * kb), _bs(96, 64, 0), _bs(256, 32, 16 * kb),
                       _k(256, 32, 2 * kb, 96, 25.0), _k(256, 32, 2 * kb, 48, 25.0),
                       _k(64, 28, 12 * kb, 48, 0.8), _k(64, 28, 12 * kb, 96, 0.8)],
    }
    return {name: KernelSet(gpu=GTX580, kernels=np.array(ks, dtype=np.int64)) for name, ks in sets.items()}
