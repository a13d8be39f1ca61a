"""The log-heavy workload: a 2-D 5-point stencil iterated over ping-pong arenas.

``out[y][x] = (c + n + s + e + w) / 5`` (C division, truncation toward zero; cells
outside the W x W grid read as 0).  Blocks are 32x32 threads (linear tid,
x = tid & 31, y = tid >> 5); each block stages a 34x34 shared tile whose halo is
loaded by the edge threads, synchronises, then reads its five taps from the tile.
Launch ``buggy_launch`` (0-based) uses a kernel without the staging barrier.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import rng
from .ir import BID, TID, Asm, Launch, Program, r0, r1, r2, r3, r4, r5, r6, r7, r8, r9, r10, r11, r12, r13, r14

TILE = 34


def stencil2d_kernel(log2w: int, with_barrier: bool = True) -> Asm:
    """r0 = input grid offset, r1 = output grid offset (row-major, W = 2^log2w)."""
    W = 1 << log2w
    bx_bits = log2w - 5                       # blocks per row = W / 32
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID)
    a.and_(r4, r2, 31).shr(r5, r2, 5)                             # tx, ty
    a.and_(r6, r3, (1 << bx_bits) - 1).shr(r7, r3, bx_bits)       # bx, by
    a.shl(r6, r6, 5).add(r6, r6, r4)                              # gx
    a.shl(r7, r7, 5).add(r7, r7, r5)                              # gy
    a.shl(r8, r7, log2w).add(r8, r8, r6)                          # gidx = gy*W + gx
    a.add(r9, r8, r0).ldg(r10, r9)                                # centre value
    a.mul(r11, r5, TILE).add(r11, r11, r4).add(r11, r11, TILE + 1)  # s = (ty+1)*34 + tx+1
    a.sts(r11, r10)
    # west halo (tx == 0)
    a.brnz(r4, "no_w").mov(r12, 0).brz(r6, "w_zero").ldg(r12, r9, -1).label("w_zero")
    a.sts(r11, r12, -1).label("no_w")
    # east halo (tx == 31)
    a.seq(r13, r4, 31).brz(r13, "no_e").mov(r12, 0).seq(r14, r6, W - 1).brnz(r14, "e_zero")
    a.ldg(r12, r9, 1).label("e_zero").sts(r11, r12, 1).label("no_e")
    # north halo (ty == 0)
    a.brnz(r5, "no_n").mov(r12, 0).brz(r7, "n_zero").ldg(r12, r9, -W).label("n_zero")
    a.sts(r11, r12, -TILE).label("no_n")
    # south halo (ty == 31)
    a.seq(r13, r5, 31).brz(r13, "no_s").mov(r12, 0).seq(r14, r7, W - 1).brnz(r14, "s_zero")
    a.ldg(r12, r9, W).label("s_zero").sts(r11, r12, TILE).label("no_s")
    if with_barrier:
        a.bar()
    a.lds(r10, r11)
    for off in (-1, 1, -TILE, TILE):
        a.lds(r12, r11, off).add(r10, r10, r12)
    a.div(r10, r10, 5)
    a.add(r9, r8, r1).stg(r9, r10).exit()
    return a


def program(log2w: int = 13, steps: int = 16, buggy_launch: Optional[int] = 8, seed: int = 4,
            values: Optional[np.ndarray] = None) -> Program:
    """W x W int32 grid uniform in [-1000, 1000] from SplitMix64(seed); ``steps`` launches
    alternating A->B and B->A; launch ``buggy_launch`` omits the staging barrier."""
    W = 1 << log2w
    assert W >= 32
    n = W * W
    k_ok = stencil2d_kernel(log2w, True)
    k_bug = stencil2d_kernel(log2w, False)
    c0, c1 = k_ok.assemble(), k_bug.assemble()
    # kernel 1 follows kernel 0 in the program: shift its branch targets
    c1 = c1.copy()
    from .ir import BRA, BRZ, BRNZ
    ops = c1["op_d_a_b"] & 0x7F
    br = np.isin(ops, [BRA, BRZ, BRNZ])
    c1["imm"][br] += len(c0)
    code = np.concatenate([c0, c1])
    if values is None:
        values = rng.uniform_range(seed, n, -1000, 1000)
    arena = np.zeros(2 * n, dtype=np.int32)
    arena[:n] = values
    nblocks = (W // 32) ** 2
    launches = []
    for t in range(steps):
        src, dst = (0, n) if t % 2 == 0 else (n, 0)
        launches.append(Launch(1 if t == buggy_launch else 0, nblocks, 1024, TILE * TILE, (src, dst)))
    return Program(code, [0, len(c0)], launches, arena, name=f"stencil2d_{W}x{W}_{steps}",
                   meta={"family": "stencil2d", "W": W, "steps": steps, "buggy_launch": buggy_launch})
