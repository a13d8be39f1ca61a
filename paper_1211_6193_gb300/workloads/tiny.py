"""Tiny straight-line programs for exhaustive interleaving checks.

Each program runs one block of 2-3 threads through at most 6 shared-memory accesses
with data-independent addresses ``(a_j * tid + b_j) % nwords``, optional barriers
between accesses (the same barriers for every thread, so no deadlock), and finally
writes every loaded value to a private global slot so that loads are observable.
After a last barrier the final shared words are copied to a dump area of the arena.
Loads go to r4..r9; r11 holds the thread's slot base.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import rng
from .ir import R as REGS, TID, Asm, Launch, Program, r1, r2, r3, r10, r11

SLOTS = 6          # private global words per thread (one per possible load)


def tiny_program(seed: int, nthreads: int = 3, nsteps: int = 6, nwords: int = 3,
                 bar_rate: float = 0.25) -> Program:
    R = rng.SplitMix64(seed)
    a = Asm()
    a.s2r(r2, TID)
    nload = 0
    steps = []
    for j in range(nsteps):
        am, bm = R.randint(0, 3), R.randint(0, nwords - 1)
        kind = ("R", "W", "A")[R.randint(0, 2)]
        a.mul(r3, r2, am).add(r3, r3, bm).rem(r3, r3, nwords)
        if kind == "R":
            a.lds(REGS[4 + nload], r3)
            nload += 1
        elif kind == "W":
            a.mul(r10, r2, 16).add(r10, r10, j + 1).sts(r3, r10)
        else:
            a.mov(r10, j + 1).atoms(r3, r10)
        steps.append((kind, am, bm))
        if j + 1 < nsteps and R.uniform() < bar_rate:
            a.bar()
            steps.append(("B", 0, 0))
    a.mul(r11, r2, SLOTS).add(r11, r11, r1)
    for k in range(nload):
        a.stg(r11, REGS[4 + k], k)
    # final barrier, then thread (w % nthreads) copies shared word w to the dump area
    a.bar()
    dump = nthreads * SLOTS
    for w in range(nwords):
        a.seq(r3, r2, w % nthreads).brz(r3, f"nodump{w}")
        a.lds(r10, r3, w - 1).stg(r3, r10, dump + w - 1).label(f"nodump{w}")
    a.exit()
    arena = np.zeros(nthreads * SLOTS + nwords, dtype=np.int32)
    return Program(a.assemble(), [0], [Launch(0, 1, nthreads, nwords, (0, 0))], arena,
                   name="tiny", meta={"steps": steps, "nwords": nwords, "nload": nload})


def tiny_batch(seed: int, count: int, **kw) -> List[Program]:
    return [tiny_program(rng.derive(seed, i), **kw) for i in range(count)]


def tiny_global_program(seed: int, nthreads: int = 3, nsteps: int = 6, nwords: int = 3,
                        bar_rate: float = 0.25) -> Program:
    """The same shape with the accesses in global memory: one block of 2-3 threads makes at
    most 6 global loads and stores (no atomics) to words ``(a_j * tid + b_j) % nwords`` of the
    arena, optional barriers between them, and finally stores every loaded value to a private
    slot after the raced words (so that loads are observable).  No shared memory."""
    R = rng.SplitMix64(seed)
    a = Asm()
    a.s2r(r2, TID)
    nload = 0
    steps = []
    for j in range(nsteps):
        am, bm = R.randint(0, 3), R.randint(0, nwords - 1)
        kind = ("R", "W")[R.randint(0, 1)]
        a.mul(r3, r2, am).add(r3, r3, bm).rem(r3, r3, nwords)
        if kind == "R":
            a.ldg(REGS[4 + nload], r3)
            nload += 1
        else:
            a.mul(r10, r2, 16).add(r10, r10, j + 1).stg(r3, r10)
        steps.append((kind, am, bm))
        if j + 1 < nsteps and R.uniform() < bar_rate:
            a.bar()
            steps.append(("B", 0, 0))
    a.mul(r11, r2, SLOTS).add(r11, r11, nwords)
    for k in range(nload):
        a.stg(r11, REGS[4 + k], k)
    a.exit()
    arena = np.zeros(nwords + nthreads * SLOTS, dtype=np.int32)
    return Program(a.assemble(), [0], [Launch(0, 1, nthreads, 0, ())], arena,
                   name="tiny_global", meta={"steps": steps, "nwords": nwords, "nload": nload})


def tiny_global_batch(seed: int, count: int, **kw) -> List[Program]:
    return [tiny_global_program(rng.derive(seed, i), **kw) for i in range(count)]
