"""The paper's Figure 1 ``sum`` program, hand-translated into the IR, and its two variants.

Figure 1 stages ``in[bid*bdim + tid]`` into dynamic shared memory (line 9), syncs
(line 10), folds the upper half onto the lower half for ``tid < bdim/2`` (lines
11-13), syncs again (line 14), and thread 0 adds ``shared[1 .. bdim/2 + bdim%2 - 1]``
into ``shared[0]`` (lines 15-18) and writes ``out[bid]`` (line 19).  ``main`` (lines
22-41) fills ``in[i] = (21 i + 29) % 100`` for N = 18, launches ``sum<<<2, 9, 9 ints>>>
(in, out)`` and then ``sum<<<1, 2, 2 ints>>>(out, out)`` with aliased arguments.

Variants of Sec. 3.2 (the cudak examples):
* ``race=True``   - the ``__syncthreads()`` of line 14 removed (the race reported at line 17);
* ``deadlock=True`` - a ``__syncthreads()`` inserted after line 11, inside the ``if``.
"""
from __future__ import annotations

import numpy as np

from .ir import (BDIM, BID, TID, Asm, Launch, Program, RZ, r0, r1, r2, r3, r4, r5, r6, r7, r8,
                 r9, r10, r11, r12, r13, r14)

N = 18
NBLOCKS = 2
NTHREADS = N // NBLOCKS
IN_OFF = 0
OUT_OFF = N


def sum_kernel(race: bool = False, deadlock: bool = False) -> Asm:
    """Kernel ``sum(int* in, int* out)``: r0 = in, r1 = out (word offsets)."""
    a = Asm()
    a.s2r(r2, TID).s2r(r3, BID).s2r(r4, BDIM)               # line 8
    a.mul(r5, r3, r4).add(r5, r5, r2).add(r5, r5, r0)
    a.ldg(r6, r5).sts(r2, r6)                                 # line 9: shared[tid] = in[..]
    a.bar()                                                   # line 10
    a.div(r7, r4, 2).slt(r8, r2, r7).brz(r8, "after_if")      # line 11: if (tid < bdim/2)
    if deadlock:
        a.bar()                                               # inserted after line 11
    a.add(r9, r7, r2).lds(r10, r2).lds(r11, r9)               # line 12
    a.add(r10, r10, r11).sts(r2, r10)
    a.label("after_if")
    if not race:
        a.bar()                                               # line 14
    a.brnz(r2, "done")                                        # line 15: if (tid == 0)
    a.rem(r12, r4, 2).add(r12, r7, r12).mov(r13, 1)           # line 16: i = 1; bound
    a.label("loop")
    a.seq(r14, r13, r12).brnz(r14, "loop_end")                # i != bound
    a.lds(r10, RZ).lds(r11, r13).add(r10, r10, r11)           # line 17
    a.sts(RZ, r10)
    a.add(r13, r13, 1).bra("loop")                            # ++i
    a.label("loop_end")
    a.lds(r10, RZ).add(r5, r1, r3).stg(r5, r10)               # line 19: out[bid] = shared[0]
    a.label("done")
    a.exit()
    return a


def host_input() -> np.ndarray:
    """``host[i] = (21*i + 29) % 100`` (Fig. 1, line 26)."""
    return np.array([(21 * i + 29) % 100 for i in range(N)], dtype=np.int32)


def program(race: bool = False, deadlock: bool = False) -> Program:
    code = sum_kernel(race=race, deadlock=deadlock).assemble()
    arena = np.zeros(N + NBLOCKS, dtype=np.int32)
    arena[IN_OFF:IN_OFF + N] = host_input()
    launches = [
        Launch(0, NBLOCKS, NTHREADS, NTHREADS, (IN_OFF, OUT_OFF)),   # line 33
        Launch(0, 1, NBLOCKS, NBLOCKS, (OUT_OFF, OUT_OFF)),         # line 34 (aliased)
    ]
    name = "fig1" + ("_race" if race else "") + ("_deadlock" if deadlock else "")
    return Program(code, [0], launches, arena, name=name)
