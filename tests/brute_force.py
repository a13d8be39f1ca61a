"""Exhaustive interleaving enumeration for tiny straight-line programs.

A pin for the oracle that shares none of its code: a thread-level interpreter of the
straight-line IR subset the tiny programs use, a depth-first search over every
interleaving of the threads' shared-memory accesses that respects the barriers, and a
symbolic commutation test that decides which pairs of accesses conflict.

Sec. 3.1 of the paper defines a race as two threads touching the same location with
no synchronisation point in between, at least one writing, and says the method finds
races "across all possible thread interleavings" of the observed accesses.  Here that
is taken literally: a pair of accesses is a race when both execution orders occur
among the interleavings and the two orders are distinguishable (the pair does not
commute).
"""
from __future__ import annotations

from typing import Dict, List, Set, Tuple

import numpy as np

from paper_1211_6193_gb300.workloads import ir

# ------------------------------------------------------------ per-thread event lists


def thread_events(prog: ir.Program, tid: int, space: str = "shared"):
    """Run one thread alone, loads symbolic; return its events and global stores.

    events: ("R", addr, pc, load_id) | ("W", addr, pc, value) | ("A", addr, pc, value) | ("B",)
    gstores: (addr, value) with value an int or ("load", load_id)
    With space == "global" the events are the global loads and stores of words
    [0, meta["nwords"]) and every other global store is a gstore.
    """
    gwords = prog.meta.get("nwords", 0) if space == "global" else 0
    launch = prog.launches[0]
    regs: Dict[int, object] = {i: 0 for i in range(16)}
    for i, v in enumerate(launch.params):
        regs[i] = int(v)
    ops, ds, as_, bs, imms = ir.decode_fields(prog.code)
    pc = prog.kernel_entry[launch.kernel]
    events, gstores, nload = [], [], 0

    def rd(r):
        return 0 if r == ir.RZ_INDEX else regs[r]

    def concrete(v):
        assert isinstance(v, int), "address or operand depends on a load"
        return v

    while pc < len(prog.code):
        op, d, a, b, imm = int(ops[pc]), int(ds[pc]), int(as_[pc]), int(bs[pc]), int(imms[pc])
        base = op & 0x7F
        B = imm if op & ir.BIMM else None
        nxt = pc + 1
        if base == ir.S2R:
            assert imm == ir.TID
            regs[d] = tid
        elif base in (ir.MOV, ir.ADD, ir.MUL, ir.REM, ir.SEQ):
            y = B if B is not None else rd(b)
            if base == ir.MOV:
                val = y
            else:
                x, y = concrete(rd(a)), concrete(y)
                val = {ir.ADD: x + y, ir.MUL: x * y, ir.REM: (x % y) if y else 0, ir.SEQ: int(x == y)}[base]
            regs[d] = val
        elif base == ir.LDS:
            regs[d] = ("load", nload)
            events.append(("R", concrete(rd(a)) + imm, pc, nload))
            nload += 1
        elif base == ir.STS:
            events.append(("W", concrete(rd(a)) + imm, pc, concrete(rd(b))))
        elif base == ir.ATOMS:
            events.append(("A", concrete(rd(a)) + imm, pc, concrete(rd(b))))
        elif base == ir.LDG and space == "global" and concrete(rd(a)) + imm < gwords:
            regs[d] = ("load", nload)
            events.append(("R", concrete(rd(a)) + imm, pc, nload))
            nload += 1
        elif base == ir.STG and space == "global" and concrete(rd(a)) + imm < gwords:
            events.append(("W", concrete(rd(a)) + imm, pc, concrete(rd(b))))
        elif base == ir.STG:
            gstores.append((concrete(rd(a)) + imm, rd(b)))
        elif base == ir.BAR:
            events.append(("B",))
        elif base == ir.BRZ:
            if concrete(rd(a)) == 0:
                nxt = imm
        elif base == ir.EXIT:
            break
        else:
            raise AssertionError(f"opcode {base} outside the tiny subset")
        pc = nxt
    return events, gstores


# ------------------------------------------------------------ interleavings


def enumerate_outcomes(prog: ir.Program, space: str = "shared"):
    """All final arenas over all barrier-respecting interleavings, plus reachable positions.
    With space == "global" the interleaved memory is the arena's words [0, meta["nwords"])."""
    launch = prog.launches[0]
    n = launch.block_dim
    nwords = launch.shmem_words if space == "shared" else prog.meta["nwords"]
    per = [thread_events(prog, t, space) for t in range(n)]
    evs = [p[0] for p in per]
    lens = [len(e) for e in evs]
    outcomes: Set[Tuple[int, ...]] = set()
    positions: Set[Tuple[int, ...]] = set()
    seen = set()
    mem0 = [0] * nwords if space == "shared" else [int(x) for x in prog.global_init[:nwords]]
    stack = [(tuple([0] * n), tuple(mem0), tuple(() for _ in range(n)))]
    while stack:
        state = stack.pop()
        if state in seen:
            continue
        seen.add(state)
        pos, mem, loads = state
        positions.add(pos)
        if all(pos[i] == lens[i] for i in range(n)):
            arena = np.array(prog.global_init, dtype=np.int64)
            if space == "global":
                arena[:nwords] = mem
            for t in range(n):
                for addr, v in per[t][1]:
                    arena[addr] = loads[t][v[1]] if isinstance(v, tuple) else v
            outcomes.add(tuple(int(x) for x in arena))
            continue
        at_bar = [pos[i] < lens[i] and evs[i][pos[i]][0] == "B" for i in range(n)]
        if all(at_bar):
            stack.append((tuple(p + 1 for p in pos), mem, loads))
            continue
        for i in range(n):
            if pos[i] == lens[i] or at_bar[i]:
                continue
            e = evs[i][pos[i]]
            m, ld = list(mem), list(loads)
            if e[0] == "R":
                ld[i] = loads[i] + (mem[e[1]],)
            elif e[0] == "W":
                m[e[1]] = e[3]
            else:
                m[e[1]] = m[e[1]] + e[3]
            p2 = list(pos)
            p2[i] += 1
            stack.append((tuple(p2), tuple(m), tuple(ld)))
    return evs, outcomes, positions


# ------------------------------------------------------------ conflicts


def _apply(kind: str, ident, value):
    """Symbolic effect of one access on a location value (base, sorted addends)."""
    base, adds = value
    if kind == "R":
        return value, value
    if kind == "W":
        return None, (("w", ident), ())
    return None, (base, tuple(sorted(adds + (ident,))))


def commute(k1: str, k2: str) -> bool:
    """Do two accesses (distinct threads, same location) give identical observations in both orders?"""
    x = ("x", ())
    r1a, s = _apply(k1, 1, x)
    r2a, fa = _apply(k2, 2, s)
    r2b, s = _apply(k2, 2, x)
    r1b, fb = _apply(k1, 1, s)
    return (r1a, r2a, fa) == (r1b, r2b, fb)


CLASS_BIT = {frozenset(["W"]): 1, frozenset(["W", "R"]): 2, frozenset(["W", "A"]): 4, frozenset(["A", "R"]): 8}


def races(evs, positions):
    """Race records implied by the interleavings: {(epoch, addr): (t1, t2, classbits, pclo, pchi)}."""
    n = len(evs)
    acc = []   # (tid, index, epoch, kind, addr, pc)
    for t in range(n):
        ep = 0
        for k, e in enumerate(evs[t]):
            if e[0] == "B":
                ep += 1
            else:
                acc.append((t, k, ep, e[0], e[1], e[2]))
    out = {}
    pcs: Dict[Tuple[int, int], List[int]] = {}
    for (t, k, ep, kind, addr, pc) in acc:
        pcs.setdefault((ep, addr), []).append(pc)
    for x in range(len(acc)):
        for y in range(len(acc)):
            t1, k1, e1, kd1, a1, _ = acc[x]
            t2, k2, e2, kd2, a2, _ = acc[y]
            if t1 >= t2 or a1 != a2 or commute(kd1, kd2):
                continue
            fwd = any(p[t1] > k1 and p[t2] <= k2 for p in positions)
            bwd = any(p[t2] > k2 and p[t1] <= k1 for p in positions)
            if not (fwd and bwd):
                continue
            assert e1 == e2
            key = (e1, a1)
            bit = CLASS_BIT[frozenset([kd1, kd2])]
            old = out.get(key)
            pair = (t1, t2)
            if old is None:
                out[key] = (pair, bit)
            else:
                out[key] = (min(old[0], pair), old[1] | bit)
    return {k: (v[0][0], v[0][1], v[1], min(pcs[k]), max(pcs[k])) for k, v in out.items()}
