"""Programs whose launches use several streams and event waits (Sec. 2 kernel configuration;
Sec. 3, streams and events), with their outcomes derived by hand.

Three kernels over a 4-thread block:
  WRITE  global[r0 + tid] = r1 + tid
  STALL  thread 0 exits, the others wait at a barrier: a deadlock (Sec. 3.1)
  COPY   global[r1 + tid] = global[r0 + tid] + 1
"""
import numpy as np

from paper_1211_6193_gb300.workloads import ir

WRITE, STALL, COPY = 0, 1, 2


def _code():
    a = ir.Asm()
    entries = [a.pc]
    a.s2r(ir.r2, ir.TID).add(ir.r3, ir.r0, ir.r2).add(ir.r4, ir.r1, ir.r2).stg(ir.r3, ir.r4).exit()
    entries.append(a.pc)
    a.s2r(ir.r2, ir.TID).brz(ir.r2, "stall_exit").bar().label("stall_exit").exit()
    entries.append(a.pc)
    a.s2r(ir.r2, ir.TID).add(ir.r3, ir.r0, ir.r2).ldg(ir.r4, ir.r3).add(ir.r4, ir.r4, 1)
    a.add(ir.r5, ir.r1, ir.r2).stg(ir.r5, ir.r4).exit()
    return a.assemble(), entries


def _launch(kernel, params=(), stream=0, wait=-1, grid=1):
    return ir.Launch(kernel, grid, 4, 0, params, stream=stream, wait=wait)


def fork_join(streams=True):
    """Launch 0 deadlocks on stream 0.  With streams:
      1 (stream 1)          WRITE [0, 4)   = 10..13   runs: nothing before it on stream 1
      2 (stream 0)          WRITE [4, 8)   = 20..23   skipped: follows the stopped launch 0
      3 (stream 1)          COPY  [0, 4) -> [8, 12)   runs: 11..14
      4 (stream 2, waits 0) WRITE [12, 16) = 30..33   skipped: waits for the stopped launch 0
      5 (stream 2)          WRITE [16, 20) = 40..43   skipped: follows the skipped launch 4
      6 (stream 3, waits 3) COPY  [8, 12) -> [20, 24) runs: 12..15
    With every launch on stream 0 and no waits, everything after launch 0 is skipped."""
    code, entries = _code()
    if streams:
        launches = [_launch(STALL), _launch(WRITE, (0, 10), stream=1), _launch(WRITE, (4, 20)),
                    _launch(COPY, (0, 8), stream=1), _launch(WRITE, (12, 30), stream=2, wait=0),
                    _launch(WRITE, (16, 40), stream=2), _launch(COPY, (8, 20), stream=3, wait=3)]
    else:
        launches = [_launch(STALL), _launch(WRITE, (0, 10)), _launch(WRITE, (4, 20)), _launch(COPY, (0, 8)),
                    _launch(WRITE, (12, 30)), _launch(WRITE, (16, 40)), _launch(COPY, (8, 20))]
    return ir.Program(code, entries, launches, np.full(24, -1, np.int32), name="fork_join" + ("" if streams else "_1"))


def fork_join_expected(streams=True):
    want = np.full(24, -1, np.int32)
    if streams:
        want[0:4] = [10, 11, 12, 13]
        want[8:12] = [11, 12, 13, 14]
        want[20:24] = [12, 13, 14, 15]
    return want


def conflicting(kind):
    """Two launches on different streams touching the same words: "ww" both write [0, 4)
    (4 conflicting words), "rw" one writes [0, 4) while the other copies it (4), "ordered" is
    "ww" with the second waiting for the first (none)."""
    code, entries = _code()
    first = _launch(WRITE, (0, 10))
    second = {"ww": _launch(WRITE, (0, 50), stream=1), "rw": _launch(COPY, (0, 8), stream=1),
              "ordered": _launch(WRITE, (0, 50), stream=1, wait=0)}[kind]
    return ir.Program(code, entries, [first, second], np.zeros(12, np.int32), name="conflict_" + kind)


def all_programs():
    """Well-formed stream programs for parity: the fork/join pattern, its one-stream form,
    and eight independent streams of three dependent launches with a join at the end."""
    code, entries = _code()
    wide = []
    for s in range(8):                       # 8 streams of 3 dependent launches
        base = 24 * s
        wide += [ir.Launch(WRITE, 1, 4, 0, (base, 100 * s), stream=s),
                 ir.Launch(COPY, 1, 4, 0, (base, base + 4), stream=s),
                 ir.Launch(COPY, 1, 4, 0, (base + 4, base + 8), stream=s)]
    wide.append(ir.Launch(COPY, 1, 4, 0, (8, 200), stream=9, wait=2))       # joins stream 0
    prog_wide = ir.Program(code, entries, wide, np.zeros(208, np.int32), name="wide_streams")
    return [fork_join(True), fork_join(False), prog_wide]


def _ancestors(launches, l):
    """Launches ordered before launch l: its stream predecessors and waits, transitively."""
    seen, todo = set(), [l]
    while todo:
        m = todo.pop()
        prev = next((k for k in range(m - 1, -1, -1) if launches[k].stream == launches[m].stream), None)
        for d in (prev, launches[m].wait if launches[m].wait >= 0 else None):
            if d is not None and d not in seen:
                seen.add(d)
                todo.append(d)
    return seen


def random_programs(seed, count):
    """Seeded programs of 1-4 streams, 1-12 launches, random event waits and a few deadlocking
    launches.  Launch l writes only words [4l, 4l + 4) and copies only from a launch ordered
    before it, so no two unordered launches share a written word (well-formed by construction)."""
    rng = np.random.default_rng(seed)
    code, entries = _code()
    out = []
    for p in range(count):
        nstreams, nl = int(rng.integers(1, 5)), int(rng.integers(1, 13))
        launches = []
        for l in range(nl):
            stream = int(rng.integers(0, nstreams))
            wait = int(rng.integers(0, l)) if l and rng.random() < 0.3 else -1
            launches.append(ir.Launch(WRITE, 1, 4, 0, (4 * l, 0), stream=stream, wait=wait))
            anc = sorted(_ancestors(launches, l))
            r = rng.random()
            if r < 0.1:
                kind, params = STALL, ()
            elif anc and r < 0.6:
                kind, params = COPY, (4 * int(rng.choice(anc)), 4 * l)
            else:
                kind, params = WRITE, (4 * l, int(rng.integers(0, 1000)))
            launches[l] = ir.Launch(kind, 1, 4, 0, params, stream=stream, wait=wait)
        out.append(ir.Program(code, entries, launches, np.full(4 * nl, -1, np.int32), name=f"streams_{seed}_{p}"))
    return out
