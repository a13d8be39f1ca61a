"""Pins of the oracle's global-memory checks, each against something other than the oracle:
hand-derived values, closed forms, and exhaustive interleaving enumeration.

Sec. 3.1 defines a race as two threads touching one location with no synchronisation point
between them, at least one writing; the paper checks shared memory.  The global check
(``check_global``) applies the same definition to global words:
  - inside one block's barrier interval (GLOBAL_RACE, like RACE);
  - between blocks of one launch, which have no synchronisation point at all until the
    kernel call ends (Sec. 2) - any two accesses to a word from different blocks, one
    writing (GLOBAL_BLOCKS: block = b1, b = b2, the smallest pair);
  - between launches that no stream order or event wait orders (Sec. 3, streams and
    events; GLOBAL_LAUNCHES: launch = l1, b = l2, the smallest pair).
``check_interblock`` counts the global words two blocks of one launch touch, one writing.
"""
import numpy as np
import pytest

import oracle
from brute_force import enumerate_outcomes, races as bf_races
from paper_1211_6193_gb300.workloads import families, fig1, ir, stencil2d, tiny
from paper_1211_6193_gb300.workloads.ir import (BID, BDIM, RZ, TID, Asm, Launch, Program, r0, r1, r2, r3, r4,
                                                r5)

G_KINDS = (oracle.GLOBAL_RACE, oracle.GLOBAL_BLOCKS, oracle.GLOBAL_LAUNCHES)
WW, WR = oracle.CLS_WW, oracle.CLS_WR


def _pcs(code, op):
    return [pc for pc in range(len(code)) if (int(code["op_d_a_b"][pc]) & 0x3F) == op]


# ------------------------------------------------------------------ programs
def every_block_writes_word0(grid):
    """Thread 0 of every block stores its block index to word 0."""
    a = Asm()
    a.s2r(r0, TID).brnz(r0, "x").s2r(r1, BID).stg(RZ, r1, 0).label("x").exit()
    return Program(a.assemble(), [0], [Launch(0, grid, 1, 0, ())], np.zeros(8, np.int32), name=f"w0x{grid}")


def writer_and_reader(writer_block, lo_w, lo_r, n=4, grid=2):
    """Block `writer_block` stores words [lo_w, lo_w + n) (thread t: word lo_w + t); every other
    block loads words [lo_r, lo_r + n) and stores each value to its own slot 64 + 8 b + t."""
    a = Asm()
    a.s2r(r0, TID).s2r(r1, BID).seq(r2, r1, writer_block).brz(r2, "read")
    a.add(r3, r0, lo_w).mov(r4, 5).stg(r3, r4, 0).exit()
    a.label("read").add(r3, r0, lo_r).ldg(r4, r3, 0)
    a.mul(r5, r1, 8).add(r5, r5, r0).stg(r5, r4, 64).exit()
    return Program(a.assemble(), [0], [Launch(0, grid, n, 0, ())], np.zeros(128, np.int32), name="w_r")


def shift_in_place(n, grid=1, gap=0, barrier=False):
    """Block b, thread t: x = g[b * (n + gap) + t + 1]; (barrier); g[b * (n + gap) + t] = x."""
    a = Asm()
    a.s2r(r0, TID).s2r(r1, BID).mul(r1, r1, n + gap).add(r2, r1, r0)
    a.ldg(r3, r2, 1)
    if barrier:
        a.bar()
    a.stg(r2, r3, 0).exit()
    words = grid * (n + gap) + 2
    init = (np.arange(words, dtype=np.int32) * 7 + 3)
    return Program(a.assemble(), [0], [Launch(0, grid, n, 0, ())], init, name=f"shift{n}x{grid}")


# ------------------------------------------------------------------ inter-block diagnostic
def test_interblock_counter_counts_conflicting_words():
    for grid, want in ((1, 0), (2, 1), (5, 1)):
        r = oracle.run([every_block_writes_word0(grid)], check_interblock=True)
        assert r.interblock_conflicts == want, grid
        assert r.arenas[0][0] == grid - 1                   # blocks run in order in the oracle
    # block 0 writes words 0..3, block 1 reads words 2..5: words 2 and 3
    assert oracle.run([writer_and_reader(0, 0, 2)], check_interblock=True).interblock_conflicts == 2
    # the same with the roles swapped (the read comes first in block order)
    assert oracle.run([writer_and_reader(1, 0, 2)], check_interblock=True).interblock_conflicts == 2
    # disjoint words: none; three readers and one writer of four words: 4
    assert oracle.run([writer_and_reader(0, 0, 8)], check_interblock=True).interblock_conflicts == 0
    assert oracle.run([writer_and_reader(2, 0, 0, grid=4)], check_interblock=True).interblock_conflicts == 4


def test_interblock_counter_ignores_one_block_and_read_sharing():
    # one block whose four threads all write word 0: no second block
    a = Asm()
    a.s2r(r0, TID).stg(RZ, r0, 0).exit()
    p = Program(a.assemble(), [0], [Launch(0, 1, 4, 0, ())], np.zeros(4, np.int32))
    assert oracle.run([p], check_interblock=True).interblock_conflicts == 0
    # the Fig. 1 program and the generated workloads share no written word between blocks
    progs = [fig1.program(), stencil2d.program(log2w=6, steps=2, buggy_launch=1)]
    progs += families.batch(n_programs=16, seed=3, max_grid=5)
    assert oracle.run(progs, check_interblock=True).interblock_conflicts == 0


def test_interblock_counter_threaded_equals_serial():
    progs = [every_block_writes_word0(7), writer_and_reader(2, 0, 0, grid=9), writer_and_reader(0, 0, 2, grid=6)]
    a = oracle.run(progs, check_interblock=True)
    b = oracle.run(progs, check_interblock=True, nthreads=4)
    assert a.interblock_conflicts == b.interblock_conflicts == 1 + 4 + 2


# ------------------------------------------------------------------ races inside a block
def test_global_race_inside_a_block_closed_form():
    """Thread t loads g[t + 1] and stores g[t] in one interval: word w (1 <= w < n) is written
    by thread w and read by thread w - 1, a write-read race with pair (w - 1, w)."""
    for n in (2, 33, 100):
        p = shift_in_place(n)
        ldg, stg = _pcs(p.code, ir.LDG)[0], _pcs(p.code, ir.STG)[0]
        r = oracle.run([p], check_global=True)
        want = [(oracle.GLOBAL_RACE, 0, 0, 0, 0, w, (w - 1) << 16 | w, WR << 24 | ldg << 12 | stg)
                for w in range(1, n)]
        assert r.report_tuples() == want, n
        # round-lockstep: every load precedes every store, so the shift reads the old values
        assert np.array_equal(r.arenas[0][:n], p.global_init[1:n + 1])
        # the global check changes no memory and is off by default
        assert oracle.run([p]).report_tuples() == []
        assert np.array_equal(oracle.run([p]).arenas[0], r.arenas[0])


def test_a_barrier_separates_global_accesses():
    r = oracle.run([shift_in_place(64, barrier=True)], check_global=True)
    assert r.report_tuples() == []


def test_same_thread_load_and_store_is_not_a_race():
    a = Asm()
    a.s2r(r0, TID).ldg(r1, r0, 0).add(r1, r1, 1).stg(r0, r1, 0).ldg(r2, r0, 0).exit()
    p = Program(a.assemble(), [0], [Launch(0, 1, 40, 0, ())], np.zeros(40, np.int32))
    r = oracle.run([p], check_global=True)
    assert r.report_tuples() == [] and list(r.arenas[0]) == [1] * 40


@pytest.mark.parametrize("nthreads,nsteps,count,nwords,bar_rate",
                         [(2, 6, 40, 3, 0.25), (3, 4, 40, 3, 0.25), (3, 5, 16, 8, 0.7)])
def test_global_races_brute_force_interleavings(nthreads, nsteps, count, nwords, bar_rate):
    """Every interleaving of the threads' global accesses that respects the barriers: a word
    races iff some pair of accesses to it occurs in both orders and does not commute."""
    progs = tiny.tiny_global_batch(2000 + 10 * nthreads + nsteps, count, nthreads=nthreads, nsteps=nsteps,
                                   nwords=nwords, bar_rate=bar_rate)
    res = oracle.run(progs, check_global=True)
    rep = res.report_tuples()
    n_racy = 0
    for i, p in enumerate(progs):
        evs, outcomes, positions = enumerate_outcomes(p, space="global")
        expect = bf_races(evs, positions)
        got = {(r[4], r[5]): (r[6] >> 16, r[6] & 0xFFFF, r[7] >> 24, (r[7] >> 12) & 0xFFF, r[7] & 0xFFF)
               for r in rep if r[1] == i}
        assert all(r[0] == oracle.GLOBAL_RACE for r in rep if r[1] == i)
        assert got == expect, f"program {i}"
        canon = tuple(int(x) for x in res.arenas[i])
        assert canon in outcomes, f"program {i}: canonical image is not an interleaving outcome"
        if not expect:
            assert outcomes == {canon}, f"program {i}: race-free yet several outcomes"
        else:
            n_racy += 1
    assert 0 < n_racy < count


# ------------------------------------------------------------------ races between blocks
def test_blocks_of_one_launch_race_hand_values():
    # every block writes word 0: write-write, smallest pair (0, 1), the one STG's pc
    p = every_block_writes_word0(3)
    stg = _pcs(p.code, ir.STG)[0]
    r = oracle.run([p], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_BLOCKS, 0, 0, 0, 0, 0, 1, WW << 24 | stg << 12 | stg)]
    # block 0 writes words 0..3 which blocks 1 and 2 read: write-read, pair (0, 1)
    p = writer_and_reader(0, 0, 0, grid=3)
    stg, ldg = _pcs(p.code, ir.STG)[0], _pcs(p.code, ir.LDG)[0]
    r = oracle.run([p], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_BLOCKS, 0, 0, 0, 0, w, 1, WR << 24 | stg << 12 | ldg)
                                 for w in range(4)]
    # block 2 writes words 0..3, blocks 0, 1, 3 read: smallest pair (0, 2)
    p = writer_and_reader(2, 0, 0, grid=4)
    r = oracle.run([p], check_global=True)
    assert [(t[3], t[5], t[6], t[7] >> 24) for t in r.report_tuples()] == [(0, w, 2, WR) for w in range(4)]


def test_two_writer_blocks_and_a_reader():
    """Blocks 1 and 2 store word 7, block 0 loads it: pairs (0, 1) and (0, 2) write-read,
    (1, 2) write-write; one record with both classes and pair (0, 1)."""
    a = Asm()
    a.s2r(r1, BID).brz(r1, "read").stg(RZ, r1, 7).exit()
    a.label("read").ldg(r2, RZ, 7).stg(RZ, r2, 9).exit()
    p = Program(a.assemble(), [0], [Launch(0, 3, 1, 0, ())], np.zeros(12, np.int32))
    stg, ldg = _pcs(p.code, ir.STG)[0], _pcs(p.code, ir.LDG)[0]
    r = oracle.run([p], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_BLOCKS, 0, 0, 0, 0, 7, 1, (WW | WR) << 24 | stg << 12 | ldg)]


def test_shift_across_block_boundaries_closed_form():
    """Blocks own adjacent ranges: thread n-1 of block b reads the first word of block b+1,
    which that block's thread 0 writes (a race between blocks on word (b+1) n, pair (b, b+1)),
    besides the n-1 races inside every block.  With a gap between the ranges only the races
    inside the blocks remain."""
    n, grid = 40, 5
    p = shift_in_place(n, grid=grid)
    ldg, stg = _pcs(p.code, ir.LDG)[0], _pcs(p.code, ir.STG)[0]
    r = oracle.run([p], check_global=True)
    inside = [(oracle.GLOBAL_RACE, 0, 0, b, 0, b * n + w, (w - 1) << 16 | w, WR << 24 | ldg << 12 | stg)
              for b in range(grid) for w in range(1, n)]
    between = [(oracle.GLOBAL_BLOCKS, 0, 0, b, 0, (b + 1) * n, b + 1, WR << 24 | ldg << 12 | stg)
               for b in range(grid - 1)]
    assert sorted(r.report_tuples()) == sorted(inside + between)
    r = oracle.run([shift_in_place(n, grid=grid, gap=3)], check_global=True)
    assert all(t[0] == oracle.GLOBAL_RACE for t in r.report_tuples()) and len(r.report_tuples()) == grid * (n - 1)


# ------------------------------------------------------------------ races between launches
def test_unordered_launches_race_hand_values():
    import stream_programs as sp
    # two streams write words 0..3: write-write, pair (0, 1)
    r = oracle.run([sp.conflicting("ww")], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_LAUNCHES, 0, 0, 0, 0, w, 1, WW << 24) for w in range(4)]
    # one writes 0..3 while the other copies them: write-read
    r = oracle.run([sp.conflicting("rw")], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_LAUNCHES, 0, 0, 0, 0, w, 1, WR << 24) for w in range(4)]
    # the second waits for the first: ordered, no race
    assert oracle.run([sp.conflicting("ordered")], check_global=True).report_tuples() == []


def test_three_unordered_launches():
    """Launches 0 and 1 (streams 0, 1) write words 0..3, launch 2 (stream 2) reads them:
    pairs (0, 1) write-write, (0, 2) and (1, 2) write-read."""
    import stream_programs as sp
    code, entries = sp._code()
    ls = [sp._launch(sp.WRITE, (0, 10)), sp._launch(sp.WRITE, (0, 50), stream=1),
          sp._launch(sp.COPY, (0, 8), stream=2)]
    p = Program(code, entries, ls, np.zeros(12, np.int32))
    r = oracle.run([p], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_LAUNCHES, 0, 0, 0, 0, w, 1, (WW | WR) << 24) for w in range(4)]
    # launch 2 waits for launch 1, which does not order it after launch 0: (0, 1), (0, 2) remain
    ls[2] = sp._launch(sp.COPY, (0, 8), stream=2, wait=1)
    r = oracle.run([Program(code, entries, ls, np.zeros(12, np.int32))], check_global=True)
    assert r.report_tuples() == [(oracle.GLOBAL_LAUNCHES, 0, 0, 0, 0, w, 1, (WW | WR) << 24) for w in range(4)]
    # launch 1 waits for launch 0 and launch 2 for launch 1: everything ordered
    ls[1] = sp._launch(sp.WRITE, (0, 50), stream=1, wait=0)
    assert oracle.run([Program(code, entries, ls, np.zeros(12, np.int32))], check_global=True).report_tuples() == []


def test_well_formed_stream_programs_have_no_global_races():
    import stream_programs as sp
    progs = sp.all_programs() + sp.random_programs(7, 40)
    a = oracle.run(progs, check_global=True)
    b = oracle.run(progs)
    assert a.report_tuples() == b.report_tuples()


# ------------------------------------------------------------------ race-free workloads
def test_global_check_adds_nothing_to_the_paper_and_generated_workloads():
    """Fig. 1 and its variants (the paper reports no global problem), the reduction, the
    stencil and a generated batch: the global check adds no record and changes nothing."""
    progs = [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True),
             families.reduction_plain(n_blocks=6), stencil2d.program(log2w=6, steps=3, buggy_launch=1)]
    progs += families.batch(n_programs=24, seed=3, max_grid=4, bug_rate=0.5)
    a = oracle.run(progs, check_global=True)
    b = oracle.run(progs)
    assert a.report_tuples() == b.report_tuples()
    assert all(np.array_equal(x, y) for x, y in zip(a.arenas, b.arenas))


# ------------------------------------------------------------------ block ranges
def test_a_block_range_runs_those_blocks_of_the_grid():
    """A launch restricted to blocks [b0, b1) of its grid (a process's share) runs exactly those
    blocks with their grid numbering: their reports and the words they write equal the whole
    grid's, restricted to them."""
    from dataclasses import replace
    p = families.reduction_plain(n_blocks=9, bdim=128, seed=1, omit_level=2)
    full = oracle.run([p])
    for b0, b1 in ((0, 3), (3, 9), (4, 5)):
        q = Program(p.code, p.kernel_entry, [replace(p.launches[0], block_begin=b0, block_count=b1 - b0)],
                    p.global_init)
        part = oracle.run([q])
        assert part.report_tuples() == [t for t in full.report_tuples() if b0 <= t[3] < b1]
        out = p.meta["n"]                    # block b writes its sum to word n + b
        got = part.arenas[0]
        assert np.array_equal(got[out + b0:out + b1], full.arenas[0][out + b0:out + b1])
        assert not np.any(got[out:out + b0]) and not np.any(got[out + b1:out + 9])
    with pytest.raises(ValueError):          # a range past the grid is rejected
        oracle.run([Program(p.code, p.kernel_entry, [replace(p.launches[0], block_begin=8, block_count=2)],
                            p.global_init)])
