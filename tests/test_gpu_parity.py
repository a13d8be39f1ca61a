"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work: final global arenas, the sorted report set and the program status must
match bit for bit.  Sizes here span several tiles, ragged block sizes and every edge
case of the method; the full-size workloads are checked on sampled blocks and through
closed forms that hold at any size.
"""
import numpy as np
import pytest

import oracle
from paper_1211_6193_gb300.workloads import families, fig1, ir, stencil2d, tiny

pytestmark = pytest.mark.gpu

MODES = ["plain", "batched"]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def assert_parity(B, progs, mode="plain", oracle_kw=None, **opts):
    want = oracle.run(progs, **(oracle_kw or {}))
    got = B.check(progs, mode=mode, **opts)
    gt, wt = got.report_tuples(), want.report_tuples()
    if gt != wt:
        gs, ws = set(gt), set(wt)
        raise AssertionError(f"{mode}: reports differ: {len(gt)} vs {len(wt)}; "
                             f"extra {sorted(gs - ws)[:5]} missing {sorted(ws - gs)[:5]}")
    for i in range(len(progs)):
        if not np.array_equal(got.arenas[i], want.arenas[i]):
            bad = np.nonzero(got.arenas[i] != want.arenas[i])[0]
            raise AssertionError(f"{mode}: program {i} ({progs[i].name}) arena differs at {bad[:8]} "
                                 f"got {got.arenas[i][bad[:8]]} want {want.arenas[i][bad[:8]]}")
    assert list(got.status & 3) == list(want.status), (got.status, want.status)
    assert not np.any(got.status & (B.ST_LOG_OVERFLOW | B.ST_INTERNAL)), got.status
    return got, want


@pytest.mark.parametrize("mode", MODES)
def test_fig1_and_variants(B, mode):
    progs = [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True)]
    got, _ = assert_parity(B, progs, mode)
    assert got.arenas[0][fig1.OUT_OFF] == 767


@pytest.mark.parametrize("mode", MODES)
def test_tiny_interleaving_programs(B, mode):
    progs = tiny.tiny_batch(77, 60, nthreads=3, nsteps=6, nwords=3)
    progs += tiny.tiny_batch(78, 30, nthreads=40, nsteps=6, nwords=5)     # two warps
    assert_parity(B, progs, mode)


@pytest.mark.parametrize("mode", MODES)
def test_family_batch_with_planted_bugs(B, mode):
    progs = families.batch(n_programs=48, seed=3, max_grid=6, bug_rate=0.5)
    assert_parity(B, progs, mode)


@pytest.mark.parametrize("mode", MODES)
def test_plain_reduction_scaled(B, mode):
    p = families.reduction_plain(n_blocks=40, bdim=1024, seed=1, omit_level=3)
    got, _ = assert_parity(B, [p], mode)
    assert len(got.reports) == 40 * 32


@pytest.mark.parametrize("mode", MODES)
def test_stencil2d_scaled(B, mode):
    p = stencil2d.program(log2w=7, steps=4, buggy_launch=2, seed=4)
    got, _ = assert_parity(B, [p], mode)
    assert len(got.reports) == 16 * 1024


def _lockstep_programs():
    out = []
    a = ir.Asm()      # same-round load vs store, atomics after stores, min-pc order
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 5).brnz(ir.r3, "w1")
    a.sts(ir.RZ, ir.r4).sts(ir.RZ, ir.r4, 1).bra("join")
    a.label("w1").lds(ir.r5, ir.RZ).mov(ir.r6, 1).atoms(ir.RZ, ir.r6, 1).lds(ir.r7, ir.RZ)
    a.stg(ir.r2, ir.r5).stg(ir.r2, ir.r7, 64)
    a.label("join").sts(ir.RZ, ir.r2, 2)
    a.slt(ir.r8, ir.r2, 16).brnz(ir.r8, "hi").mov(ir.r9, 0).mov(ir.r9, 0).mov(ir.r9, 0)
    a.lds(ir.r9, ir.RZ, 3).stg(ir.r2, ir.r9, 128).bra("end")
    a.label("hi").mov(ir.r9, 7).sts(ir.RZ, ir.r9, 3)
    a.label("end").bar()
    a.brnz(ir.r2, "out").lds(ir.r10, ir.RZ).stg(ir.RZ, ir.r10, 192).lds(ir.r10, ir.RZ, 1)
    a.stg(ir.RZ, ir.r10, 193).lds(ir.r10, ir.RZ, 2).stg(ir.RZ, ir.r10, 194).lds(ir.r10, ir.RZ, 3)
    a.stg(ir.RZ, ir.r10, 195).label("out").exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 3, 64, 4, ())], np.full(196, -1, np.int32)))
    a = ir.Asm()      # many warps storing to one word in one round: highest tid wins
    a.s2r(ir.r2, ir.TID).sts(ir.RZ, ir.r2).sts(ir.r2, ir.r2, 1).bar().brnz(ir.r2, "x")
    a.lds(ir.r3, ir.RZ).stg(ir.RZ, ir.r3).label("x").exit()
    for bdim in (64, 1000, 1024):
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, bdim, 1025, ())], np.zeros(1, np.int32)))
    a = ir.Asm()      # stores and atomic adds to the same word in one round
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 10).mov(ir.r5, 1).brnz(ir.r3, "w1")
    a.sts(ir.RZ, ir.r4).bra("j")
    a.label("w1").atoms(ir.RZ, ir.r5).label("j").bar()
    a.brnz(ir.r2, "x").lds(ir.r6, ir.RZ).stg(ir.RZ, ir.r6).label("x").exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 256, 1, ())], np.zeros(1, np.int32)))
    return out


@pytest.mark.parametrize("mode", MODES)
def test_round_semantics_programs(B, mode):
    assert_parity(B, _lockstep_programs(), mode)


def _edge_programs():
    out = []
    p = fig1.program()
    out.append(ir.Program(p.code, [0], [], np.arange(5, dtype=np.int32), name="no_launch"))
    a = ir.Asm()      # errors: x/0, x%0, shared and global out of bounds
    a.s2r(ir.r2, ir.TID).mov(ir.r4, 5).div(ir.r6, ir.r4, ir.RZ).rem(ir.r7, ir.r4, 0).add(ir.r8, ir.r2, -3)
    a.lds(ir.r9, ir.r8).ldg(ir.r10, ir.r2, 100).sts(ir.r2, ir.r2, -3).bar().atoms(ir.r2, ir.r4, -4)
    a.add(ir.r11, ir.r6, ir.r7).add(ir.r11, ir.r11, ir.r9).add(ir.r11, ir.r11, ir.r10).stg(ir.r2, ir.r11)
    a.stg(ir.r2, ir.r2, 1).exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 40, 4, (0,))], np.full(40, 77, np.int32)))
    a = ir.Asm()      # no shared memory at all, 1-thread blocks, ragged block sizes
    a.s2r(ir.r2, ir.TID).s2r(ir.r3, ir.BID).s2r(ir.r4, ir.BDIM).mul(ir.r5, ir.r3, ir.r4).add(ir.r5, ir.r5, ir.r2)
    a.mul(ir.r6, ir.r5, 3).add(ir.r6, ir.r6, 1).stg(ir.r5, ir.r6).exit()
    for g, b in ((1, 1), (7, 33), (3, 1000), (2, 1024)):
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, g, b, 0, ())], np.zeros(g * b, np.int32)))
    a = ir.Asm()      # the largest shared array: every thread sweeps 12 words of 12288
    a.s2r(ir.r2, ir.TID)
    for j in range(12):
        a.sts(ir.r2, ir.r2, 1024 * j)
    a.bar()
    for j in range(12):
        a.lds(ir.r3, ir.r2, 1024 * j).add(ir.r4, ir.r4, ir.r3)
    a.stg(ir.r2, ir.r4).exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 1024, 12288, ())], np.zeros(1024, np.int32)))
    a = ir.Asm()      # endless loop stopped by the round budget; the next launch is skipped
    a.s2r(ir.r2, ir.TID).label("top").add(ir.r3, ir.r3, 1).sts(ir.r2, ir.r3).bra("top")
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 70, 70, ()), ir.Launch(0, 1, 32, 32, ())],
                          np.zeros(1, np.int32), name="budget"))
    # a 4096-instruction program (filler) with a reduction tail
    spec = families.FamilySpec("reduction", 3, 96, 96, 4096 - 64, None, 0)
    out.append(families.build_family(spec, seed=4))
    return out


@pytest.mark.parametrize("mode", MODES)
def test_edge_cases(B, mode):
    progs = _edge_programs()
    assert max(p.ncode for p in progs) <= ir.MAX_CODE
    assert_parity(B, progs, mode, oracle_kw={"round_budget": 3000}, round_budget=3000,
                  loop_log_records=1 << 18)


def _large_interval_programs():
    """Barrier intervals of 1, 2, 3 and 6 tiles of 2048 records, some ending exactly on a
    tile boundary, with write-read races on a few words between them."""
    out = []
    for k in (2, 4, 6, 3):
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID)
        for j in range(k):                           # k stores per thread: k * 1024 records
            a.sts(ir.r2, ir.r2, 1024 * j)
        a.bar()
        for j in range(k):                           # k loads per thread, one of them racy below
            a.lds(ir.r3, ir.r2, 1024 * j).add(ir.r4, ir.r4, ir.r3)
        a.and_(ir.r5, ir.r2, 7).sts(ir.r5, ir.r2)    # 1024 stores to 8 words in the same interval
        a.bar().stg(ir.r2, ir.r4).exit()
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 3, 1024, 1024 * k, ())], np.zeros(1024, np.int32)))
    return out


def _uneven_block_logs_programs():
    """Blocks whose logs differ in length from block to block: block b has (389 b) mod
    (bdim + 7) active threads (none when b is a multiple of 5), each making three stores, a
    load and, in blocks with b mod 3 = 1 where the second barrier is skipped, a racing store.
    Record counts are odd and even, some blocks log nothing, and with 96-thread blocks a work
    item of the race check holds many blocks, so staged copies run across block ends."""
    out = []
    for bdim, grid in ((96, 200), (1024, 24)):
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID).s2r(ir.r3, ir.BID)
        a.mul(ir.r4, ir.r3, 389).rem(ir.r4, ir.r4, bdim + 7)
        a.rem(ir.r5, ir.r3, 5).sne(ir.r5, ir.r5, 0).mul(ir.r4, ir.r4, ir.r5)
        a.slt(ir.r7, ir.r2, ir.r4).brz(ir.r7, "skip")
        for j in range(3):
            a.sts(ir.r2, ir.r2, bdim * j)
        a.label("skip").bar().brz(ir.r7, "skip2")
        a.add(ir.r8, ir.r2, 1).rem(ir.r8, ir.r8, ir.r4).lds(ir.r9, ir.r8)
        a.label("skip2").rem(ir.r10, ir.r3, 3).seq(ir.r10, ir.r10, 1).brnz(ir.r10, "nobar").bar()
        a.label("nobar").brz(ir.r7, "out").sts(ir.r2, ir.r9)
        a.label("out").mul(ir.r11, ir.r3, bdim).add(ir.r11, ir.r11, ir.r2).stg(ir.r11, ir.r9).exit()
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, grid, bdim, 3 * bdim, ())],
                              np.zeros(grid * bdim, np.int32)))
    return out


@pytest.mark.parametrize("mode", MODES)
def test_blocks_with_uneven_logs(B, mode):
    assert_parity(B, _uneven_block_logs_programs(), mode)


@pytest.mark.parametrize("mode", MODES)
def test_intervals_larger_than_a_staged_tile(B, mode):
    assert_parity(B, _large_interval_programs(), mode)


def _many_racy_addresses_programs():
    """One interval with more racy words than one round of exact summaries holds (3072):
    thread t and t ^ 1 both store to words t + 1024 j (j < k), a write-write race per
    word; k = 8 gives 8192 racy words, k = 3 exactly 3072, and a read of each word by a
    third thread adds the write-read class."""
    out = []
    for k, extra_read in ((8, False), (3, False), (12, True)):
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID).xor(ir.r3, ir.r2, 1)
        for j in range(k):
            a.sts(ir.r2, ir.r2, 1024 * j).sts(ir.r3, ir.r2, 1024 * j)
        if extra_read:
            a.xor(ir.r4, ir.r2, 2)
            for j in range(k):
                a.lds(ir.r5, ir.r4, 1024 * j).add(ir.r6, ir.r6, ir.r5)
        a.bar().stg(ir.r2, ir.r6).exit()
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 1024, 1024 * k, ())], np.zeros(1024, np.int32)))
    return out


@pytest.mark.parametrize("mode", MODES)
def test_more_racy_words_than_one_summary_round(B, mode):
    got, _ = assert_parity(B, _many_racy_addresses_programs(), mode)
    races = [r for r in got.report_tuples() if r[0] == oracle.RACE]
    assert len(races) == 2 * (8 + 3 + 12) * 1024


@pytest.mark.parametrize("variant", range(1, 8))
def test_every_check_variant(B, variant):
    """Each race-check kernel shape on its own: the table sized to small and large shared
    arrays, intervals with more racy words than a summary round holds, intervals spanning
    stages, blocks of uneven (and empty) logs in one work item, and a batch of generated
    programs with planted bugs."""
    groups = [  # one batch each, so that each sizes the table to its own largest shared array
        _many_racy_addresses_programs(), _large_interval_programs()[:2], _uneven_block_logs_programs(),
        families.batch(n_programs=24, seed=31, max_grid=12, bug_rate=0.5),
        [fig1.program(race=True)], [families.reduction_plain(n_blocks=20, bdim=256, seed=2, omit_level=2)],
        [stencil2d.program(log2w=6, steps=3, buggy_launch=1, seed=5)],
    ]
    for progs in groups:
        for mode in MODES:
            assert_parity(B, progs, mode, check_variant=variant)


def _uninit_programs():
    out = []
    a = ir.Asm()     # warp 0 writes, everyone reads after the barrier
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).brnz(ir.r3, "skip").sts(ir.r2, ir.r2).label("skip").bar()
    a.lds(ir.r4, ir.r2).stg(ir.r2, ir.r4).exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 3, 100, 100, ())], np.zeros(100, np.int32)))
    for delay in (0, 1, 3):   # a load in the same round as the store, one and three rounds later
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 5).brnz(ir.r3, "w1").sts(ir.RZ, ir.r4).bra("end")
        a.label("w1")
        for _ in range(delay):
            a.mov(ir.r9, 0)
        a.lds(ir.r5, ir.RZ).label("end").exit()
        out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 64, 1, ())], np.zeros(1, np.int32)))
    a = ir.Asm()     # atomics initialise; loads of a word written only in a later interval
    a.s2r(ir.r2, ir.TID).mov(ir.r3, 1).atoms(ir.RZ, ir.r3).bar().lds(ir.r4, ir.RZ).lds(ir.r5, ir.RZ, 1)
    a.lds(ir.r6, ir.r2, 2).bar().brnz(ir.r2, "x").sts(ir.RZ, ir.r3, 1).label("x").exit()
    out.append(ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 40, 64, ())], np.zeros(1, np.int32)))
    return out


@pytest.mark.parametrize("mode", MODES)
def test_uninitialised_shared_reads(B, mode):
    groups = [_uninit_programs(), families.batch(n_programs=40, seed=8, max_grid=6, bug_rate=0.5),
              [families.reduction_plain(n_blocks=6, bdim=512, seed=3, omit_level=None)]]
    for progs in groups:
        got, _ = assert_parity(B, progs, mode, oracle_kw={"check_uninit": True}, check_uninit=True)
    assert any(r[0] == oracle.ERR_UNINIT_SHARED for r in assert_parity(
        B, _uninit_programs(), mode, oracle_kw={"check_uninit": True}, check_uninit=True)[0].report_tuples())


@pytest.mark.parametrize("mode", MODES)
def test_fused_race_check(B, mode):
    """The interpreter keeping each word's summary itself (no access log): the same reports
    as the oracle on Figure 1, interleaving programs, generated batches with planted bugs,
    reductions, the 2-D stencil, reducing barriers, loops with barriers, deadlocks, more racy
    words than one round holds, shared arrays too large to fuse (they keep the log), and with
    the uninitialised-read check on."""
    from rbar_programs import all_programs
    groups = [
        [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True)],
        tiny.tiny_batch(5, 40),
        families.batch(n_programs=40, seed=17, max_grid=10, bug_rate=0.5),
        [families.reduction_plain(n_blocks=12, bdim=1024, seed=2, omit_level=3)],
        [stencil2d.program(log2w=6, steps=3, buggy_launch=1, seed=5)],
        all_programs(),
        _many_racy_addresses_programs(),
    ]
    for progs in groups:
        assert_parity(B, progs, mode, fused_check=True)
    assert_parity(B, _uninit_programs(), mode, oracle_kw={"check_uninit": True}, check_uninit=True,
                  fused_check=True)


def test_fused_race_check_matches_the_log_path_on_a_larger_batch(B):
    """128 generated programs (the first of the batched workload's seeded batch, every family
    and planted bug kind, shared arrays up to 48 KB, some too large to fuse): the fused check
    and the access log + race-check kernel give the same reports, arenas and status."""
    progs = families.batch(n_programs=128, seed=3)
    log = B.check(progs, mode="batched")
    fused = B.check(progs, mode="batched", fused_check=True)
    assert fused.report_tuples() == log.report_tuples()
    assert len(log.reports) > 0
    assert all(np.array_equal(a, b) for a, b in zip(fused.arenas, log.arenas))
    assert list(fused.status) == list(log.status)


@pytest.mark.parametrize("mode", MODES)
def test_streams_and_event_waits(B, mode):
    """Sec. 3, streams and events: launches of several streams with event waits (batched
    mode runs launches of different streams at the same time); a deadlock skips its own
    stream and what waits on it, and nothing else."""
    from stream_programs import all_programs, fork_join_expected
    got, _ = assert_parity(B, all_programs(), mode)
    assert np.array_equal(got.arenas[0], fork_join_expected(True))
    assert np.array_equal(got.arenas[1], fork_join_expected(False))


@pytest.mark.parametrize("mode", MODES)
def test_streams_on_random_dependency_graphs(B, mode):
    """Seeded programs of 1-4 streams with random event waits and deadlocking launches."""
    from stream_programs import random_programs
    assert_parity(B, random_programs(11, 40), mode)


def test_stream_wait_on_a_later_launch_is_rejected(B):
    import stream_programs as sp
    p = sp.fork_join(True)
    p.launches[2] = ir.Launch(0, 1, 4, 0, (4, 20), stream=0, wait=5)
    with pytest.raises(B.SimtCheckError):
        B.check([p])


@pytest.mark.parametrize("mode", MODES)
def test_reducing_barriers(B, mode):
    """__syncthreads_and/_or/_count: predicates over full and partial warps, reducing and
    plain barriers meeting, a deadlock at a reducing barrier, reducing barriers in a loop."""
    from rbar_programs import all_programs
    assert_parity(B, all_programs(), mode)


def test_race_check_disabled_keeps_memory_and_barrier_reports(B):
    progs = families.batch(n_programs=24, seed=8, max_grid=4, bug_rate=0.6)
    want = oracle.run(progs, check_races=False)
    got = B.check(progs, mode="batched", check_races=False)
    assert got.report_tuples() == want.report_tuples()
    assert all(np.array_equal(a, b) for a, b in zip(got.arenas, want.arenas))
    assert not any(r[0] == oracle.RACE for r in got.report_tuples())


def test_waves_and_graph_and_repeat(B):
    progs = families.batch(n_programs=40, seed=12, max_grid=12, bug_rate=0.4)
    want = oracle.run(progs)
    with B.Context(mode="batched", use_graph=True, log_budget_mb=1, report_cap=16) as ctx:
        with ctx.load_programs(progs) as b:
            for _ in range(3):                    # graph replays give identical results
                b.run_and_check()
                assert [tuple(int(x) for x in r) for r in b.fetch_reports()] == want.report_tuples()
                for i in range(len(progs)):
                    assert np.array_equal(b.fetch_memory(i), want.arenas[i])
            # the whole-batch forms: one copy of every arena (pageable and page-locked), every status
            for pinned in (False, True):
                whole = b.fetch_all_memory(pinned=pinned)
                assert len(whole) == len(progs)
                assert all(np.array_equal(x, w) for x, w in zip(whole, want.arenas))
            st = b.all_status()
            assert list(st) == [b.status(i) for i in range(len(progs))]
            assert list(st & 3) == list(want.status)


@pytest.mark.parametrize("use_graph", [False, True])
def test_report_buffer_grown_after_a_one_wave_run(B, use_graph):
    """More reports than the initial buffer holds, in one wave: only the emission runs again,
    and later runs of the same batch use the grown buffer."""
    progs = families.batch(n_programs=30, seed=21, max_grid=10, bug_rate=0.6)
    want = oracle.run(progs)
    assert len(want.report_tuples()) > 64
    with B.Context(mode="batched", use_graph=use_graph, report_cap=16) as ctx, ctx.load_programs(progs) as b:
        for _ in range(2):
            b.run_and_check()
            assert [tuple(int(x) for x in r) for r in b.fetch_reports()] == want.report_tuples()
            assert all(np.array_equal(x, w) for x, w in zip(b.fetch_all_memory(), want.arenas))


def test_context_memory_pool(B):
    """Without a caller allocator the context allocates from its own pool: batch after batch
    on one context (memory reused), both modes, results as the oracle's."""
    progs = families.batch(n_programs=12, seed=44, max_grid=10, bug_rate=0.5)
    want = oracle.run(progs)
    for mode in MODES:
        with B.Context(mode=mode, torch_allocator=False) as ctx:
            for _ in range(3):
                with ctx.load_programs(progs) as b:
                    b.run_and_check()
                    assert [tuple(int(x) for x in r) for r in b.fetch_reports()] == want.report_tuples()
                    assert all(np.array_equal(x, w) for x, w in zip(b.fetch_all_memory(), want.arenas))


def test_log_overflow_is_reported_not_silent(B):
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).mov(ir.r3, 50).label("l").sts(ir.r2, ir.r3).sub(ir.r3, ir.r3, 1).brnz(ir.r3, "l").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 64, ())], np.zeros(1, np.int32))
    got = B.check([p], loop_log_records=64)
    assert got.status[0] & B.ST_LOG_OVERFLOW


def test_full_size_plain_reduction(B):
    """The 2^24-element workload (16384 blocks x 1024 threads): block sums in closed form,
    the 32 races per block in closed form, and the first blocks against the oracle."""
    p = families.reduction_plain()
    got = B.check([p], mode="plain")
    n = 16384 * 1024
    sums = p.global_init[:n].astype(np.int64).reshape(16384, 1024).sum(axis=1).astype(np.int32)
    assert np.array_equal(got.arenas[0][n:], sums)
    assert got.status[0] == 0
    rep = got.reports
    assert len(rep) == 16384 * 32
    assert np.all(rep["kind"] == oracle.RACE) and np.all(rep["epoch"] == 4)
    j = np.tile(np.arange(32, dtype=np.uint32), 16384)
    assert np.array_equal(rep["block"], np.repeat(np.arange(16384, dtype=np.uint32), 32))
    assert np.array_equal(rep["a"], 32 + j) and np.array_equal(rep["b"], (j << 16) | (32 + j))
    want = oracle.run([p], max_blocks=8)
    assert got.report_tuples()[:8 * 32] == want.report_tuples()
    assert got.stats.shared_accesses == 16384 * 4094


def tag_wrap_program(iters: int = 300000) -> ir.Program:
    """One block of two threads runs `iters` barrier intervals: each thread stores its own
    word every interval (no race), and every 1024th interval thread t also reads word t + 1
    (thread 0's read races with thread 1's store of word 1).  More than 2^18 intervals on
    one checker CTA make the checker's 18-bit interval tags wrap."""
    from paper_1211_6193_gb300.workloads.ir import Asm, Launch, Program, TID, r0, r1, r2, r3, r4
    a = Asm()
    a.s2r(r0, TID).mov(r1, iters)
    a.label("loop").sts(r0, r1, 0).and_(r2, r1, 1023).seq(r3, r2, 0).brz(r3, "skip")
    a.lds(r4, r0, 1)
    a.label("skip").bar().sub(r1, r1, 1).brnz(r1, "loop").exit()
    return Program(a.assemble(), [0], [Launch(0, 1, 2, 3, ())], np.zeros(4, np.int32), name=f"tag_wrap_{iters}")


@pytest.mark.parametrize("variant", [0, 1, 5, 6, 7])
def test_checker_interval_tags_wrap(B, variant):
    p = tag_wrap_program()
    got, want = assert_parity(B, [p], "plain", check_variant=variant, loop_log_records=1 << 20)
    # iterations 300000, 299999, ... 1: the racy ones are those whose counter is a multiple of 1024
    assert len(got.reports) == 300000 // 1024
    assert all(r[0] == B.RACE and r[5] == 1 and r[6] == 1 for r in got.report_tuples())


def test_batched_two_ctas_per_sm(B):
    """Batched mode with two CTAs per SM (ctas_per_sm 2): the programs of large blocks run one
    block per CTA, the others in the persistent kernel - both kernels in one run, the stencil's
    four dependent launches in the first - with the same results."""
    progs = families.batch(n_programs=48, seed=3, max_grid=6, bug_rate=0.5)
    progs += [stencil2d.program(log2w=7, steps=4, buggy_launch=2, seed=4)]
    got, _ = assert_parity(B, progs, "batched", ctas_per_sm=2)
    assert 0 < got.stats.one_per_cta_blocks < got.stats.blocks, got.stats
    got, _ = assert_parity(B, progs, "batched", ctas_per_sm=2, use_graph=True)
    assert 0 < got.stats.one_per_cta_blocks < got.stats.blocks
    one, _ = assert_parity(B, progs, "batched", ctas_per_sm=1)
    assert one.stats.one_per_cta_blocks == 0


def _wide_stream_programs(seed, count, bdim=1024):
    """The seeded stream programs with blocks of `bdim` threads; launch l's words move to
    [bdim l, bdim (l + 1)), so that unordered launches still share none."""
    import stream_programs as sp
    out = []
    for p in sp.random_programs(seed, count):
        ls = []
        for l in p.launches:
            pr = tuple(l.params)
            if l.kernel == sp.WRITE:
                pr = (pr[0] // 4 * bdim, pr[1])
            elif l.kernel == sp.COPY:
                pr = (pr[0] // 4 * bdim, pr[1] // 4 * bdim)
            ls.append(ir.Launch(l.kernel, 1, bdim, 0, pr, stream=l.stream, wait=l.wait))
        out.append(ir.Program(p.code, p.kernel_entry, ls, np.full(bdim * len(ls), -1, np.int32),
                              name=p.name + f"_b{bdim}"))
    return out


def test_one_block_per_cta_streams_and_deadlocks(B):
    """Streams, event waits and deadlocking launches in the one-block-per-CTA kernel: its CTAs
    wait (bounded) for the launches their launch follows and skip what a stop skips."""
    progs = _wide_stream_programs(11, 24)
    got, _ = assert_parity(B, progs, "batched", ctas_per_sm=2)
    assert got.stats.one_per_cta_blocks == got.stats.blocks == sum(len(p.launches) for p in progs)
