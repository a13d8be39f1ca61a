"""GPU parity of the global-memory race check (sr_opts.check_global) against the oracle.

Reports (kinds 9-11 and everything else) are compared exactly.  Arenas are compared word for
word except where a race between blocks or between unordered launches makes a value depend on
timing: the GPU runs such blocks (and, in batched mode, such launches) at the same time while
the oracle runs them in order, so both results are correct executions; those words are masked,
each mask derived from the program's structure below.
"""
import numpy as np
import pytest

import oracle
import stream_programs as sp
from paper_1211_6193_gb300.workloads import families, fig1, stencil2d, tiny
from test_oracle_global import every_block_writes_word0, shift_in_place, writer_and_reader

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


def assert_parity(B, progs, mode, masks=None, **opts):
    want = oracle.run(progs, check_global=True)
    got = B.check(progs, mode=mode, check_global=True, **opts)
    gt, wt = got.report_tuples(), want.report_tuples()
    if gt != wt:
        gs, ws = set(gt), set(wt)
        raise AssertionError(f"{mode}: reports differ: {len(gt)} vs {len(wt)}; "
                             f"extra {sorted(gs - ws)[:5]} missing {sorted(ws - gs)[:5]}")
    for i in range(len(progs)):
        keep = np.ones(want.arenas[i].size, dtype=bool)
        if masks and masks.get(i) is not None:
            keep[np.asarray(masks[i], dtype=np.int64)] = False
        if not np.array_equal(got.arenas[i][keep], want.arenas[i][keep]):
            bad = np.nonzero((got.arenas[i] != want.arenas[i]) & keep)[0]
            raise AssertionError(f"{mode}: program {i} ({progs[i].name}) arena differs at {bad[:8]}")
    assert list(got.status & 3) == list(want.status), (got.status, want.status)
    assert not np.any(got.status & (B.ST_LOG_OVERFLOW | B.ST_INTERNAL)), got.status
    return got, want


@pytest.mark.parametrize("mode", MODES)
def test_paper_and_generated_workloads_have_no_global_races(B, mode):
    progs = [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True),
             families.reduction_plain(n_blocks=8), stencil2d.program(log2w=7, steps=3, buggy_launch=1)]
    progs += families.batch(n_programs=24, seed=3, max_grid=6, bug_rate=0.5)
    got, _ = assert_parity(B, progs, mode)
    assert not any(r[0] >= B.GLOBAL_RACE for r in got.report_tuples())
    assert 0 < got.stats.global_records <= got.stats.global_accesses     # in-bounds accesses are logged


@pytest.mark.parametrize("mode", MODES)
def test_races_inside_blocks(B, mode):
    progs = [shift_in_place(n) for n in (2, 31, 33, 100, 1024)] + [shift_in_place(64, barrier=True)]
    progs += tiny.tiny_global_batch(2033, 40, nthreads=3, nsteps=6, nwords=3)
    progs += tiny.tiny_global_batch(2034, 20, nthreads=40, nsteps=6, nwords=5)
    got, _ = assert_parity(B, progs, mode)
    assert sum(r[0] == B.GLOBAL_RACE for r in got.report_tuples()) > 1000


@pytest.mark.parametrize("mode", MODES)
def test_races_between_blocks(B, mode):
    n, grid = 40, 5
    progs = [every_block_writes_word0(1), every_block_writes_word0(9), writer_and_reader(0, 0, 2),
             writer_and_reader(2, 0, 0, grid=4), shift_in_place(n, grid=grid), shift_in_place(n, grid=grid, gap=3)]
    masks = {1: [0],                                              # last writer of word 0
             2: [64 + 8 + t for t in range(4)],                   # block 1 copied words 2..5
             3: [64 + 8 * b + t for b in (0, 1, 3) for t in range(4)],
             4: [b * n + n - 1 for b in range(grid - 1)]}         # the reads of the next block's word
    assert_parity(B, progs, mode, masks)


def test_races_between_blocks_many_tiles(B):
    """300 blocks of 1024 threads shifting one array in place: 307,200 records, 150 sort tiles
    and 3 digit passes, 299 races between neighbouring blocks, 1023 inside every block."""
    n, grid = 1024, 300
    p = shift_in_place(n, grid=grid)
    for mode in MODES:
        got, _ = assert_parity(B, [p], mode, {0: [b * n + n - 1 for b in range(grid - 1)]})
        kinds = [r[0] for r in got.report_tuples()]
        assert kinds.count(B.GLOBAL_BLOCKS) == grid - 1 and kinds.count(B.GLOBAL_RACE) == grid * (n - 1)


def test_races_between_unordered_launches(B):
    code, entries = sp._code()
    three = [sp._launch(sp.WRITE, (0, 10)), sp._launch(sp.WRITE, (0, 50), stream=1),
             sp._launch(sp.COPY, (0, 8), stream=2)]
    from paper_1211_6193_gb300.workloads.ir import Program
    progs = [sp.conflicting("ww"), sp.conflicting("rw"), sp.conflicting("ordered"),
             Program(code, entries, three, np.zeros(12, np.int32), name="three"), sp.fork_join(True)]
    progs += sp.all_programs() + sp.random_programs(11, 30)
    # plain mode runs launches one after another in index order, like the oracle
    got, _ = assert_parity(B, progs, "plain")
    assert sum(r[0] == B.GLOBAL_LAUNCHES for r in got.report_tuples()) == 12
    # batched mode runs unordered launches at the same time: the racing words are timing-dependent
    assert_parity(B, progs, "batched", {0: range(4), 1: range(8, 12), 3: list(range(4)) + list(range(8, 12))})


def test_entry_buffer_grows_and_waves(B):
    """More global race entries than the first buffer holds (the run is repeated with a larger
    one), and launches split into several waves (a program whose launches are not all ordered
    stays in one wave)."""
    progs = [shift_in_place(1024, grid=12), sp.conflicting("ww"), shift_in_place(512, grid=3)]
    masks = {0: [b * 1024 + 1023 for b in range(11)], 2: [b * 512 + 511 for b in range(2)]}
    got, _ = assert_parity(B, progs, "plain", masks, report_cap=1000)
    assert len(got.reports) > 12000
    # 1 MB of log budget: the first program's 12 x 2048 global records (x 3 buffers) fill a wave
    got, _ = assert_parity(B, progs, "plain", masks, log_budget_mb=1)
    assert got.stats.waves >= 2
    got, _ = assert_parity(B, progs, "batched", {**masks, 1: range(4)}, log_budget_mb=1, use_graph=True)
    assert got.stats.waves >= 2


def test_global_check_changes_nothing_else(B):
    """With the check on, every other report, the arenas and the status are those of a run
    without it (plain and batched, the log path replacing the fused check)."""
    progs = families.batch(n_programs=32, seed=9, max_grid=5, bug_rate=0.5)
    for mode in MODES:
        a = B.check(progs, mode=mode, check_global=True, fused_check=True)
        b = B.check(progs, mode=mode)
        assert a.report_tuples() == b.report_tuples()
        assert all(np.array_equal(x, y) for x, y in zip(a.arenas, b.arenas))
