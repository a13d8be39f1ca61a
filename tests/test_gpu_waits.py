"""Failure detection on the GPU without a GPU fault: every device-side wait of the
interpreter is bounded by ``sr_opts.spin_limit``; a wait that runs out marks the program
SR_ST_INTERNAL, the block or launch stops, and the call returns with the GPU usable.

The programs below make two waits run out for certain with a limit of one poll:
  - the clock wait of a load (round-lockstep across warps): warp 0 reaches its load after
    a few thousand cheap rounds while warp 1 is still in a loop of memory instructions,
    each of which costs more than an ALU round;
  - the launch-dependency wait of the batched kernel: launch 1 (same stream) waits for a
    one-warp launch 0 that runs a loop of ~10^5 rounds.
The code-staging copy of each CTA is not governed by spin_limit (it waits only for its
own bulk copy), so it completes in both cases."""
import numpy as np
import pytest

import oracle
from paper_1211_6193_gb300.workloads.ir import Asm, Launch, Program, RZ, TID, r0, r1, r2, r3, r4

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def lopsided_block(fast_iters: int = 2000, slow_iters: int = 2000) -> Program:
    """Two warps: warp 0 counts down with ALU only, then loads; warp 1 loops over a shared
    load and store of its own word per iteration, then exits."""
    a = Asm()
    a.s2r(r0, TID).slt(r1, r0, 32).brz(r1, "slow")
    a.mov(r2, fast_iters).label("fast").sub(r2, r2, 1).brnz(r2, "fast")
    a.lds(r3, RZ, 0).stg(r0, r3, 0).exit()
    a.label("slow").mov(r2, slow_iters)
    a.label("loop").lds(r4, r0, 0).add(r4, r4, 1).sts(r0, r4, 0).sub(r2, r2, 1).brnz(r2, "loop")
    a.exit()
    return Program(a.assemble(), [0], [Launch(0, 1, 64, 64, ())], np.zeros(64, np.int32), name="lopsided")


def slow_then_dependent(iters: int = 100000) -> Program:
    """Launch 0: one warp counts down `iters` times, then thread 0 writes word 0.  Launch 1
    (same stream, so it follows launch 0): thread 0 writes word 1."""
    a = Asm()
    a.s2r(r0, TID).mov(r2, iters).label("loop").sub(r2, r2, 1).brnz(r2, "loop")
    a.brnz(r0, "done").mov(r3, 7).stg(RZ, r3, 0).label("done").exit()
    k1 = a.pc
    a.s2r(r0, TID).brnz(r0, "done1").mov(r3, 9).stg(RZ, r3, 1).label("done1").exit()
    return Program(a.assemble(), [0, k1], [Launch(0, 1, 32, 0, ()), Launch(1, 1, 32, 0, ())],
                   np.zeros(4, np.int32), name="slow_then_dependent")


# warp 1 of the lopsided block logs 2 x 32 shared accesses per iteration: 128,000 records
LOG = 1 << 18


def test_programs_are_valid_and_race_free_without_a_limit(B):
    for p in (lopsided_block(), slow_then_dependent()):
        want = oracle.run([p])
        for mode in ("plain", "batched"):
            got = B.check([p], mode=mode, loop_log_records=LOG)
            assert got.report_tuples() == want.report_tuples() == [], (p.name, mode)
            assert np.array_equal(got.arenas[0], want.arenas[0]), (p.name, mode)
            assert int(got.status[0]) == 0, (p.name, mode)


@pytest.mark.parametrize("mode", ["plain", "batched"])
def test_clock_wait_runs_out(B, mode):
    p = lopsided_block()
    for _ in range(2):                    # the context stays usable: run twice
        got = B.check([p], mode=mode, spin_limit=1, loop_log_records=LOG)
        assert int(got.status[0]) & B.ST_INTERNAL, got.status
    # and an ordinary run afterwards is exact
    want = oracle.run([p])
    got = B.check([p], mode=mode, loop_log_records=LOG)
    assert np.array_equal(got.arenas[0], want.arenas[0]) and int(got.status[0]) == 0


def test_launch_dependency_wait_runs_out(B):
    p = slow_then_dependent()
    got = B.check([p], mode="batched", spin_limit=1)
    st = int(got.status[0])
    assert st & B.ST_INTERNAL, st
    # launch 0 finished; launch 1 gave up waiting for it and was skipped
    assert got.arenas[0][0] == 7 and got.arenas[0][1] == 0
    # plain mode orders launches on the CUDA stream and has no such wait
    got = B.check([p], mode="plain", spin_limit=1)
    assert int(got.status[0]) == 0 and got.arenas[0][0] == 7 and got.arenas[0][1] == 9
