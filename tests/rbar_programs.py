"""Programs that use __syncthreads_and/_or/_count (BARAND / BAROR / BARPOPC), for the GPU
parity tests: hand-checkable predicates over full and partial warps, reducing and plain
barriers meeting (divergence), a deadlock at a reducing barrier, and reducing barriers
inside a loop."""
import numpy as np

from paper_1211_6193_gb300.workloads import ir


def predicate_values(bdim, limit):
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, limit)
    a.bar_count(ir.r4, ir.r3).bar_and(ir.r5, ir.r3).bar_or(ir.r6, ir.r3)
    a.mul(ir.r7, ir.r2, 3).stg(ir.r7, ir.r4).stg(ir.r7, ir.r5, 1).stg(ir.r7, ir.r6, 2).exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, 2, bdim, 0, ())], np.full(3 * bdim, -1, np.int32),
                      name=f"rbar_values_{bdim}_{limit}")


def odd_count(bdim, grid=5, seed=0):
    vals = np.random.default_rng(seed).integers(-1000, 1000, grid * bdim, dtype=np.int32)
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).s2r(ir.r3, ir.BID).mul(ir.r4, ir.r3, bdim).add(ir.r4, ir.r4, ir.r2)
    a.ldg(ir.r5, ir.r4).and_(ir.r6, ir.r5, 1).bar_count(ir.r7, ir.r6)
    a.brnz(ir.r2, "x").stg(ir.r3, ir.r7, grid * bdim).label("x").exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, grid, bdim, 0, ())],
                      np.concatenate([vals, np.zeros(grid, np.int32)]), name=f"rbar_odd_{bdim}")


def mixed_with_plain(bdim=100, split=40):
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, split).brz(ir.r3, "plain")
    a.bar_count(ir.r4, ir.r3).bar_and(ir.r5, ir.r3).stg(ir.r2, ir.r4).stg(ir.r2, ir.r5, bdim).exit()
    a.label("plain").bar().bar().exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, 3, bdim, 0, ())], np.full(2 * bdim, -1, np.int32),
                      name="rbar_mixed")


def deadlock_then_skip():
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, 5).brnz(ir.r3, "x").bar_count(ir.r4, ir.r3)
    a.stg(ir.r2, ir.r4).label("x").exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 64, 0, ()), ir.Launch(0, 1, 64, 0, ())],
                      np.full(64, -1, np.int32), name="rbar_deadlock")


def interval_split(sync=True):
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).add(ir.r3, ir.r2, 1).and_(ir.r3, ir.r3, 63).sts(ir.r2, ir.r2)
    if sync:
        a.bar_or(ir.r4, ir.r2)
    a.lds(ir.r5, ir.r3).stg(ir.r2, ir.r5).exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 64, 64, ())], np.zeros(64, np.int32),
                      name=f"rbar_split_{sync}")


def loop_until_all_done(bdim=96):
    """Each thread counts down from tid % 7; the block loops until __syncthreads_and says
    every counter reached 0, counting the iterations with __syncthreads_count."""
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).rem(ir.r3, ir.r2, 7).mov(ir.r8, 0)
    a.label("top").seq(ir.r4, ir.r3, 0).bar_and(ir.r5, ir.r4).brnz(ir.r5, "done")
    a.slt(ir.r6, ir.RZ, ir.r3).sub(ir.r3, ir.r3, ir.r6).bar_count(ir.r7, ir.r6).add(ir.r8, ir.r8, ir.r7)
    a.bra("top")
    a.label("done").stg(ir.r2, ir.r8).exit()
    return ir.Program(a.assemble(), [0], [ir.Launch(0, 2, bdim, 0, ())], np.zeros(bdim, np.int32),
                      name="rbar_loop")


def all_programs():
    out = [predicate_values(b, l) for b, l in ((100, 37), (100, 100), (100, 0), (33, 32), (1, 1),
                                               (1024, 1000), (64, 63))]
    out += [odd_count(b, seed=b) for b in (33, 100, 512)]
    out += [mixed_with_plain(), deadlock_then_skip(), interval_split(True), interval_split(False),
            loop_until_all_done()]
    return out
