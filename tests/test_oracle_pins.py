"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* values the paper prints for its Figure 1 program and the two cudak variants (Sec. 3.2),
  kept as a text fixture in tests/golden/fig1_sum.txt;
* C99 integer semantics written out by hand;
* exhaustive interleaving enumeration on tiny programs (tests/brute_force.py);
* closed forms (numpy) for the workload families, and the race sets that the planted
  bugs must produce, derived from the race definition of Sec. 3.1;
* invariants: schedule independence of race-free programs, host-thread parallelism.
"""
import numpy as np
import pytest

import oracle
from conftest import golden
from paper_1211_6193_gb300.workloads import families, fig1, ir, stencil2d, tiny
from brute_force import enumerate_outcomes, races as bf_races


def reports_of(res, kind=None):
    out = res.report_tuples()
    return [r for r in out if kind is None or r[0] == kind]


def find_pc(code, pred):
    ops, ds, as_, bs, imms = ir.decode_fields(code)
    return [pc for pc in range(len(code)) if pred(int(ops[pc]) & 0x7F, int(ds[pc]), int(as_[pc]),
                                                    int(bs[pc]), int(imms[pc]))]


# ------------------------------------------------------------------ Figure 1 (Sec. 3.2)
G = golden("fig1_sum.txt")


def test_fig1_input_matches_paper():
    assert list(fig1.host_input()) == G["INPUT"]


def test_fig1_output_767():
    r = oracle.run([fig1.program()])
    out = r.arenas[0][fig1.OUT_OFF:]
    assert out[0] == G["OUTPUT"][0]
    assert list(out) == G["FINAL_OUT"]
    assert reports_of(r) == [] and r.status[0] == 0
    assert list(r.arenas[0][:fig1.N]) == G["INPUT"]          # input untouched


def test_fig1_race_variant():
    p = fig1.program(race=True)
    r = oracle.run([p])
    assert r.arenas[0][fig1.OUT_OFF] == G["RACE_VARIANT_OUTPUT"][0]
    assert r.status[0] == 0
    # line 12 load of shared[tid] and the line-17 load shared[i] (the loop body)
    pc_line12 = find_pc(p.code, lambda op, d, a, b, imm: op == ir.LDS and a == 2)[0]
    pc_line17 = find_pc(p.code, lambda op, d, a, b, imm: op == ir.LDS and a == 13)[0]
    # hand trace: in epoch 1 threads 1..3 write shared[1..3] (line 12) and thread 0 reads
    # them in the loop of line 17 with no barrier in between; everything else is same-thread
    exp = [(oracle.RACE, 0, 0, blk, 1, x, (0 << 16) | x,
            (oracle.CLS_WR << 24) | (pc_line12 << 12) | pc_line17)
           for blk in (0, 1) for x in (1, 2, 3)]
    assert reports_of(r) == exp
    # the paper locates the race at source line 17: the highest pc of every record is there
    assert all((rec[7] & 0xFFF) == pc_line17 for rec in exp) and G["RACE_VARIANT_LINE"] == [17]


def test_fig1_deadlock_variant():
    p = fig1.program(deadlock=True)
    r = oracle.run([p])
    assert G["DEADLOCK_VARIANT_REPORTS_DEADLOCK"] == [1]
    assert r.status[0] & oracle.ST_DEADLOCK
    bars = find_pc(p.code, lambda op, *_: op == ir.BAR)
    inner, line14 = bars[1], bars[2]
    exp = []
    for blk in (0, 1):
        # all 9 threads wait, 4 at the inserted barrier and 5 at line 14: divergent barrier
        exp.append((oracle.DIVERGENCE, 0, 0, blk, 1, inner, line14, 9 << 16))
        # then 4 threads wait at line 14 while 5 have exited: deadlock
        exp.append((oracle.DEADLOCK, 0, 0, blk, 2, line14, line14, (4 << 16) | 5))
    assert reports_of(r) == exp
    assert list(r.arenas[0][fig1.OUT_OFF:]) == [0, 0]        # the second launch never ran


# ------------------------------------------------------------------ integer semantics
INT_MIN, INT_MAX = -(1 << 31), (1 << 31) - 1

ALU_CASES = [  # (op, x, y, expected) - C99 int rules written out by hand
    (ir.ADD, INT_MAX, 1, INT_MIN), (ir.SUB, INT_MIN, 1, INT_MAX), (ir.MUL, 65536, 65536, 0),
    (ir.MUL, 46341, 46341, -2147479015), (ir.MUL, -3, 7, -21),
    (ir.DIV, -7, 2, -3), (ir.DIV, 7, -2, -3), (ir.DIV, -7, -2, 3), (ir.DIV, INT_MIN, -1, INT_MIN),
    (ir.REM, -7, 2, -1), (ir.REM, 7, -2, 1), (ir.REM, INT_MIN, -1, 0), (ir.REM, -8, 4, 0),
    (ir.AND, -1, 0x0F0F, 0x0F0F), (ir.OR, 0x100, 0x011, 0x111), (ir.XOR, -1, 5, -6),
    (ir.SHL, 1, 33, 2), (ir.SHL, 1, 31, INT_MIN), (ir.SHL, 3, 0, 3),
    (ir.SHR, -8, 1, -4), (ir.SHR, -1, 31, -1), (ir.SHR, 8, 35, 1), (ir.SHR, INT_MIN, 31, -1),
    (ir.MIN, -5, 3, -5), (ir.MAX, -5, 3, 3), (ir.SLT, -1, 0, 1), (ir.SLT, 0, -1, 0),
    (ir.SLE, 4, 4, 1), (ir.SEQ, 9, 9, 1), (ir.SNE, 9, 9, 0), (ir.MOV, 0, -12345, -12345),
]


def test_alu_semantics_hand_values():
    a = ir.Asm()
    for i, (op, x, y, _) in enumerate(ALU_CASES):
        a.mov(ir.r4, x).mov(ir.r5, y).alu(op, ir.r6, ir.r4, ir.r5).stg(ir.r0, ir.r6, i)
    # immediate second operand gives the same result
    a.mov(ir.r4, -7).div(ir.r6, ir.r4, 2).stg(ir.r0, ir.r6, len(ALU_CASES))
    a.exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 1, 0, (0,))], np.zeros(len(ALU_CASES) + 1, np.int32))
    r = oracle.run([p])
    assert list(r.arenas[0][:-1]) == [c[3] for c in ALU_CASES]
    assert r.arenas[0][-1] == -3
    assert reports_of(r) == []


def test_div_by_zero_and_out_of_bounds_records():
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).mov(ir.r4, 5)
    pc_div = a.pc
    a.div(ir.r6, ir.r4, ir.RZ)                 # x / 0 -> 0, ERR_DIV0
    pc_rem = a.pc
    a.rem(ir.r7, ir.r4, 0)                     # x % 0 -> 0, ERR_DIV0
    a.add(ir.r8, ir.r2, -3)                    # tid - 3: negative for tids 0..2
    pc_lds = a.pc
    a.lds(ir.r9, ir.r8)                        # shared words -3..4: OOB for tids 0,1,2 and 7
    pc_ldg = a.pc
    a.ldg(ir.r10, ir.r2, 100)                  # global OOB for every thread
    pc_sts = a.pc
    a.sts(ir.r2, ir.r2, -3)                    # same words as the load, same threads
    a.bar()                                    # epoch 1 from here on
    pc_atoms = a.pc
    a.atoms(ir.r2, ir.r4, -4)                  # words -4..3: OOB for tids 0..3
    a.add(ir.r11, ir.r6, ir.r7).add(ir.r11, ir.r11, ir.r9).add(ir.r11, ir.r11, ir.r10)
    a.stg(ir.r2, ir.r11)                       # word tid = 0 (every operand was suppressed to 0)
    pc_stg = a.pc
    a.stg(ir.r2, ir.r2, 1)                     # word tid + 1 = tid: OOB only for tid 7 (word 8)
    a.exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 8, 4, (0,))], np.full(8, 77, np.int32))
    r = oracle.run([p])
    # the later store of thread t to word t+1 overwrites thread t+1's earlier zero
    assert list(r.arenas[0]) == [0, 0, 1, 2, 3, 4, 5, 6]
    # (a = pc, b = lowest tid, c = number of thread executions) per erroneous instruction
    E = lambda kind, ep, pc, t, c: (kind, 0, 0, 0, ep, pc, t, c)
    assert reports_of(r) == sorted([
        E(oracle.ERR_OOB_SHARED, 0, pc_lds, 0, 4), E(oracle.ERR_OOB_SHARED, 0, pc_sts, 0, 4),
        E(oracle.ERR_OOB_GLOBAL, 0, pc_ldg, 0, 8), E(oracle.ERR_DIV0, 0, pc_div, 0, 8),
        E(oracle.ERR_DIV0, 0, pc_rem, 0, 8), E(oracle.ERR_OOB_SHARED, 1, pc_atoms, 0, 4),
        E(oracle.ERR_OOB_GLOBAL, 1, pc_stg, 7, 1),
    ], key=lambda t: (t[4], t[0], t[5]))


def test_special_registers():
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).s2r(ir.r3, ir.BID).s2r(ir.r4, ir.BDIM).s2r(ir.r5, ir.GDIM).s2r(ir.r6, ir.WARPSIZE)
    a.mul(ir.r7, ir.r3, ir.r4).add(ir.r7, ir.r7, ir.r2).mul(ir.r7, ir.r7, 5)
    for k, reg in enumerate((ir.r2, ir.r3, ir.r4, ir.r5, ir.r6)):
        a.stg(ir.r7, reg, k)
    a.exit()
    g, b = 3, 40
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, g, b, 0, ())], np.zeros(g * b * 5, np.int32))
    r = oracle.run([p])
    got = r.arenas[0].reshape(g, b, 5)
    for bi in range(g):
        for t in range(b):
            assert list(got[bi, t]) == [t, bi, b, g, 32]


def test_falling_off_the_end_is_exit_and_step_limit():
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).stg(ir.r2, ir.r2)   # no EXIT: running past the end exits
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 4, 0, ())], np.zeros(4, np.int32))
    r = oracle.run([p])
    assert list(r.arenas[0]) == [0, 1, 2, 3] and r.status[0] == 0
    # an endless loop stops at the round budget with a STEP_LIMIT record
    a = ir.Asm()
    a.label("top").add(ir.r3, ir.r3, 1).bra("top")
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 33, 0, ())], np.zeros(1, np.int32))
    r = oracle.run([p], round_budget=1000)
    assert r.status[0] & oracle.ST_STEP_LIMIT
    assert reports_of(r) == [(oracle.STEP_LIMIT, 0, 0, 0, 0, 1000, 33, 0)]


# ------------------------------------------------------------------ round-lockstep reading
def test_lockstep_round_rules_hand_derived():
    """The canonical schedule, derived by hand for a 64-thread block (two warps).

    Both warps run pcs 0-3 in rounds 0-3; at round 3 warp 1 branches, so in round 4
    warp 0 executes pc 4 (stores) while warp 1 executes pc 7 (a load of the same word).
    """
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 5).brnz(ir.r3, "w1")          # pcs 0-3
    a.sts(ir.RZ, ir.r4).sts(ir.RZ, ir.r4, 1).bra("join")                               # pcs 4-6 (warp 0)
    a.label("w1").lds(ir.r5, ir.RZ).mov(ir.r6, 1).atoms(ir.RZ, ir.r6, 1).lds(ir.r7, ir.RZ)  # pcs 7-10
    a.stg(ir.r2, ir.r5).stg(ir.r2, ir.r7, 64)
    a.label("join").sts(ir.RZ, ir.r2, 2)                  # every thread stores its tid to sh[2]
    # min-pc order inside warp 0: lanes >= 16 fall through to the lower pc and load sh[3]
    # before lanes < 16 (branch to a higher pc) store 7 there
    # (three filler instructions first: with 16-wide warps the store would land before the load)
    a.slt(ir.r8, ir.r2, 16).brnz(ir.r8, "hi").mov(ir.r9, 0).mov(ir.r9, 0).mov(ir.r9, 0)
    a.lds(ir.r9, ir.RZ, 3).stg(ir.r2, ir.r9, 128).bra("end")
    a.label("hi").mov(ir.r9, 7).sts(ir.RZ, ir.r9, 3)
    a.label("end").bar()
    a.brnz(ir.r2, "out").lds(ir.r10, ir.RZ).stg(ir.RZ, ir.r10, 192).lds(ir.r10, ir.RZ, 1)
    a.stg(ir.RZ, ir.r10, 193).lds(ir.r10, ir.RZ, 2).stg(ir.RZ, ir.r10, 194).lds(ir.r10, ir.RZ, 3)
    a.stg(ir.RZ, ir.r10, 195).label("out").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 4, ())], np.full(196, -1, np.int32))
    r = oracle.run([p])
    A = r.arenas[0]
    # round 4: warp 1's load of sh[0] sees the pre-round value 0, not warp 0's store of 5
    assert list(A[32:64]) == [0] * 32
    # round 5 vs 6: warp 0 stores sh[1] = 5 in round 5 while warp 1 adds 32 x 1 in round 6;
    # its later load (round 7) of sh[0] sees warp 0's round-4 store
    assert list(A[64 + 32:128]) == [5] * 32
    assert A[193] == 5 + 32
    # sh[2]: 64 stores in one round (warp 1 reaches the join later) -> last writer wins;
    # warp 1 (tids 32..63) stores after warp 0, highest tid 63 last
    assert A[194] == 63
    # lanes 16..31 of warp 0 load sh[3] before lanes 0..15 store 7 to it
    assert list(A[128 + 16:128 + 32]) == [0] * 16
    assert A[195] == 7 and A[192] == 5


def test_same_round_store_then_atomic_order():
    """Stores of a round apply before its atomic adds (warp 0 stores 10 while warp 1's
    32 lanes add 1 in the same round): 10 + 32."""
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 10).mov(ir.r5, 1).brnz(ir.r3, "w1")
    a.sts(ir.RZ, ir.r4).bra("j")
    a.label("w1").atoms(ir.RZ, ir.r5).label("j").bar()
    a.brnz(ir.r2, "x").lds(ir.r6, ir.RZ).stg(ir.RZ, ir.r6).label("x").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 1, ())], np.zeros(1, np.int32))
    r = oracle.run([p])
    assert r.arenas[0][0] == 42
    rec = reports_of(r, oracle.RACE)
    # warp 0's 32 lanes all store (write-write, smallest pair (0, 1)) and warp 1 adds
    assert len(rec) == 1 and rec[0][6] == (0 << 16) | 1
    assert (rec[0][7] >> 24) == oracle.CLS_WW | oracle.CLS_WA


# ------------------------------------------------------------------ __syncthreads_and/_or/_count
def _rbar_values(bdim, pred_limit):
    """Every thread: pred = tid < pred_limit; COUNT, AND, OR of it; stores the three results."""
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, pred_limit)
    a.bar_count(ir.r4, ir.r3).bar_and(ir.r5, ir.r3).bar_or(ir.r6, ir.r3)
    a.mul(ir.r7, ir.r2, 3).stg(ir.r7, ir.r4).stg(ir.r7, ir.r5, 1).stg(ir.r7, ir.r6, 2).exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, bdim, 0, ())], np.full(3 * bdim, -1, np.int32))
    r = oracle.run([p])
    return r, r.arenas[0].reshape(bdim, 3)


@pytest.mark.parametrize("bdim,limit", [(100, 37), (100, 100), (100, 0), (33, 32), (1, 1), (1024, 1000)])
def test_reducing_barriers_hand_values(bdim, limit):
    r, got = _rbar_values(bdim, limit)
    n = min(bdim, limit)
    assert reports_of(r) == [] and r.status[0] == 0
    assert (got[:, 0] == n).all()                     # __syncthreads_count
    assert (got[:, 1] == int(n == bdim)).all()        # __syncthreads_and
    assert (got[:, 2] == int(n > 0)).all()            # __syncthreads_or


@pytest.mark.parametrize("bdim", [33, 100, 512])
def test_reducing_barrier_count_closed_form(bdim):
    """Per block, the number of odd inputs, counted by __syncthreads_count and stored by
    thread 0: numpy's count of the same values."""
    grid = 5
    rng = np.random.default_rng(bdim)
    vals = rng.integers(-1000, 1000, grid * bdim, dtype=np.int32)
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).s2r(ir.r3, ir.BID).mul(ir.r4, ir.r3, bdim).add(ir.r4, ir.r4, ir.r2)
    a.ldg(ir.r5, ir.r4).and_(ir.r6, ir.r5, 1).bar_count(ir.r7, ir.r6)
    a.brnz(ir.r2, "x").stg(ir.r3, ir.r7, grid * bdim).label("x").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, grid, bdim, 0, ())],
                   np.concatenate([vals, np.zeros(grid, np.int32)]))
    r = oracle.run([p])
    want = (vals.reshape(grid, bdim) & 1).sum(axis=1)
    assert list(r.arenas[0][grid * bdim:]) == list(want)


def test_reducing_barrier_mixed_with_plain_barrier():
    """Threads 0..39 reach BARAND/BARPOPC with a true predicate, the others a plain BAR:
    DIVERGENCE is reported, and the plain waiters count as false."""
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, 40).brz(ir.r3, "plain")
    a.bar_count(ir.r4, ir.r3).bar_and(ir.r5, ir.r3).stg(ir.r2, ir.r4).stg(ir.r2, ir.r5, 100).exit()
    a.label("plain").bar().bar().exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 100, 0, ())], np.full(200, -1, np.int32))
    r = oracle.run([p])
    A = r.arenas[0]
    assert list(A[:40]) == [40] * 40 and list(A[40:100]) == [-1] * 60
    assert list(A[100:140]) == [0] * 40
    pc_cnt = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.BARPOPC)[0]
    pc_and = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.BARAND)[0]
    pcs_bar = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.BAR)
    assert reports_of(r) == [(oracle.DIVERGENCE, 0, 0, 0, 0, pc_cnt, pcs_bar[0], 100 << 16),
                             (oracle.DIVERGENCE, 0, 0, 0, 1, pc_and, pcs_bar[1], 100 << 16)]


def test_reducing_barriers_in_a_loop_closed_form():
    """Threads count down from tid % 7 until __syncthreads_and sees every counter at 0,
    summing __syncthreads_count of the threads still counting: the total number of
    decrements, sum(tid % 7), in every thread."""
    from rbar_programs import loop_until_all_done
    r = oracle.run([loop_until_all_done(96)])
    assert reports_of(r) == [] and list(r.arenas[0]) == [sum(t % 7 for t in range(96))] * 96


def test_reducing_barrier_deadlock_and_race_interval():
    """A reducing barrier is a barrier: it ends the race interval; with exited threads it
    deadlocks like BAR and the block stops before any result is used."""
    def prog(sync):
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID).add(ir.r3, ir.r2, 1).and_(ir.r3, ir.r3, 63).sts(ir.r2, ir.r2)
        if sync:
            a.bar_or(ir.r4, ir.r2)
        a.lds(ir.r5, ir.r3).stg(ir.r2, ir.r5).exit()
        return ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 64, ())], np.zeros(64, np.int32))
    assert reports_of(oracle.run([prog(True)])) == []
    assert len(reports_of(oracle.run([prog(False)]), oracle.RACE)) == 64
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).slt(ir.r3, ir.r2, 5).brnz(ir.r3, "x").bar_count(ir.r4, ir.r3)
    a.stg(ir.r2, ir.r4).label("x").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 0, ()), ir.Launch(0, 1, 64, 0, ())],
                   np.full(64, -1, np.int32))
    r = oracle.run([p])
    pc = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.BARPOPC)[0]
    assert reports_of(r) == [(oracle.DEADLOCK, 0, 0, 0, 0, pc, pc, (59 << 16) | 5)]
    assert r.status[0] & oracle.ST_DEADLOCK and list(r.arenas[0]) == [-1] * 64


# ------------------------------------------------------------------ uninitialised shared reads
def test_uninitialised_reads_hand_values():
    """Warp 0 stores sh[tid]; after the barrier every thread loads sh[tid]: the 32 loads of
    warp 1 read words no thread wrote (one record at the load's pc: min tid 32, count 32).
    The check is off unless asked for."""
    a = ir.Asm()
    a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).brnz(ir.r3, "skip").sts(ir.r2, ir.r2).label("skip").bar()
    a.lds(ir.r4, ir.r2).stg(ir.r2, ir.r4).exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 2, 64, 64, ())], np.zeros(64, np.int32))
    pc = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.LDS)[0]
    r = oracle.run([p], check_uninit=True)
    assert reports_of(r) == [(oracle.ERR_UNINIT_SHARED, 0, 0, blk, 1, pc, 32, 32) for blk in (0, 1)]
    assert reports_of(oracle.run([p])) == []


def test_uninitialised_reads_follow_the_round_rule():
    """A load sees the writes of earlier rounds only: warp 1 loading sh[0] in the round
    where warp 0 stores it reads an unwritten word; a round later it does not.  Atomic
    adds count as writes; a store of a later interval does not help an earlier load."""
    def prog(delay):
        a = ir.Asm()
        a.s2r(ir.r2, ir.TID).shr(ir.r3, ir.r2, 5).mov(ir.r4, 5).brnz(ir.r3, "w1")
        a.sts(ir.RZ, ir.r4).bra("end")
        a.label("w1")
        for _ in range(delay):
            a.mov(ir.r9, 0)
        a.lds(ir.r5, ir.RZ).label("end").exit()
        return ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 64, 1, ())], np.zeros(1, np.int32))
    r0 = reports_of(oracle.run([prog(0)], check_uninit=True))
    assert [t[0] for t in r0] == [oracle.RACE, oracle.ERR_UNINIT_SHARED] and r0[1][6:] == (32, 32)
    assert [t[0] for t in reports_of(oracle.run([prog(1)], check_uninit=True))] == [oracle.RACE]
    a = ir.Asm()                        # ATOMS initialises; a later-interval store does not count
    a.s2r(ir.r2, ir.TID).mov(ir.r3, 1).atoms(ir.RZ, ir.r3).bar().lds(ir.r4, ir.RZ).lds(ir.r5, ir.RZ, 1)
    a.bar().brnz(ir.r2, "x").sts(ir.RZ, ir.r3, 1).label("x").exit()
    p = ir.Program(a.assemble(), [0], [ir.Launch(0, 1, 40, 2, ())], np.zeros(1, np.int32))
    pc = find_pc(p.code, lambda op, d, a_, b, imm: op == ir.LDS)[1]
    assert reports_of(oracle.run([p], check_uninit=True)) == [(oracle.ERR_UNINIT_SHARED, 0, 0, 0, 1, pc, 0, 40)]


def test_uninitialised_reads_only_in_planted_bugs():
    """No bug-free generated program (all families) reads a shared word it did not write;
    every report comes from a program with a planted off-by-one or missing barrier."""
    progs = families.batch(n_programs=96, seed=8, max_grid=3, bug_rate=0.4)
    progs += [families.reduction_plain(n_blocks=3), stencil2d.program(log2w=6, steps=2, buggy_launch=None)]
    r = oracle.run(progs, check_uninit=True)
    hit = {t[1] for t in reports_of(r, oracle.ERR_UNINIT_SHARED)}
    assert hit and all(progs[i].meta.get("bug") in ("off_by_one", "missing_barrier") for i in hit)
    # and the other reports are exactly those of the run without the check
    assert [t for t in r.report_tuples() if t[0] != oracle.ERR_UNINIT_SHARED] == oracle.run(progs).report_tuples()


# ------------------------------------------------------------------ exhaustive interleavings
@pytest.mark.parametrize("nthreads,nsteps,count,nwords,bar_rate",
                         [(2, 6, 40, 3, 0.25), (3, 4, 40, 3, 0.25), (3, 6, 16, 8, 0.6)])
def test_brute_force_interleavings(nthreads, nsteps, count, nwords, bar_rate):
    progs = tiny.tiny_batch(1000 + 10 * nthreads + nsteps, count, nthreads=nthreads, nsteps=nsteps,
                            nwords=nwords, bar_rate=bar_rate)
    res = oracle.run(progs)
    rep = res.report_tuples()
    n_racy = 0
    for i, p in enumerate(progs):
        evs, outcomes, positions = enumerate_outcomes(p)
        expect = bf_races(evs, positions)
        got = {(r[4], r[5]): (r[6] >> 16, r[6] & 0xFFFF, r[7] >> 24, (r[7] >> 12) & 0xFFF, r[7] & 0xFFF)
               for r in rep if r[1] == i and r[0] == oracle.RACE}
        assert got == expect, f"program {i}"
        assert all(r[0] == oracle.RACE for r in rep if r[1] == i)
        canon = tuple(int(x) for x in res.arenas[i])
        assert canon in outcomes, f"program {i}: canonical image is not an interleaving outcome"
        if not expect:
            assert outcomes == {canon}, f"program {i}: race-free yet several outcomes"
        else:
            n_racy += 1
    assert 0 < n_racy < count          # the sample exercises both cases


def test_commutation_table_is_the_race_rule():
    from brute_force import commute
    # read-read and atomic-atomic commute; every pair involving a write, and atomic-read, do not
    assert commute("R", "R") and commute("A", "A")
    assert not any(commute(x, y) for x, y in [("W", "W"), ("W", "R"), ("R", "W"), ("W", "A"),
                                              ("A", "W"), ("A", "R"), ("R", "A")])


# ------------------------------------------------------------------ closed forms
def _block_sums(values, bdim):
    return values.astype(np.int64).reshape(-1, bdim).sum(axis=1).astype(np.int32)


def test_plain_reduction_closed_form_and_race_set():
    nb, bdim = 6, 1024
    p = families.reduction_plain(n_blocks=nb, bdim=bdim, seed=1, omit_level=3)
    r = oracle.run([p])
    n = nb * bdim
    assert np.array_equal(r.arenas[0][n:], _block_sums(p.global_init[:n], bdim))
    assert r.status[0] == 0
    # level 3 (stride 64) lost its barrier, so level 4 (stride 32, tid < 32) reads
    # sh[32..63] in the same interval in which threads 32..63 wrote them
    lds = find_pc(p.code, lambda op, d, a, b, imm: op == ir.LDS and a == 2 and imm == 0)
    pc_l3 = lds[3]
    pc_l4_hi = find_pc(p.code, lambda op, d, a, b, imm: op == ir.LDS and a == 2 and imm == 32)[0]
    exp = [(oracle.RACE, 0, 0, blk, 4, 32 + j, (j << 16) | (32 + j),
            (oracle.CLS_WR << 24) | (pc_l3 << 12) | pc_l4_hi) for blk in range(nb) for j in range(32)]
    assert reports_of(r) == exp


@pytest.mark.parametrize("bdim", [32, 96, 160, 512, 1000 // 32 * 32])
def test_reduction_any_blockdim(bdim):
    spec = families.FamilySpec("reduction", 5, bdim, bdim, 20, None, 0)
    p = families.build_family(spec, seed=bdim)
    r = oracle.run([p])
    n = 5 * bdim
    assert np.array_equal(r.arenas[0][n:], _block_sums(p.global_init[:n], bdim))
    assert reports_of(r) == []


@pytest.mark.parametrize("bdim,s_idx", [(256, 2), (128, 0), (1024, 5)])
def test_reduction_planted_missing_barrier(bdim, s_idx):
    spec = families.FamilySpec("reduction", 2, bdim, bdim, 20, "missing_barrier", s_idx)
    p = families.build_family(spec, seed=7)
    r = oracle.run([p])
    s_next = bdim >> (s_idx + 2)               # stride of the level after the missing barrier
    races = reports_of(r, oracle.RACE)
    for blk in range(2):
        got = sorted(rec[5] for rec in races if rec[3] == blk)
        assert got == list(range(s_next, 2 * s_next))
        assert all(rec[6] == (((rec[5] - s_next) << 16) | rec[5]) for rec in races if rec[3] == blk)
    n = 2 * bdim
    assert np.array_equal(r.arenas[0][n:], _block_sums(p.global_init[:n], bdim))


@pytest.mark.parametrize("bdim,level", [(256, 1), (64, 0), (512, 3)])
def test_reduction_planted_off_by_one(bdim, level):
    spec = families.FamilySpec("reduction", 1, bdim, bdim + 1, 20, "off_by_one", level)
    p = families.build_family(spec, seed=11)
    r = oracle.run([p])
    s = bdim >> (level + 1)
    lvl_lds = [pc for pc in find_pc(p.code, lambda op, d, a, b, imm: op == ir.LDS and a == 2 and imm == 0)][level]
    lvl_sts = find_pc(p.code, lambda op, d, a, b, imm: op == ir.STS and a == 2 and imm == 0)[level + 1]
    # thread s (let in by tid <= s) reads sh[s], sh[2s] and writes sh[s]; thread 0 reads
    # sh[0 + s]: one write-read race on word s, accesses spanning the level's first load
    # and its store
    assert reports_of(r) == [
        (oracle.RACE, 0, 0, 0, level + 1, s, (0 << 16) | s, (oracle.CLS_WR << 24) | (lvl_lds << 12) | lvl_sts)]


def test_reduction_planted_divergent_barrier():
    bdim, level = 256, 2
    spec = families.FamilySpec("reduction", 1, bdim, bdim, 20, "divergent_barrier", level)
    p = families.build_family(spec, seed=5)
    r = oracle.run([p])
    bars = find_pc(p.code, lambda op, *_: op == ir.BAR)
    inner, level_end = bars[1 + level], bars[2 + level]
    recs = reports_of(r)
    s = bdim >> (level + 1)
    assert recs[0] == (oracle.DIVERGENCE, 0, 0, 0, level + 1, inner, level_end, bdim << 16)
    assert recs[-1][0] == oracle.DEADLOCK and r.status[0] & oracle.ST_DEADLOCK
    assert (recs[-1][7] & 0xFFFF) == bdim - s       # the threads outside the branch exit


@pytest.mark.parametrize("bdim,radius", [(32, 1), (64, 8), (96, 3)])
def test_stencil1d_closed_form(bdim, radius):
    g = 4
    spec = families.FamilySpec("stencil1d", g, bdim, bdim + 2 * radius + 5, 20, None, 0, radius=radius)
    p = families.build_family(spec, seed=3 * bdim + radius)
    r = oracle.run([p])
    n = g * bdim
    x = np.concatenate([np.zeros(radius, np.int64), p.global_init[:n].astype(np.int64), np.zeros(radius, np.int64)])
    exp = sum(x[j:j + n] for j in range(2 * radius + 1)).astype(np.int32)
    assert np.array_equal(r.arenas[0][n:], exp)
    assert reports_of(r) == []


def test_stencil1d_missing_barrier_race_set():
    bdim, radius, g = 64, 2, 2
    spec = families.FamilySpec("stencil1d", g, bdim, bdim + 2 * radius, 20, "missing_barrier", 0, radius=radius)
    p = families.build_family(spec, seed=9)
    r = oracle.run([p])
    # cell c is written by one thread (centre: c - r; left halo: c < r by thread c; right
    # halo: c >= bdim + r by thread c - 2r) and read by threads max(0, c-2r)..min(c, bdim-1);
    # it races iff some reader is not its writer
    exp = []
    for c in range(bdim + 2 * radius):
        w = c if c < radius else (c - 2 * radius if c >= bdim + radius else c - radius)
        readers = set(range(max(0, c - 2 * radius), min(c, bdim - 1) + 1))
        if readers - {w}:
            exp.append(c)
    assert 0 not in exp and bdim + 2 * radius - 1 not in exp
    for blk in range(g):
        got = sorted(rec[5] for rec in reports_of(r, oracle.RACE) if rec[3] == blk)
        assert got == exp


@pytest.mark.parametrize("bdim", [32, 96, 320, 1024])
def test_transpose_closed_form(bdim):
    g = 3
    spec = families.FamilySpec("transpose", g, bdim, 32 * 33, 20, None, 0)
    p = families.build_family(spec, seed=bdim)
    r = oracle.run([p])
    n = g * 1024
    exp = p.global_init[:n].reshape(g, 32, 32).transpose(0, 2, 1).reshape(-1)
    assert np.array_equal(r.arenas[0][n:], exp)
    assert reports_of(r) == []


@pytest.mark.parametrize("bdim,elems", [(32, 3), (256, 1), (384, 2)])
def test_histogram_closed_form(bdim, elems):
    g = 3
    spec = families.FamilySpec("histogram", g, bdim, 300, 20, None, 0, elems=elems)
    p = families.build_family(spec, seed=bdim + elems)
    r = oracle.run([p])
    n = g * bdim * elems
    vals = (p.global_init[:n].astype(np.int64) & 255).reshape(g, -1)
    exp = np.stack([np.bincount(v, minlength=256) for v in vals]).reshape(-1).astype(np.int32)
    assert np.array_equal(r.arenas[0][n:], exp)
    assert reports_of(r) == []


def test_histogram_missing_barrier_after_zeroing():
    # zeroing stores and atomic adds share one interval: write-atomic races on bins
    bdim, elems = 64, 2
    spec = families.FamilySpec("histogram", 1, bdim, 256, 20, "missing_barrier", 0, elems=elems)
    p = families.build_family(spec, seed=21)
    r = oracle.run([p])
    races = reports_of(r, oracle.RACE)
    assert races and all((rec[7] >> 24) & oracle.CLS_WA for rec in races)
    vals = p.global_init[:bdim * elems].astype(np.int64) & 255
    touched = set(int(v) for v in vals)
    # a bin races iff some thread other than its zeroing thread adds to it
    owner = {b: b % bdim for b in range(256)}
    adders = {}
    for t in range(bdim):
        for e in range(elems):
            adders.setdefault(int(vals[t * elems + e]), set()).add(t)
    exp = sorted(b for b in touched if adders[b] - {owner[b]})
    assert sorted(rec[5] for rec in races) == exp


def _stencil2d_numpy(grid, steps):
    g = grid.astype(np.int64)
    for _ in range(steps):
        p = np.pad(g, 1)
        s = p[1:-1, 1:-1] + p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:]
        g = np.sign(s) * (np.abs(s) // 5)               # C division truncates toward zero
    return g.astype(np.int32)


def test_stencil2d_closed_form_and_race_set():
    log2w, steps, bug = 6, 4, 2
    p = stencil2d.program(log2w=log2w, steps=steps, buggy_launch=bug, seed=4)
    W = 1 << log2w
    r = oracle.run([p])
    n = W * W
    final = r.arenas[0][:n] if steps % 2 == 0 else r.arenas[0][n:]
    exp = _stencil2d_numpy(p.global_init[:n].reshape(W, W), steps).reshape(-1)
    assert np.array_equal(final, exp)
    # launch `bug` lost its staging barrier: every centre cell of the 34x34 tile is
    # written by its owner and read by a neighbour in the same interval; halo cells
    # are written and read by the same edge thread, so they never race
    code = p.code[p.kernel_entry[1]:]
    base = p.kernel_entry[1]
    sts_c = base + find_pc(code, lambda op, d, a, b, imm: op == ir.STS and imm == 0)[0]
    lds = {imm: base + pc for pc in find_pc(code, lambda op, *_: op == ir.LDS)
           for imm in [int(code["imm"][pc])]}
    races = reports_of(r, oracle.RACE)
    nblocks = (W // 32) ** 2
    assert len(races) == nblocks * 1024
    assert all(rec[2] == bug and rec[4] == 0 for rec in races)
    for rec in races[:1024]:
        cell = rec[5]
        ty, tx = cell // 34 - 1, cell % 34 - 1
        tid = ty * 32 + tx
        nbrs = [t for t, ok in [(tid - 32, ty > 0), (tid - 1, tx > 0), (tid + 1, tx < 31), (tid + 32, ty < 31)] if ok]
        t1 = min(min(tid, t) for t in nbrs)
        t2 = min(max(tid, t) for t in nbrs if min(tid, t) == t1)
        pchi = lds[34] if ty > 0 else lds[-34]
        assert rec[6] == (t1 << 16) | t2
        assert rec[7] == (oracle.CLS_WR << 24) | (sts_c << 12) | pchi


# ------------------------------------------------------------------ invariants
def _small_batch(seed, n, bug_rate):
    return families.batch(n_programs=n, seed=seed, max_grid=3, bug_rate=bug_rate)


def test_race_free_programs_are_schedule_independent():
    progs = _small_batch(31, 24, 0.0)
    a = oracle.run(progs)
    b = oracle.run(progs, schedule="sequential")
    for i in range(len(progs)):
        assert np.array_equal(a.arenas[i], b.arenas[i])
    assert a.report_tuples() == b.report_tuples() == []


def test_parallel_blocks_match_serial_and_no_interblock_conflicts():
    progs = _small_batch(32, 24, 0.5) + [stencil2d.program(log2w=6, steps=2, buggy_launch=1)]
    a = oracle.run(progs, check_interblock=True)
    b = oracle.run(progs, nthreads=4)
    assert a.interblock_conflicts == 0
    assert a.report_tuples() == b.report_tuples()
    assert all(np.array_equal(x, y) for x, y in zip(a.arenas, b.arenas))
    assert np.array_equal(a.status, b.status)


def test_opcode_numbers_agree_with_ir_module():
    import re, os
    hdr = open(os.path.join(os.path.dirname(oracle.__file__), "simt_oracle.h")).read()
    body = re.search(r"enum \{\s*ORC_MOV = 1,(.*?)\};", hdr, re.S).group(1)
    names = ["MOV"] + [n.strip()[4:] for n in body.replace("\n", " ").split(",") if n.strip()]
    for i, nm in enumerate(names, start=1):
        assert getattr(ir, nm) == i, nm


# ---------------------------------------------------------------- streams and events
def test_streams_fork_join_hand_values():
    """Sec. 3, streams and events: a deadlock stops its own stream and what waits on it, not
    the other streams.  Expected arenas are derived by hand in tests/stream_programs.py."""
    import stream_programs as sp
    for streams in (True, False):
        res = oracle.run([sp.fork_join(streams)], check_streams=True)
        assert np.array_equal(res.arenas[0], sp.fork_join_expected(streams)), res.arenas[0]
        assert list(res.status) == [oracle.ST_DEADLOCK]
        # the one report: launch 0's block 0 deadlocks (thread 0 exited, three wait at pc 3)
        assert [(r[0], r[2], r[3]) for r in res.report_tuples()] == [(oracle.DEADLOCK, 0, 0)]
        assert res.stream_conflicts == 0


def test_stream_conflict_diagnostic():
    """Launches no stream order or event wait orders must not share a written global word
    (the result would depend on timing); the diagnostic counts such words."""
    import stream_programs as sp
    assert oracle.run([sp.conflicting("ww")], check_streams=True).stream_conflicts == 4
    assert oracle.run([sp.conflicting("rw")], check_streams=True).stream_conflicts == 4
    assert oracle.run([sp.conflicting("ordered")], check_streams=True).stream_conflicts == 0
    # every generated workload is one stream, hence conflict-free by construction
    assert oracle.run(families.batch(n_programs=12, seed=3, max_grid=4), check_streams=True).stream_conflicts == 0


def test_stream_waits_must_name_an_earlier_launch():
    import stream_programs as sp
    p = sp.fork_join(True)
    p.launches[2] = ir.Launch(0, 1, 4, 0, (4, 20), stream=0, wait=5)
    with pytest.raises(ValueError):
        oracle.run([p])


def _stream_model(p):
    """The three kernels of tests/stream_programs.py executed directly: launches in index
    order; a launch whose stream predecessor or awaited launch stopped or was skipped is
    skipped; STALL stops its launch (deadlock)."""
    import stream_programs as sp
    arena, dead, status = p.global_init.astype(np.int64).copy(), set(), 0
    for l, L in enumerate(p.launches):
        prev = next((k for k in range(l - 1, -1, -1) if p.launches[k].stream == L.stream), None)
        if (prev is not None and prev in dead) or (L.wait >= 0 and L.wait in dead):
            dead.add(l)
            continue
        if L.kernel == sp.STALL:
            dead.add(l)
            status = oracle.ST_DEADLOCK
        elif L.kernel == sp.WRITE:
            arena[L.params[0]:L.params[0] + 4] = L.params[1] + np.arange(4)
        else:
            arena[L.params[1]:L.params[1] + 4] = arena[L.params[0]:L.params[0] + 4] + 1
    return arena.astype(np.int32), status


def test_streams_on_random_dependency_graphs_match_a_direct_model():
    import stream_programs as sp
    progs = sp.random_programs(7, 60)
    res = oracle.run(progs, check_streams=True, check_interblock=True)
    assert res.stream_conflicts == 0 and res.interblock_conflicts == 0
    for i, p in enumerate(progs):
        want, st = _stream_model(p)
        assert np.array_equal(res.arenas[i], want), p.name
        assert int(res.status[i]) == st, p.name
    assert 10 < sum(int(s) for s in res.status) < 50        # both outcomes well represented
