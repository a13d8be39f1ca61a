"""Multi-GPU execution (one process per GPU), two ways.

1. ``run_sharded``: a batch of independent programs.  Programs never communicate (Sec. 2:
   only the launches of one program share an arena), so ranks run disjoint subsets of the
   batch with no data-path collective; the only exchange is the final gather of reports,
   status and arenas to rank 0.  Programs are assigned by a longest-processing-time greedy on
   the access-log bytes the library reserves for them (the work of the check grows with them),
   deterministic in program order so every rank computes the same plan.

2. ``run_split``: one large program.  The blocks of a launch are independent until the
   kernel call ends (Sec. 2), so every launch's grid is split into contiguous block ranges,
   one per rank (``Launch.block_begin/block_count``: block indices keep the grid's
   numbering).  At each launch boundary - the implicit grid-wide synchronisation - the ranks
   exchange what they wrote: an all-reduce of the per-word change of the arena, exact because
   the blocks of a launch must not write a word another block touches (a word two ranks both
   changed is counted in ``conflicts``), and of the launch's status bits, so that a deadlock
   or step limit on any rank skips the launches that follow it on every rank (Sec. 3.1; Sec.
   3, streams and events).  Launches run in index order, which respects every stream and wait.

Collectives are ``torch.distributed`` (gloo on CPU ranks; the host-side exchange needs no
GPU-to-GPU path).
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, replace
from typing import Callable, List, Optional, Sequence

import numpy as np

from .workloads.ir import Launch, Program

REPORT_FIELDS = ("kind", "prog", "launch", "block", "epoch", "a", "b", "c")


def program_cost(p: Program) -> int:
    """Work estimate: the access-log bytes the library reserves for the program (what the
    interpreter writes and the race check reads), plus 8 bytes per simulated thread."""
    from .serving import predicted_log_bytes
    return max(1, predicted_log_bytes(p) + 8 * p.total_threads())


def shard(programs: Sequence[Program], world: int) -> List[List[int]]:
    """Indices of the programs each rank runs (LPT greedy on program_cost)."""
    order = sorted(range(len(programs)), key=lambda i: (-program_cost(programs[i]), i))
    heap = [(0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + program_cost(programs[i]), r))
    for r in range(world):
        out[r].sort()
    return out


@dataclass
class ShardResult:
    arenas: List[np.ndarray]
    status: np.ndarray
    reports: np.ndarray      # structured, canonical order, global program indices


def run_sharded(programs: Sequence[Program], executor: Callable, rank: int, world: int, group=None):
    """Run this rank's share with ``executor(list_of_programs) -> (arenas, status, reports)``
    (reports numbered locally) and gather everything to rank 0, which returns the merged
    ShardResult in the batch's global numbering; other ranks return None."""
    import torch.distributed as dist

    plan = shard(programs, world)
    mine = plan[rank]
    arenas, status, reports = executor([programs[i] for i in mine])
    reports = np.array(reports, copy=True)
    if len(reports):
        reports["prog"] = np.asarray(mine, dtype=np.uint32)[reports["prog"]]
    payload = (mine, [np.asarray(a) for a in arenas], np.asarray(status), reports)
    gathered = [None] * world if rank == 0 else None
    if world > 1:
        dist.gather_object(payload, gathered, dst=0, group=group)
    else:
        gathered = [payload]
    if rank != 0:
        return None
    out_arenas: List = [None] * len(programs)
    out_status = np.zeros(len(programs), dtype=np.uint32)
    parts = []
    for idx, ar, st, rep in gathered:
        for j, i in enumerate(idx):
            out_arenas[i] = ar[j]
            out_status[i] = st[j]
        parts.append(rep)
    reps = np.concatenate(parts) if parts else np.zeros(0)
    if len(reps):
        reps = reps[np.lexsort(tuple(reps[f] for f in reversed(("prog", "launch", "block", "epoch", "kind", "a",
                                                                   "b", "c"))))]
    return ShardResult(out_arenas, out_status, reps)


# ------------------------------------------------------------------ one program, split by blocks
def block_range(grid: int, rank: int, world: int):
    """Contiguous, balanced share [b0, b1) of a grid for `rank` (possibly empty)."""
    return grid * rank // world, grid * (rank + 1) // world


@dataclass
class SplitResult:
    arena: np.ndarray
    status: int
    reports: np.ndarray      # rank 0: every rank's reports in canonical order; others: their own
    conflicts: int           # words two ranks both changed in one launch (blocks racing across ranks)


ST_STOP = 1 | 2              # deadlock, step limit: the launches that follow are skipped


def run_split(program: Program, executor: Callable, rank: int, world: int, group=None) -> SplitResult:
    """Run ``program`` with each launch's blocks split across the ranks.  ``executor(program)``
    runs a one-launch program and returns (arena, status bits, reports); it sees this rank's
    block range in ``block_begin/block_count`` and the arena as the launch starts."""
    import torch
    import torch.distributed as dist

    def allreduce(x: np.ndarray, op) -> np.ndarray:
        t = torch.from_numpy(np.ascontiguousarray(x))
        if world > 1:
            dist.all_reduce(t, op=op, group=group)
        return t.numpy()

    arena = np.array(program.global_init, dtype=np.int32, copy=True)
    launches = program.launches
    dead = set()
    status, conflicts, parts = 0, 0, []
    for l, L in enumerate(launches):
        prev = next((k for k in range(l - 1, -1, -1) if launches[k].stream == L.stream), None)
        if (prev is not None and prev in dead) or (L.wait >= 0 and L.wait in dead):
            dead.add(l)                                   # skipped on every rank alike
            continue
        b0, b1 = block_range(L.grid, rank, world)
        new, st, reps = arena, 0, None
        if b1 > b0:
            one = replace(L, stream=0, wait=-1, block_begin=b0, block_count=b1 - b0)
            sub = Program(program.code, program.kernel_entry, [one], arena, name=program.name)
            new, st, reps = executor(sub)
            new = np.asarray(new, dtype=np.int32)
        # the exchange at the launch boundary: every rank's change of every word, summed
        delta = new.astype(np.int64) - arena.astype(np.int64)
        changed = (delta != 0).astype(np.int32)
        delta = allreduce(delta, dist.ReduceOp.SUM)
        changed = allreduce(changed, dist.ReduceOp.SUM)
        bits = allreduce(np.array([(int(st) >> k) & 1 for k in range(4)], dtype=np.int32), dist.ReduceOp.MAX)
        arena = ((arena.astype(np.int64) + delta) & 0xFFFFFFFF).astype(np.uint32).view(np.int32)
        conflicts += int(np.count_nonzero(changed > 1))
        st_all = int(sum(int(b) << k for k, b in enumerate(bits)))
        status |= st_all
        if st_all & ST_STOP:
            dead.add(l)
        if reps is not None and len(reps):
            reps = np.array(reps, copy=True)
            reps["launch"] = l
            parts.append(reps)
    mine = np.concatenate(parts) if parts else np.zeros(0, dtype=_report_dtype())
    if world > 1:
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(mine, gathered, dst=0, group=group)
        if rank == 0:
            mine = np.concatenate([g for g in gathered if len(g)] or [np.zeros(0, dtype=_report_dtype())])
    if rank == 0 and len(mine):
        order = ("prog", "launch", "block", "epoch", "kind", "a", "b", "c")      # canonical report order
        mine = mine[np.lexsort(tuple(mine[f] for f in reversed(order)))]
    return SplitResult(arena, status, mine, conflicts)


def _report_dtype():
    return np.dtype([(n, "<u4") for n in REPORT_FIELDS])


def library_executor(**opts) -> Callable:
    """The library as a rank's executor: ``f(programs) -> (arenas, status, reports)`` for
    run_sharded, or ``f(program) -> (arena, status, reports)`` for run_split."""
    from . import binding

    def run(progs):
        single = isinstance(progs, Program)
        r = binding.check([progs] if single else list(progs), **opts)
        if single:
            return r.arenas[0], int(r.status[0]), r.reports
        return r.arenas, r.status, r.reports
    return run
