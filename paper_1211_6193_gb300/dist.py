"""Multi-GPU sharding of a batch of independent programs (one process per GPU).

Programs never communicate (Sec. 2: only the launches of one program share an arena),
so ranks run disjoint subsets of the batch with no data-path collective; the only
exchange is the final gather of reports, status and arenas to rank 0 (host side,
``torch.distributed`` object collectives - gloo on CPU ranks).

Assignment balances a static cost estimate per program (threads x static length, plus
its access-log bound) with a longest-processing-time greedy, deterministic in the
program order so every rank computes the same plan.
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from typing import Callable, List, Sequence

import numpy as np

from .workloads.ir import Program

REPORT_FIELDS = ("kind", "prog", "launch", "block", "epoch", "a", "b", "c")


def program_cost(p: Program) -> int:
    """Static work estimate: simulated threads x static instructions (at least 1)."""
    return max(1, sum(l.grid * l.block_dim for l in p.launches) * max(1, p.ncode))


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
