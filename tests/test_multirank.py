"""Multi-rank sharding on CPU ranks (gloo, world size 2): every program runs on exactly
one rank, and the merged reports/arenas equal a single-rank run.  The per-rank executor
here is the oracle (no GPU needed); the GPU path plugs the library in the same place."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1211_6193_gb300 import dist as sdist
from paper_1211_6193_gb300.workloads import families, fig1


def _programs():
    return families.batch(n_programs=14, seed=21, max_grid=3, bug_rate=0.5) + \
        [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True)]


def _oracle_exec(progs):
    r = oracle.run(progs)
    return r.arenas, r.status, r.reports


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = sdist.run_sharded(_programs(), _oracle_exec, rank, world)
    if rank == 0:
        np.save(os.path.join(outdir, "reports.npy"), res.reports)
        np.save(os.path.join(outdir, "status.npy"), res.status)
        np.savez(os.path.join(outdir, "arenas.npz"), *res.arenas)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_plan_is_a_balanced_partition():
    progs = _programs()
    plan = sdist.shard(progs, 3)
    assert sorted(i for r in plan for i in r) == list(range(len(progs)))
    loads = [sum(sdist.program_cost(progs[i]) for i in r) for r in plan]
    assert max(loads) - min(loads) <= max(sdist.program_cost(p) for p in progs)
    assert sdist.shard(progs, 3) == plan            # deterministic: every rank agrees


def test_two_gloo_ranks_match_single_rank(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    ref = oracle.run(_programs())
    reps = np.load(tmp_path / "reports.npy")
    assert [tuple(int(x) for x in r) for r in reps] == ref.report_tuples()
    assert np.array_equal(np.load(tmp_path / "status.npy"), ref.status)
    ar = np.load(tmp_path / "arenas.npz")
    for i, a in enumerate(ref.arenas):
        assert np.array_equal(ar[f"arr_{i}"], a)
