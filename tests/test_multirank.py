"""Multi-rank execution on CPU ranks (gloo): sharding a batch (every program runs on exactly
one rank) and splitting one program's launches by block range with the arena exchange at
every launch boundary; merged reports, arenas and status equal a single-rank run.  The
per-rank executor here is the oracle (no GPU needed); tests/test_gpu_multirank.py plugs the
library in the same place."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1211_6193_gb300 import dist as sdist
from paper_1211_6193_gb300.workloads import families, fig1, stencil2d


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


def _split_programs():
    import stream_programs as sp
    return [stencil2d.program(log2w=6, steps=4, buggy_launch=2, seed=4),
            families.reduction_plain(n_blocks=7, bdim=256, seed=1, omit_level=3),
            fig1.program(), fig1.program(race=True), fig1.program(deadlock=True), sp.fork_join(True),
            sp.fork_join(False)]


def _oracle_one(prog):
    r = oracle.run([prog])
    return r.arenas[0], int(r.status[0]), r.reports


def _split_worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for i, p in enumerate(_split_programs()):
        res = sdist.run_split(p, _oracle_one, rank, world)
        if rank == 0:
            np.save(os.path.join(outdir, f"rep{i}.npy"), res.reports)
            np.save(os.path.join(outdir, f"arena{i}.npy"), res.arena)
            np.save(os.path.join(outdir, f"st{i}.npy"), np.array([res.status, res.conflicts]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_launches_across_gloo_ranks_match_single_rank(tmp_path, world):
    port = _free_port()
    mp.start_processes(_split_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    for i, p in enumerate(_split_programs()):
        ref = oracle.run([p])
        reps = np.load(tmp_path / f"rep{i}.npy")
        assert [tuple(int(x) for x in r) for r in reps] == ref.report_tuples(), (world, p.name)
        assert np.array_equal(np.load(tmp_path / f"arena{i}.npy"), ref.arenas[0]), (world, p.name)
        st, conflicts = np.load(tmp_path / f"st{i}.npy")
        assert int(st) == int(ref.status[0]) and int(conflicts) == 0, (world, p.name)


def test_block_ranges_partition_the_grid():
    for grid in (1, 2, 7, 16384):
        for world in (1, 2, 3, 8):
            rs = [sdist.block_range(grid, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == grid
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(e - b for b, e in rs) - min(e - b for b, e in rs) <= 1


def test_cost_is_the_reserved_log_bytes():
    from paper_1211_6193_gb300 import serving
    p = families.reduction_plain(n_blocks=5)
    assert sdist.program_cost(p) == serving.predicted_log_bytes(p) + 8 * p.total_threads()
