"""The multi-rank paths with the library as every rank's executor: two processes (gloo for
the host-side exchange) on the one GPU a test box has.  Neither waits on the other's
kernels - each rank runs whole launches of its own and the ranks meet only in host
collectives - so sharing one GPU is safe.  Results must equal a single-rank oracle run.

  - run_sharded: a batch of independent programs, each run by exactly one rank;
  - run_split: one program per call, every launch's blocks split between the ranks, the
    arena exchanged at each launch boundary."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1211_6193_gb300.workloads import families, fig1, stencil2d

pytestmark = pytest.mark.gpu


def _batch():
    return families.batch(n_programs=24, seed=21, max_grid=40, bug_rate=0.5) + \
        [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True)]


def _split_programs():
    import stream_programs as sp
    return [stencil2d.program(log2w=8, steps=4, buggy_launch=2, seed=4),
            families.reduction_plain(n_blocks=300, bdim=1024, seed=1, omit_level=3),
            fig1.program(deadlock=True), sp.fork_join(True)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    import torch
    import torch.distributed as dist

    from paper_1211_6193_gb300 import dist as sdist
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    for mode in ("plain", "batched"):
        ex = sdist.library_executor(mode=mode)
        res = sdist.run_sharded(_batch(), ex, rank, world)
        if rank == 0:
            np.save(os.path.join(outdir, f"shard_{mode}_rep.npy"), res.reports)
            np.save(os.path.join(outdir, f"shard_{mode}_st.npy"), res.status)
            np.savez(os.path.join(outdir, f"shard_{mode}_ar.npz"), *res.arenas)
        for i, p in enumerate(_split_programs()):
            r = sdist.run_split(p, ex, rank, world)
            if rank == 0:
                np.save(os.path.join(outdir, f"split_{mode}_{i}_rep.npy"), r.reports)
                np.save(os.path.join(outdir, f"split_{mode}_{i}_ar.npy"), r.arena)
                np.save(os.path.join(outdir, f"split_{mode}_{i}_st.npy"), np.array([r.status, r.conflicts]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_one_gpu_match_the_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import build
    build.build()
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    ref = oracle.run(_batch())
    for mode in ("plain", "batched"):
        reps = np.load(tmp_path / f"shard_{mode}_rep.npy")
        assert [tuple(int(x) for x in r) for r in reps] == ref.report_tuples(), mode
        assert np.array_equal(np.load(tmp_path / f"shard_{mode}_st.npy") & 3, ref.status), mode
        ar = np.load(tmp_path / f"shard_{mode}_ar.npz")
        for i, a in enumerate(ref.arenas):
            assert np.array_equal(ar[f"arr_{i}"], a), (mode, i)
        for i, p in enumerate(_split_programs()):
            want = oracle.run([p])
            reps = np.load(tmp_path / f"split_{mode}_{i}_rep.npy")
            assert [tuple(int(x) for x in r) for r in reps] == want.report_tuples(), (mode, p.name)
            assert np.array_equal(np.load(tmp_path / f"split_{mode}_{i}_ar.npy"), want.arenas[0]), (mode, p.name)
            st, conflicts = np.load(tmp_path / f"split_{mode}_{i}_st.npy")
            assert (int(st) & 3) == int(want.status[0]) and int(conflicts) == 0, (mode, p.name)
