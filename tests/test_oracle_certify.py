"""Certification of a reading on the full-size workloads (CPU only).

Reading: programs must not share a written global word between the blocks of a launch,
because blocks run concurrently on the GPU while the oracle runs them in order (Sec. 2:
nothing but the end of a kernel call orders the blocks of a grid).  The oracle's
``check_interblock`` diagnostic counts such words; it is pinned in test_oracle_global.py.
Here it runs on every 64th program of the 4096-program batch at full size; the whole batch
and the full 8192^2 stencil are certified inside the full-size GPU parity tests, which run
the oracle over them anyway."""
import os

import oracle
from paper_1211_6193_gb300.workloads import families, stencil2d


def test_full_size_batch_sample_has_no_interblock_conflicts():
    progs = families.batch(n_programs=4096, seed=3, indices=range(0, 4096, 64))
    r = oracle.run(progs, check_interblock=True, nthreads=os.cpu_count() or 1)
    assert r.interblock_conflicts == 0


def test_stencil_sample_has_no_interblock_conflicts():
    p = stencil2d.program(log2w=13, steps=2, buggy_launch=1, seed=4)
    r = oracle.run([p], check_interblock=True, max_blocks=512, nthreads=os.cpu_count() or 1)
    assert r.interblock_conflicts == 0
