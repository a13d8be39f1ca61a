"""Full-size parity: the batched workload (4096 seed-generated programs, 1.97M blocks, in both
batched shapes) and the log-heavy stencil (8192^2 int32, 16 launches) in the launch
configuration bench.py times,
every report, every arena word and every status compared with the oracle (run on all host
cores, a slice of programs at a time so that host memory stays bounded)."""
import os

import numpy as np
import pytest

import oracle
from paper_1211_6193_gb300.workloads import families, stencil2d

pytestmark = pytest.mark.gpu
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import binding, build
    build.build()
    binding.load_library()
    return binding


def _same_reports(got, want, prog_offset=0):
    assert len(got) == len(want), (len(got), len(want))
    for f in want.dtype.names:
        w = want[f] + np.uint32(prog_offset) if f == "prog" else want[f]
        bad = np.nonzero(got[f] != w)[0]
        assert bad.size == 0, (f, bad[:5], got[bad[:5]], want[bad[:5]])


def test_full_size_batched(B):
    """Both batched shapes: one CTA per SM, and two CTAs per SM - the autotuner's pick for this
    workload, the one bench.py times - each against one oracle run."""
    progs = families.batch(n_programs=4096, seed=3)
    with B.Context(mode="batched") as c1, c1.load_programs(progs) as b1, \
            B.Context(mode="batched", ctas_per_sm=2) as c2, c2.load_programs(progs) as b2:
        runs = []
        for b in (b1, b2):
            b.run_and_check()
            reps = b.fetch_reports()
            assert b.stats().shared_accesses == 6102466019
            cut = np.searchsorted(reps["prog"], np.arange(0, len(progs) + 1, dtype=np.uint32))
            runs.append((b, reps, b.all_status(), cut))
        assert b1.stats().one_per_cta_blocks == 0
        assert 0 < b2.stats().one_per_cta_blocks < b2.stats().blocks
        step = 256
        for i0 in range(0, len(progs), step):
            i1 = min(len(progs), i0 + step)
            # check_interblock certifies the reading that no two blocks of a launch share a
            # written global word (blocks run concurrently here, in order in the oracle)
            want = oracle.run(progs[i0:i1], nthreads=CORES, check_interblock=True)
            assert want.interblock_conflicts == 0, i0
            for b, reps, status, cut in runs:
                _same_reports(reps[cut[i0]:cut[i1]], want.reports, prog_offset=i0)
                for k in range(i0, i1):
                    assert np.array_equal(b.fetch_memory(k), want.arenas[k - i0]), k
                assert list(status[i0:i1] & 3) == list(want.status)
                assert not np.any(status[i0:i1] & (B.ST_LOG_OVERFLOW | B.ST_INTERNAL))


def test_full_size_stencil(B):
    p = stencil2d.program(log2w=13, steps=16, buggy_launch=8, seed=4)
    got = B.check([p], mode="plain")
    want = oracle.run([p], nthreads=CORES, check_interblock=True)
    assert want.interblock_conflicts == 0
    _same_reports(got.reports, want.reports)
    assert np.array_equal(got.arenas[0], want.arenas[0])
    assert int(got.status[0]) == int(want.status[0]) == 0
    assert got.stats.shared_accesses == want.shared_accesses
    # launch 8 omits the staging barrier: every block reports its 32 x 32 interior writes
    # racing with the neighbours' reads (1024 races per block, 65536 blocks)
    assert len(got.reports) == 65536 * 1024
