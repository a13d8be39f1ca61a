"""Serving: continuous batching over streams.  CPU tests cover the arrival trace and the
admission estimate; the GPU test checks that every job's result is the same alone and in
the mix, and that batches really overlapped."""
import numpy as np
import pytest

from paper_1211_6193_gb300 import serving
from paper_1211_6193_gb300.workloads import families, fig1


def test_poisson_trace_rate_and_order():
    t = serving.poisson_trace(2000.0, 5.0, seed=5)
    assert all(a < b for a, b in zip(t, t[1:])) and 0 <= t[0] and t[-1] < 5.0
    assert abs(len(t) / 5.0 - 2000.0) < 4 * np.sqrt(2000.0 * 5.0) / 5.0     # within 4 sigma
    gaps = np.diff(t)
    assert abs(np.mean(gaps) - 1 / 2000.0) < 0.05 / 2000.0 * 10


def test_predicted_log_bytes_hand_values():
    # reduction, 1024 threads: the longest path makes 1 + 3 x 10 + 1 = 32 shared accesses and
    # crosses 10 barriers (staging + 9 of the 10 level barriers; the level-3 one is missing);
    # error-capable pcs: 1 LDG, 1 STS, 30 level LDS/STS, 1 LDS, 1 STG -> 34
    p = families.reduction_plain(n_blocks=5)
    cyc, acc, bars, errs = serving._kernel_bound(p.code, 0)
    assert (cyc, acc, bars, errs) == (False, 32, 10, 34)
    misc = (bars + 1) * (1 + errs) + 1
    assert serving.predicted_log_bytes(p) == 5 * (((32 * 1024 + 2 * misc + 1) & ~1) * 8)
    # Figure 1 has a loop: the fixed per-block region applies
    cyc, *_ = serving._kernel_bound(fig1.program().code, 0)
    assert cyc


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import binding, build
    build.build()
    pool = serving.job_pool(12, seed=5, max_grid=24) + [fig1.program(race=True), fig1.program(deadlock=True)]
    # the admission estimate is what the library reserves
    for p in pool[:4]:
        with binding.Context() as ctx, ctx.load_programs([p]) as b:
            assert b.stats().log_bytes == serving.predicted_log_bytes(p)
    arrivals = serving.poisson_trace(4000.0, 0.02, seed=7)
    jobs = [serving.Job(k, pool[k % len(pool)], t) for k, t in enumerate(arrivals)]
    srv = serving.Server(log_budget_bytes=64 << 20, max_inflight=3, max_batch_jobs=4)
    results, st = srv.serve(jobs)
    srv.close()
    assert st.jobs == len(jobs) and st.batches >= 3 and st.max_inflight_seen >= 2
    import oracle
    alone = {}
    for j in jobs:
        key = id(j.program)
        if key not in alone:
            alone[key] = binding.check([j.program])
            # and alone it is the oracle's result
            want = oracle.run([j.program])
            assert alone[key].report_tuples() == want.report_tuples(), j.program.name
            assert np.array_equal(alone[key].arenas[0], want.arenas[0]), j.program.name
            assert int(alone[key].status[0]) & 3 == int(want.status[0]), j.program.name
        a, r = alone[key], results[j.jid]
        # every field but `prog` (the job's slot in its micro-batch)
        assert [tuple(int(x) for x in t)[:1] + tuple(int(x) for x in t)[2:] for t in r.reports] == \
            [t[:1] + t[2:] for t in a.report_tuples()], j.jid
        assert np.array_equal(r.arena, a.arenas[0]), j.jid
        assert r.status == int(a.status[0]), j.jid


@pytest.mark.gpu
def test_serving_job_pool_matches_the_oracle():
    """The 512-program pool the serving benchmark draws its jobs from (seed 5, full-size
    grids), run as one batch, against the oracle on every program (a slice at a time)."""
    import os

    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1211_6193_gb300 import binding, build
    build.build()
    pool = serving.job_pool(512, seed=5)
    got = binding.check(pool, mode="batched")
    reps = got.reports
    cut = np.searchsorted(reps["prog"], np.arange(0, len(pool) + 1, dtype=np.uint32))
    for i0 in range(0, len(pool), 128):
        i1 = min(len(pool), i0 + 128)
        want = oracle.run(pool[i0:i1], nthreads=os.cpu_count() or 1)
        w = want.reports.copy()
        w["prog"] += np.uint32(i0)
        assert [tuple(int(x) for x in r) for r in reps[cut[i0]:cut[i1]]] == [tuple(int(x) for x in r) for r in w]
        for k in range(i0, i1):
            assert np.array_equal(got.arenas[k], want.arenas[k - i0]), k
        assert list(got.status[i0:i1] & 3) == list(want.status)
