"""Autotuner: selection and caching on the CPU with a fake measurement; on the GPU, every
candidate shape gives the same reports and the tuned options reproduce the oracle."""
import numpy as np
import pytest

from paper_1211_6193_gb300 import autotune
from paper_1211_6193_gb300.workloads import families, fig1


def _fake(times_i, times_c, digest="d", fused=(9.0, 0.0)):
    calls = []

    def measure(programs, opts):
        calls.append(dict(opts))
        if opts.get("fused_check"):
            return fused[0], fused[1], digest
        key = autotune._key({k: v for k, v in opts.items() if k in ("interp_variant", "ctas_per_sm")})
        return times_i.get(key, 1.0), times_c.get(opts.get("check_variant", 0), 1.0), digest

    return measure, calls


def test_picks_fastest_interp_then_fastest_checker_behind_it():
    progs = [fig1.program()]
    m, calls = _fake({"interp_variant=1": 3.0, "interp_variant=2": 2.0}, {1: 5.0, 2: 4.0, 3: 1.5, 4: 2.5, 5: 3.0, 6: 2.0, 7: 2.2})
    t = autotune.tune(progs, "plain", measure=m, device="fake")
    assert t.options == {"mode": "plain", "interp_variant": 2, "check_variant": 3}
    # checker variants, then the fused check, were all timed behind the chosen interpreter
    assert [c.get("check_variant") for c in calls[2:]] == list(autotune.CHECK_VARIANTS) + [None]
    assert calls[-1]["fused_check"] == 1
    assert all(c["interp_variant"] == 2 for c in calls[2:])
    m, _ = _fake({"ctas_per_sm=1": 1.0, "ctas_per_sm=2": 2.0}, {1: 1.0})
    assert autotune.tune(progs, "batched", measure=m, device="fake").options == \
        {"mode": "batched", "ctas_per_sm": 1, "check_variant": 1}


def test_fused_check_kept_only_when_the_whole_run_is_faster():
    progs = [fig1.program()]
    # interpreter 2.0 + checker 1.5 = 3.5: fused 3.4 wins, 3.6 does not
    checks = {1: 2.0, 2: 2.0, 3: 1.5, 4: 2.0, 5: 2.0, 6: 2.0, 7: 2.0}
    m, _ = _fake({"interp_variant=1": 3.0, "interp_variant=2": 2.0}, checks, fused=(3.3, 0.1))
    t = autotune.tune(progs, "plain", measure=m, device="fake")
    assert t.options == {"mode": "plain", "interp_variant": 2, "fused_check": 1}
    assert t.fused_ms == pytest.approx(3.4)
    m, _ = _fake({"interp_variant=1": 3.0, "interp_variant=2": 2.0}, checks, fused=(3.5, 0.1))
    assert autotune.tune(progs, "plain", measure=m, device="fake").options == \
        {"mode": "plain", "interp_variant": 2, "check_variant": 3}
    m, calls = _fake({}, {}, fused=(0.1, 0.0))
    t = autotune.tune(progs, "plain", measure=m, device="fake", fused=False)
    assert "fused_check" not in t.options and t.fused_ms is None
    assert not any(c.get("fused_check") for c in calls)


def test_shapes_the_library_rejects_are_skipped():
    def measure(programs, opts):
        if opts.get("ctas_per_sm") == 2 or opts.get("fused_check"):
            raise autotune.NotApplicable("shared memory does not fit")
        return 1.0, float(opts.get("check_variant", 0)), "d"

    t = autotune.tune([fig1.program()], "batched", measure=measure, device="fake")
    assert t.options == {"mode": "batched", "ctas_per_sm": 1, "check_variant": 1}
    assert list(t.interp_ms) == ["ctas_per_sm=1"]

    def never(programs, opts):
        raise autotune.NotApplicable("no")

    with pytest.raises(autotune.NotApplicable):
        autotune.tune([fig1.program()], "batched", measure=never, device="fake")


def test_disagreeing_variants_are_an_error():
    n = iter(range(100))

    def measure(programs, opts):
        return 1.0, 1.0, str(next(n))

    with pytest.raises(RuntimeError):
        autotune.tune([fig1.program()], "plain", measure=measure, device="fake")


def test_cache_round_trip_and_signature(tmp_path):
    progs = families.batch(n_programs=6, seed=4, max_grid=8)
    path = str(tmp_path / "tune.json")
    m, calls = _fake({}, {4: 0.5})
    first = autotune.tune(progs, "batched", measure=m, cache_path=path, device="fake")
    assert not first.cached and first.options["check_variant"] == 4
    ncalls = len(calls)
    again = autotune.tune(progs, "batched", measure=m, cache_path=path, device="fake")
    assert again.cached and again.options == first.options and len(calls) == ncalls
    # another device, mode or launch shape is another signature
    s = autotune.signature(progs, "batched", "fake")
    assert s != autotune.signature(progs, "plain", "fake")
    assert s != autotune.signature(progs, "batched", "fake", fused=False)
    assert s != autotune.signature(progs, "batched", "other")
    assert s != autotune.signature(progs[:-1], "batched", "fake")


@pytest.mark.gpu
def test_tuned_options_on_the_gpu_match_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1211_6193_gb300 import binding, build
    build.build()
    progs = families.batch(n_programs=24, seed=9, max_grid=16, bug_rate=0.5)
    t = autotune.tune(progs, "batched", measure=autotune.gpu_measure(repeats=1))
    assert set(t.check_ms) == {str(v) for v in autotune.CHECK_VARIANTS}
    got = binding.check(progs, **t.options)
    want = oracle.run(progs)
    assert got.report_tuples() == want.report_tuples()
    assert all(np.array_equal(a, b) for a, b in zip(got.arenas, want.arenas))
