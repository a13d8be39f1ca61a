"""GPU test of sr_check_program_noalloc, the entry point for callers that cannot
allocate device memory (frameworks that own all device memory through their own
allocator, processes that forbid cudaMalloc after start-up).  Everything it needs besides
the caller's arena and report buffer lives in a fixed __device__ array inside the library.

Its results must equal those of the allocating entry points (load_programs,
run_and_check, fetch_reports, fetch_memory, sr_batch_status) on the same programs, on two
calls in a row (the array keeps the previous call's contents)."""
import ctypes as C

import numpy as np
import pytest

from paper_1211_6193_gb300.workloads import families, fig1, stencil2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import binding, build
    build.build()
    return torch, binding, binding.load_library()


def _programs():
    from stream_programs import all_programs
    return [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True),
            families.reduction_plain(n_blocks=64),
            stencil2d.program(log2w=7, steps=3, buggy_launch=1)] + \
        families.batch(n_programs=6, seed=17, max_grid=8, bug_rate=0.7) + all_programs()


def _noalloc(env, prog, cap):
    torch, binding, lib = env
    m = binding._Marshalled([prog])
    arena = torch.from_numpy(np.array(prog.global_init, dtype=np.int32)).cuda()
    reps = torch.zeros(max(1, cap) * 8, dtype=torch.int32, device="cuda")
    n, st = C.c_uint64(), C.c_uint32()
    rc = lib.sr_check_program_noalloc(m.array, arena.data_ptr(), reps.data_ptr(), cap, C.byref(n), C.byref(st),
                                      torch.cuda.current_stream().cuda_stream)
    out = reps[: int(n.value) * 8].cpu().numpy().view(binding.REPORT_DTYPE) if rc == 0 else None
    return rc, out, arena.cpu().numpy(), int(n.value), int(st.value)


def test_noalloc_matches_allocating_entry_points_on_two_calls(env):
    torch, binding, lib = env
    for prog in _programs():
        ref = binding.check([prog])
        for call in range(2):
            rc, reps, arena, n, st = _noalloc(env, prog, len(ref.reports) + 4)
            assert rc == binding.SR_OK, (prog.name, call, rc)
            assert n == len(ref.reports)
            assert [tuple(int(x) for x in r) for r in reps] == ref.report_tuples(), (prog.name, call)
            assert np.array_equal(arena, ref.arenas[0]), (prog.name, call)
            assert st == int(ref.status[0]), (prog.name, call)


def test_noalloc_rejects_what_does_not_fit(env):
    torch, binding, lib = env
    # a report buffer that is too small: the count is still returned
    prog = fig1.program(race=True)
    rc, _, _, n, _ = _noalloc(env, prog, 2)
    assert rc == binding.SR_E_RANGE and n == 6
    # logs beyond the fixed scratch (the full 2^24-element reduction needs gigabytes)
    big = families.reduction_plain(n_blocks=16384)
    rc, _, _, _, _ = _noalloc(env, big, 16)
    assert rc == binding.SR_E_RANGE


def test_noalloc_runs_launches_in_several_waves(env):
    """Launches whose logs each fit the array but not together run wave by wave (the log
    space is reused, the report total carries over from wave to wave)."""
    torch, binding, lib = env
    from paper_1211_6193_gb300 import serving
    prog = stencil2d.program(log2w=9, steps=3, buggy_launch=1)
    one = stencil2d.program(log2w=9, steps=1, buggy_launch=None)
    per_launch = serving.predicted_log_bytes(one)          # the library's static bound
    fixed_min = 8 * (1 << 14) * 16                          # the checker's staging alone
    assert per_launch <= binding.NOALLOC_SCRATCH_BYTES - fixed_min - (1 << 20)   # one launch fits
    assert 2 * per_launch > binding.NOALLOC_SCRATCH_BYTES - fixed_min           # two do not: 3 waves
    ref = binding.check([prog])
    assert len(ref.reports) > 0                  # launch 1 omits the staging barrier
    for call in range(2):
        rc, reps, arena, n, st = _noalloc(env, prog, len(ref.reports) + 4)
        assert rc == binding.SR_OK, (call, rc)
        assert [tuple(int(x) for x in r) for r in reps] == ref.report_tuples(), call
        assert np.array_equal(arena, ref.arenas[0]), call
        assert st == int(ref.status[0]), call


def test_noalloc_refuses_a_capturing_stream(env):
    """On a stream that is being captured the call returns SR_E_INVAL before touching the
    stream, and the caller's capture goes on unharmed."""
    torch, binding, lib = env
    prog = fig1.program()
    m = binding._Marshalled([prog])
    arena = torch.from_numpy(np.array(prog.global_init, dtype=np.int32)).cuda()
    reps = torch.zeros(64, dtype=torch.int32, device="cuda")
    x = torch.zeros(4, device="cuda")
    n, st = C.c_uint64(), C.c_uint32()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=side):
        x.add_(1)
        rc = lib.sr_check_program_noalloc(m.array, arena.data_ptr(), reps.data_ptr(), 8, C.byref(n), C.byref(st),
                                          torch.cuda.current_stream().cuda_stream)
        still = torch.cuda.is_current_stream_capturing()
        x.add_(1)
    assert rc == binding.SR_E_INVAL and still
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 2.0
    # the array was not touched: the next call outside the capture is correct
    rc2, reps2, arena2, n2, st2 = _noalloc(env, prog, 8)
    ref = binding.check([prog])
    assert rc2 == binding.SR_OK and np.array_equal(arena2, ref.arenas[0]) and n2 == len(ref.reports)
