"""The library built with SR_DEBUG_BOUNDS (internal index checks before every register,
code, log-region, checker and gather access; a failed check skips the access and is reported
as SR_ST_BOUNDS / SR_E_BOUNDS instead of faulting).  It stands in for a memory checker that
cannot run on these GPUs.  This test runs parity programs of every kind through the debug
library, in a process of its own so that it is the only libsimtcheck loaded there: no check
may fail and every result must equal the oracle's."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SCRIPT = r'''
import sys
sys.path[:0] = [ROOT, HERE]
import numpy as np
import oracle
from paper_1211_6193_gb300 import binding, build
binding.load_library(build.DEBUG_LIB)
from paper_1211_6193_gb300.workloads import families, fig1, stencil2d, tiny
import stream_programs as sp
from test_gpu_parity import tag_wrap_program
progs = [fig1.program(), fig1.program(race=True), fig1.program(deadlock=True),
         families.reduction_plain(n_blocks=40), stencil2d.program(log2w=7, steps=4, buggy_launch=2)]
progs += families.batch(n_programs=48, seed=3, max_grid=6, bug_rate=0.5)
progs += tiny.tiny_batch(77, 30, nthreads=40, nsteps=6, nwords=5) + sp.all_programs()
checked = 0
for opts in ({"mode": "plain"}, {"mode": "batched"}, {"mode": "plain", "check_variant": 1},
             {"mode": "batched", "check_uninit": True}, {"mode": "plain", "check_global": True}):
    kw = {"check_uninit": True} if opts.get("check_uninit") else {}
    if opts.get("check_global"):
        kw["check_global"] = True
    want = oracle.run(progs, **kw)
    got = binding.check(progs, **opts)
    assert got.report_tuples() == want.report_tuples(), opts
    for i in range(len(progs)):
        assert np.array_equal(got.arenas[i], want.arenas[i]), (opts, i)
    assert not np.any(got.status & binding.ST_BOUNDS), (opts, got.status)
    assert list(got.status & 3) == list(want.status), opts
    checked += len(progs)
p = tag_wrap_program(20000)
got = binding.check([p], mode="plain", loop_log_records=1 << 17)
assert got.report_tuples() == oracle.run([p]).report_tuples() and not (got.status[0] & binding.ST_BOUNDS)
print("debug build ok", checked + 1)
'''


def test_debug_build_has_no_failed_index_check_and_matches_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_6193_gb300 import build
    build.build(debug=True)
    code = f"ROOT = {ROOT!r}\nHERE = {HERE!r}\n" + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
