"""C-ABI checks that need no GPU: the library builds, loads, exports every entry point
declared in include/*.h, and validates programs on the host."""
import ctypes
import os
import subprocess
import re

import numpy as np
import pytest

from paper_1211_6193_gb300 import binding, build
from paper_1211_6193_gb300.workloads import families, fig1, ir

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load_library()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["load_programs", "run_and_check", "fetch_reports", "fetch_memory", "sr_create", "sr_destroy",
              "sr_batch_status", "sr_free_batch", "sr_last_error", "sr_validate_program", "sr_batch_stats"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    assert sorted(binding.EXPORTS) == sorted(n for n in declared_functions() if n in binding.EXPORTS)
    assert set(declared_functions()) <= set(binding.EXPORTS) | set()


def test_struct_layouts_match_header(tmp_path):
    # 8-byte instruction, 32-byte report, launch = 13 words
    assert ctypes.sizeof(binding.sr_instr) == 8
    assert ctypes.sizeof(binding.sr_launch) == 52
    assert binding.REPORT_DTYPE.itemsize == 32
    assert ir.INSTR_DTYPE.itemsize == 8
    # the C compiler's layout of the header's sr_launch equals the binding's
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "simtcheck.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sr_launch),'
                   ' offsetof(sr_launch, params), offsetof(sr_launch, stream), offsetof(sr_launch, wait),'
                   ' offsetof(sr_launch, block_count), sizeof(sr_opts), offsetof(sr_opts, check_global),'
                   ' sizeof(sr_stats), offsetof(sr_stats, ms_global), offsetof(sr_stats, global_records));'
                   ' return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(binding.sr_launch), binding.sr_launch.params.offset, binding.sr_launch.stream.offset,
            binding.sr_launch.wait.offset, binding.sr_launch.block_count.offset, ctypes.sizeof(binding.sr_opts),
            binding.sr_opts.check_global.offset, ctypes.sizeof(binding.sr_stats), binding.sr_stats.ms_global.offset,
            binding.sr_stats.global_records.offset]
    assert got == want


def test_opcode_numbers_match_header():
    txt = open(os.path.join(ROOT, "include", "simtcheck.h")).read()
    body = re.search(r"enum \{\s*SR_OP_MOV = 1,(.*?)\};", txt, re.S).group(1)
    names = ["MOV"] + [n.strip()[6:] for n in body.replace("\n", " ").split(",") if n.strip()]
    for i, nm in enumerate(names, start=1):
        assert getattr(ir, nm) == i, nm
    assert "#define SR_BIMM 0x80u" in txt and ir.BIMM == 0x80


def test_all_programs_sentinel_matches_header():
    txt = open(os.path.join(ROOT, "include", "simtcheck.h")).read()
    assert re.search(r"#define SR_ALL_PROGRAMS 0x([0-9A-Fa-f]+)u", txt).group(1).lower() == \
        f"{binding.SR_ALL_PROGRAMS:x}"


def _validate(lib, prog):
    m = binding._Marshalled([prog])
    buf = ctypes.create_string_buffer(256)
    return lib.sr_validate_program(m.array, buf, 256), buf.value.decode()


def test_host_validation_accepts_generated_programs(lib):
    for p in [fig1.program(), fig1.program(race=True), families.reduction_plain(n_blocks=2)] + \
            families.batch(n_programs=16, seed=5, max_grid=2):
        assert _validate(lib, p) == (0, "")


@pytest.mark.parametrize("mutate,needle", [
    (lambda c: c.__setitem__(0, ((int(c[0]["op_d_a_b"]) & 0xFFFFFF00) | 63, int(c[0]["imm"]))), "opcode"),
    (lambda c: c.__setitem__(1, (ir.encode(ir.ADD, 20, 1, 2)[0], 0)), "register"),
    (lambda c: c.__setitem__(2, ir.encode(ir.BRA, 0, 0, 0, 10_000)), "branch"),
    (lambda c: c.__setitem__(2, ir.encode(ir.S2R, 3, 0, 0, 9)), "special"),
    (lambda c: c.__setitem__(2, ir.encode(ir.LDS | ir.BIMM, 3, 1, 0, 0)), "opcode"),
])
def test_host_validation_rejects_bad_programs(lib, mutate, needle):
    p = fig1.program()
    code = p.code.copy()
    mutate(code)
    q = ir.Program(code, p.kernel_entry, p.launches, p.global_init)
    rc, msg = _validate(lib, q)
    assert rc == binding.SR_E_INVAL and needle in msg


@pytest.mark.parametrize("launch,needle", [
    (ir.Launch(0, 0, 32, 0, ()), "grid"),
    (ir.Launch(0, 1, 1025, 0, ()), "block_dim"),
    (ir.Launch(0, 1, 32, 12289, ()), "shmem"),
    (ir.Launch(3, 1, 32, 0, ()), "kernel"),
])
def test_host_validation_rejects_bad_launches(lib, launch, needle):
    p = fig1.program()
    q = ir.Program(p.code, p.kernel_entry, [launch], p.global_init)
    rc, msg = _validate(lib, q)
    assert rc == binding.SR_E_INVAL and needle in msg
