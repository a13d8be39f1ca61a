"""Sensitivity of the oracle pins: plant plausible mistakes in a temporary copy of the
oracle's C source (never in the committed oracle) and check that the pin suite fails for
every one of them."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "simt_oracle.c")

MUTANTS = {
    "stores_lowest_tid_wins": (
        "for (uint64_t i = 0; i < B->sst.n; ++i) B->sh[B->sst.v[i].addr] = B->sst.v[i].val;",
        "for (uint64_t i = B->sst.n; i-- > 0;) B->sh[B->sst.v[i].addr] = B->sst.v[i].val;"),
    "atomic_atomic_is_race": (
        "if (!bit) continue;",
        "if (!bit && !(k1 == K_A && k2 == K_A)) continue; if (!bit) bit = ORC_CLS_WA;"),
    "history_not_cleared_at_barrier": ("  B->acc.n = 0;\n  if (B->gacc.n)", "  if (B->gacc.n)"),
    "global_history_not_cleared_at_barrier": ("  B->gacc.n = 0;\n", ""),
    "same_thread_pairs_race": ("if (p->tid == q->tid) continue;", ""),
    "stores_visible_within_round": (
        "if (B->deferred) st_push(&B->sst, addr, vb); else B->sh[addr] = vb;", "B->sh[addr] = vb;"),
    "atomics_before_stores": (
        "  for (uint64_t i = 0; i < B->sst.n; ++i) B->sh[B->sst.v[i].addr] = B->sst.v[i].val;\n",
        "  for (uint64_t i = 0; i < B->ats.n; ++i) B->sh[B->ats.v[i].addr] = "
        "add32(B->sh[B->ats.v[i].addr], B->ats.v[i].val); B->ats.n = 0;\n"
        "  for (uint64_t i = 0; i < B->sst.n; ++i) B->sh[B->sst.v[i].addr] = B->sst.v[i].val;\n"),
    "max_pc_reconvergence": (
        "if (B->st[t] == ST_RUN && B->pc[t] < p) p = B->pc[t];",
        "if (B->st[t] == ST_RUN && (p == UINT32_MAX || B->pc[t] > p)) p = B->pc[t];"),
    "largest_pair_reported": (
        "if (lo < t1 || (lo == t1 && hi < t2))", "if (t1 == UINT32_MAX || lo > t1 || (lo == t1 && hi > t2))"),
    "floor_division": (
        "return va / vb;                          /* C99: truncation toward zero */",
        "return (va % vb && ((va < 0) != (vb < 0))) ? va / vb - 1 : va / vb;"),
    "no_abort_after_deadlock": ("if (st & (ORC_ST_DEADLOCK | ORC_ST_STEP_LIMIT)) dead[l] = 1;", ""),
    "event_wait_ignored": ("dep_wait[l] = P->launches[l].wait ? (int32_t)P->launches[l].wait - 1 : -1;",
                           "dep_wait[l] = -1;"),
    "streams_ignored": ("if (P->launches[m].stream == P->launches[l].stream) { dep_prev[l] = (int32_t)m; break; }",
                        "{ dep_prev[l] = (int32_t)m; break; }"),
    "skip_not_propagated": ("dead[l] = 1;                                            /* skipped */", ""),
    "divergence_unchecked": ("if (pmin != pmax)        /* all threads wait", "if (0)        /* all threads wait"),
    "logical_right_shift": ("return va < 0 ? ~((~va) >> s) : (va >> s);", "return as_i32((uint32_t)va >> s);"),
    "pc_range_not_recorded": ("if (p->pc < pclo) pclo = p->pc;\n      if (p->pc > pchi) pchi = p->pc;", ""),
    "shared_bound_off_by_one": (
        "if (addr < 0 || (uint32_t)addr >= B->shw) { note_err(B, pc, t); break; }",
        "if (addr < 0 || (uint32_t)addr >= B->shw + 1) { note_err(B, pc, t); break; }"),
    "count_barrier_over_last_warp_only": (
        "for (uint32_t t = 0; t < B->n; ++t) if (B->st[t] == ST_WAIT && B->bp[t]) ++nP;",
        "for (uint32_t t = (B->n - 1) / 32 * 32; t < B->n; ++t) if (B->st[t] == ST_WAIT && B->bp[t]) ++nP;"),
    "and_barrier_is_or": ("if (B->bk[t] == 1) reg_write(B, t, B->bd[t], nP == nW);",
                          "if (B->bk[t] == 1) reg_write(B, t, B->bd[t], nP > 0);"),
    "plain_barrier_counts_as_true": ("B->bp[t] = base != ORC_BAR && va != 0;",
                                     "B->bp[t] = base == ORC_BAR || va != 0;"),
    "written_marked_at_issue": ("if (!B->deferred) B->written[addr] = 1;", "B->written[addr] = 1;"),
    "atomics_do_not_initialise": ("  for (uint64_t i = 0; i < B->ats.n; ++i) B->written[B->ats.v[i].addr] = 1;\n", ""),
    "interblock_counter_never_increments": ("res->interblock_conflicts++;", ";"),
    "interblock_same_block_conflicts": ("if (cur == me || cur == -2) return;", "if (cur == -2) return;"),
    "global_block_pairs_include_same_block": ("if (p->block == q->block) continue;", ""),
    "global_block_pair_largest": (
        "if (lo < b1 || (lo == b1 && hi < b2)) { b1 = lo; b2 = hi; }",
        "if (b1 == UINT32_MAX || lo > b1 || (lo == b1 && hi > b2)) { b1 = lo; b2 = hi; }"),
    "launch_order_ignored": (
        "if (before[(size_t)l * nl + m]) continue;   /* ordered: m completes before l starts */", ""),
    "launch_reads_dropped": ("if (rd) lacc_push(&prog_acc, (laccess_t){la.v[k].addr, l, K_R});", ""),
    "global_loads_not_checked": (
        "acc_push(&B->gacc, (access_t){(uint32_t)addr, t, is_write ? K_W : K_R, pc});",
        "if (is_write) acc_push(&B->gacc, (access_t){(uint32_t)addr, t, K_W, pc});"),
    "global_interval_check_skipped": (
        "if (B->gacc.n) interval_races(B, &B->gacc, ORC_REP_GLOBAL_RACE);", ""),
    "warps_of_16": (
        "uint32_t lo = 32 * w, hi = lo + 32 < B->n ? lo + 32 : B->n;",
        "uint32_t lo = 16 * w, hi = lo + 16 < B->n ? lo + 16 : B->n; if (lo >= B->n) continue;"),
}


@pytest.fixture(scope="module")
def workspace(tmp_path_factory):
    d = tmp_path_factory.mktemp("mutants")
    for sub in ("oracle", "tests", "paper_1211_6193_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("_build", "_lib", "__pycache__", "csrc"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    return str(d)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_oracle_mistake(workspace, name):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert before in src, "mutation anchor no longer present in the oracle source"
    mutated = src.replace(before, after)
    if name == "warps_of_16":
        mutated = mutated.replace("B.nwarps = (L->block_dim + 31) / 32;", "B.nwarps = (L->block_dim + 15) / 16;")
    open(os.path.join(workspace, "oracle", "simt_oracle.c"), "w").write(mutated)
    shutil.rmtree(os.path.join(workspace, "oracle", "_build"), ignore_errors=True)
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "tests/test_oracle_pins.py", "tests/test_oracle_global.py"], cwd=workspace,
                           capture_output=True, text=True,
                           timeout=120)
        caught = r.returncode != 0
    except subprocess.TimeoutExpired:
        caught = True
    assert caught, f"the pins did not notice mutation {name}"
