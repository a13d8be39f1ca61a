// host_prep.h - host-side preparation of simulated programs shared by the entry points of
// libsimtcheck: validation, register renaming, instruction packing and the static bound
// of a kernel's per-block access log.  Internal; not part of the C ABI.
#pragma once
#include <algorithm>
#include <cstdio>
#include <vector>
#include <cuda_runtime.h>
#include <stdint.h>

#include "simtcheck.h"
#include "sr_internal.h"

namespace sr {
namespace host {

// barriers: __syncthreads and its reducing forms _and / _or / _count
inline bool is_barrier(uint32_t b) { return b == SR_OP_BAR || (b >= SR_OP_BARAND && b <= SR_OP_BARPOPC); }
inline bool is_reducing_barrier(uint32_t b) { return b >= SR_OP_BARAND && b <= SR_OP_BARPOPC; }

// which operand fields an opcode reads or writes
inline bool op_writes_d(uint32_t b) {
  return (b >= SR_OP_MOV && b <= SR_OP_SNE) || b == SR_OP_S2R || b == SR_OP_LDG || b == SR_OP_LDS ||
         is_reducing_barrier(b);
}
inline bool op_reads_a(uint32_t b) {
  return (b >= SR_OP_ADD && b <= SR_OP_SNE) || b == SR_OP_LDG || b == SR_OP_STG || b == SR_OP_LDS ||
         b == SR_OP_STS || b == SR_OP_ATOMS || b == SR_OP_BRZ || b == SR_OP_BRNZ || is_reducing_barrier(b);
}
inline bool op_reads_b(uint32_t op) {
  const uint32_t b = op & 0x7Fu;
  return ((b >= SR_OP_MOV && b <= SR_OP_SNE) && !(op & SR_BIMM)) || b == SR_OP_STG || b == SR_OP_STS ||
         b == SR_OP_ATOMS;
}
inline bool is_shared_access(uint32_t b) { return b == SR_OP_LDS || b == SR_OP_STS || b == SR_OP_ATOMS; }
inline bool can_err(uint32_t b) {
  return b == SR_OP_LDS || b == SR_OP_STS || b == SR_OP_ATOMS || b == SR_OP_LDG || b == SR_OP_STG ||
         b == SR_OP_DIV || b == SR_OP_REM;
}

// Static bound for one kernel: the largest number of shared accesses and barriers a
// single thread can execute, or "unbounded" if the control-flow graph from the entry
// has a cycle.
struct KernelBound {
  bool cyclic = false;
  uint32_t accesses = 0, barriers = 0, err_pcs = 0;
  uint32_t gaccesses = 0;   // global loads and stores on the longest such path
};
// Workspace of bound_kernel: 5 arrays of ncode + 1 entries (callers own the memory).
struct BoundScratch {
  uint8_t* colour;
  uint32_t* acc;
  uint32_t* bar;
  uint32_t* stack_pc;
  uint32_t* stack_next;
  uint32_t* gacc;
};
inline KernelBound bound_kernel(const sr_instr* code, uint32_t ncode, uint32_t entry, const BoundScratch& w) {
  KernelBound kb;
  // iterative DFS with colours; longest paths by memoised post-order
  for (uint32_t i = 0; i <= ncode; ++i) { w.colour[i] = 0; w.acc[i] = 0; w.bar[i] = 0; w.gacc[i] = 0; }
  uint32_t depth = 0;
  auto succ = [&](uint32_t pc, uint32_t i, uint32_t& out) -> bool {
    if (pc >= ncode) return false;
    const uint32_t b = code[pc].op_d_a_b & 0x7Fu;
    const uint32_t t = (uint32_t)code[pc].imm;
    if (b == SR_OP_EXIT) return false;
    if (b == SR_OP_BRA) { if (i == 0) { out = t; return true; } return false; }
    if (b == SR_OP_BRZ || b == SR_OP_BRNZ) {
      if (i == 0) { out = pc + 1; return true; }
      if (i == 1) { out = t; return true; }
      return false;
    }
    if (i == 0) { out = pc + 1; return true; }
    return false;
  };
  w.stack_pc[depth] = entry;
  w.stack_next[depth] = 0;
  ++depth;
  w.colour[entry] = 1;
  while (depth) {
    const uint32_t top = depth - 1;
    uint32_t nxt;
    if (succ(w.stack_pc[top], w.stack_next[top], nxt)) {
      w.stack_next[top]++;
      if (w.colour[nxt] == 1) { kb.cyclic = true; return kb; }
      if (w.colour[nxt] == 0) {
        w.colour[nxt] = 1;
        w.stack_pc[depth] = nxt;
        w.stack_next[depth] = 0;
        ++depth;
      }
      continue;
    }
    const uint32_t pc = w.stack_pc[top];
    uint32_t a = 0, br = 0, g = 0, s;
    for (uint32_t i = 0; succ(pc, i, s); ++i) {
      a = a > w.acc[s] ? a : w.acc[s];
      br = br > w.bar[s] ? br : w.bar[s];
      g = g > w.gacc[s] ? g : w.gacc[s];
    }
    if (pc < ncode) {
      const uint32_t b = code[pc].op_d_a_b & 0x7Fu;
      a += is_shared_access(b);
      br += is_barrier(b);
      g += (b == SR_OP_LDG || b == SR_OP_STG);
      kb.err_pcs += can_err(b);
    }
    w.acc[pc] = a;
    w.bar[pc] = br;
    w.gacc[pc] = g;
    w.colour[pc] = 2;
    --depth;
  }
  kb.accesses = w.acc[entry];
  kb.barriers = w.bar[entry];
  kb.gaccesses = w.gacc[entry];
  return kb;
}

inline int validate(const sr_program* p, char* msg, size_t len) {
  auto bad = [&](const char* fmt, uint32_t x, uint32_t y) {
    if (msg && len) snprintf(msg, len, fmt, x, y);
    return SR_E_INVAL;
  };
  if (!p || !p->code || p->ncode == 0 || p->ncode > SR_MAX_CODE) return bad("code size %u outside 1..%u", p ? p->ncode : 0, SR_MAX_CODE);
  if (!p->kernel_entry || p->nkernels == 0) return bad("no kernels (%u, %u)", 0, 0);
  for (uint32_t k = 0; k < p->nkernels; ++k)
    if (p->kernel_entry[k] >= p->ncode) return bad("kernel %u entry %u out of range", k, p->kernel_entry[k]);
  for (uint32_t pc = 0; pc < p->ncode; ++pc) {
    const uint32_t w = p->code[pc].op_d_a_b, op = w & 0xFFu, b = op & 0x7Fu;
    const uint32_t d = (w >> 8) & 0xFFu, ra = (w >> 16) & 0xFFu, rb = (w >> 24) & 0xFFu;
    const int32_t imm = p->code[pc].imm;
    const bool alu = b >= SR_OP_MOV && b <= SR_OP_SNE;
    if (b < SR_OP_MOV || b > SR_OP_BARPOPC || (op & 0x40u) || ((op & SR_BIMM) && !alu))
      return bad("pc %u: bad opcode 0x%x", pc, op);
    auto reg_ok = [](uint32_t r) { return r < 16 || r == SR_RZ; };
    if ((op_writes_d(b) && !reg_ok(d)) || (op_reads_a(b) && !reg_ok(ra)) || (op_reads_b(op) && !reg_ok(rb)))
      return bad("pc %u: bad register field (op %u)", pc, b);
    if ((b == SR_OP_BRA || b == SR_OP_BRZ || b == SR_OP_BRNZ) && (imm < 0 || (uint32_t)imm > p->ncode))
      return bad("pc %u: branch target %u out of range", pc, (uint32_t)imm);
    if (b == SR_OP_S2R && (imm < 0 || imm > SR_SREG_WARPSIZE)) return bad("pc %u: bad special register %u", pc, (uint32_t)imm);
  }
  if (p->nlaunches && !p->launches) return bad("launch table missing (%u launches)", p->nlaunches, 0);
  for (uint32_t l = 0; l < p->nlaunches; ++l) {
    const sr_launch& L = p->launches[l];
    if (L.kernel >= p->nkernels) return bad("launch %u: kernel %u out of range", l, L.kernel);
    if (L.grid == 0 || L.grid > (1u << 30)) return bad("launch %u: grid %u", l, L.grid);
    if (L.block_dim == 0 || L.block_dim > SR_MAX_BLOCK_DIM) return bad("launch %u: block_dim %u", l, L.block_dim);
    if (L.shmem_words > SR_MAX_SHMEM_WORDS) return bad("launch %u: shmem_words %u", l, L.shmem_words);
    if (L.nparams > 4) return bad("launch %u: nparams %u", l, L.nparams);
    if (L.wait > l) return bad("launch %u: waits for launch %u, which is not an earlier one", l, L.wait - 1);
    if ((L.block_count == 0 && L.block_begin != 0) || (uint64_t)L.block_begin + L.block_count > L.grid)
      return bad("launch %u: block range starting at %u outside the grid", l, L.block_begin);
  }
  if (p->global_words >= (1ull << 31)) return bad("global arena too large (%u)", (uint32_t)(p->global_words >> 20), 0);
  if (p->global_words && !p->global_init) return bad("global_init missing (%u words)", (uint32_t)p->global_words, 0);
  return SR_OK;
}

// Register renaming of one program: the registers it touches (plus the parameter
// registers r0..r(maxp-1)) become rows 0..n-1 in ascending order, the zero row is n.
struct RegMap {
  uint8_t row[256];
  uint32_t nrows;
};
inline RegMap map_registers(const sr_program& P) {
  bool used[16] = {};
  uint32_t maxp = 0;
  for (uint32_t l = 0; l < P.nlaunches; ++l) maxp = std::max(maxp, P.launches[l].nparams);
  for (uint32_t r = 0; r < maxp; ++r) used[r] = true;
  for (uint32_t pc = 0; pc < P.ncode; ++pc) {
    const uint32_t w = P.code[pc].op_d_a_b, op = w & 0xFFu, b = op & 0x7Fu;
    const uint32_t d = (w >> 8) & 0xFFu, ra = (w >> 16) & 0xFFu, rb = (w >> 24) & 0xFFu;
    if (op_writes_d(b) && d < 16) used[d] = true;
    if (op_reads_a(b) && ra < 16) used[ra] = true;
    if (op_reads_b(op) && rb < 16) used[rb] = true;
  }
  RegMap m;
  uint32_t n = 0;
  for (uint32_t r = 0; r < 16; ++r) m.row[r] = used[r] ? (uint8_t)n++ : 0;
  m.nrows = n + 1;
  return m;
}

// pack one instruction: sources that are RZ or unused read the zero row; destinations
// that are RZ or absent become kNoDest
inline uint2 pack(const sr_instr& in, const RegMap& m) {
  const uint32_t w = in.op_d_a_b, op = w & 0xFFu, b = op & 0x7Fu;
  uint32_t d = (w >> 8) & 0xFFu, ra = (w >> 16) & 0xFFu, rb = (w >> 24) & 0xFFu;
  const uint32_t zrow = m.nrows - 1;
  d = (op_writes_d(b) && d != SR_RZ) ? m.row[d] : sr::kNoDest;
  ra = (op_reads_a(b) && ra != SR_RZ) ? m.row[ra] : zrow;
  rb = (op_reads_b(op) && rb != SR_RZ) ? m.row[rb] : zrow;
  return make_uint2(sr::pk_make(b, (op & SR_BIMM) ? 1u : 0u, d, ra, rb, 0), (uint32_t)in.imm);
}

// The EXIT sentinel after a program's last instruction (running past the end exits).
inline uint2 exit_sentinel(const RegMap& m) {
  return make_uint2(sr::pk_make(SR_OP_EXIT, 0, sr::kNoDest, m.nrows - 1, m.nrows - 1, 0), 0);
}

// Fill in the run lengths of n packed instructions (straight-line successors only: a run
// never contains a branch, so it is valid from any entry pc).
inline void set_run_lengths(uint2* code, uint32_t n) {
  uint32_t next = 0;
  for (uint32_t pc = n; pc-- > 0;) {
    const uint32_t run = sr::pk_plain_alu(sr::pk_op(code[pc].x)) ? std::min(sr::kRunMax, 1 + next) : 0u;
    code[pc].x = (code[pc].x & ((1u << 22) - 1)) | run << 22;
    next = run;
  }
}

inline uint32_t key_bits_for(uint32_t shw) {
  uint32_t b = 1;
  while ((1u << b) < shw) ++b;
  return b;
}


// The launches (indices within the program, or `none`) that launch l follows: the previous
// launch of its stream and the launch it waits for (Sec. 3, streams and events).
inline void launch_deps(const sr_launch* launches, uint32_t l, uint32_t none, uint32_t& prev, uint32_t& wait) {
  prev = none;
  for (uint32_t m = l; m-- > 0;)
    if (launches[m].stream == launches[l].stream) {
      prev = m;
      break;
    }
  wait = launches[l].wait ? launches[l].wait - 1 : none;
}

// Access-log region (records per block, even) of one launch: the static bound of its
// kernel, or `loop_records` for kernels with loops, plus room for barrier/error records.
inline uint64_t launch_log_cap(const KernelBound& k, uint32_t block_dim, uint32_t check_races, uint32_t loop_records) {
  uint64_t recs, misc;
  if (k.cyclic) {
    recs = loop_records;
    misc = 4ull * (1 + k.err_pcs) > 256 ? 4ull * (1 + k.err_pcs) : 256;
  } else {
    recs = (uint64_t)k.accesses * block_dim;
    misc = (uint64_t)(k.barriers + 1) * (1 + k.err_pcs) + 1;
  }
  if (!check_races) recs = 0;
  return (recs + 2 * misc + 1) & ~1ull;
}

// Global-log region (records per block, even) of one launch for the global-memory race
// check: the kernel's static bound of global loads and stores per thread, or `loop_records`
// for kernels with loops.
inline uint64_t launch_glog_cap(const KernelBound& k, uint32_t block_dim, uint32_t loop_records) {
  const uint64_t recs = k.cyclic ? (uint64_t)loop_records : (uint64_t)k.gaccesses * block_dim;
  return (recs + 1) & ~1ull;
}

// Launch-order bit matrix of one program (Sec. 3, streams and events): bit l * nl + m is set
// when launch m precedes launch l through stream order and event waits, transitively.
// Returns false (nothing written) when every pair of launches is ordered.
inline bool launch_order_bits(const sr_launch* launches, uint32_t nl, std::vector<uint32_t>& bits) {
  std::vector<uint8_t> before((size_t)nl * nl, 0);
  for (uint32_t l = 0; l < nl; ++l) {
    uint32_t prev, wait;
    launch_deps(launches, l, UINT32_MAX, prev, wait);
    for (uint32_t d : {prev, wait}) {
      if (d == UINT32_MAX) continue;
      before[(size_t)l * nl + d] = 1;
      for (uint32_t m = 0; m < nl; ++m)
        if (before[(size_t)d * nl + m]) before[(size_t)l * nl + m] = 1;
    }
  }
  bool all = true;
  for (uint32_t l = 0; l < nl && all; ++l)
    for (uint32_t m = 0; m < l; ++m)
      if (!before[(size_t)l * nl + m]) { all = false; break; }
  if (all) return false;
  bits.assign(((size_t)nl * nl + 31) / 32, 0u);
  for (size_t i = 0; i < (size_t)nl * nl; ++i)
    if (before[i]) bits[i / 32] |= 1u << (i % 32);
  return true;
}

}  // namespace host
}  // namespace sr
