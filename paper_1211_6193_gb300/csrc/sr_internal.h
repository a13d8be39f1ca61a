// sr_internal.h - device-side data layout shared by the kernels and the host runtime of
// libsimtcheck.  Nothing here is part of the public C ABI (include/simtcheck.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "simtcheck.h"

namespace sr {

// Packed instructions (device copy), x word: op:6 | immediate operand:1 | d:5 | a:5 | b:5 |
// run:10, y word: the immediate.  Register fields are rows of the program's compacted
// register file (only the registers the program uses, plus one zero row last); a destination
// of kNoDest drops the write (RZ or an opcode without a result).  `run` is the number of
// consecutive MOV, ADD and MUL instructions starting at this one, at most kRunMax, 0 for any
// other instruction: such a run touches no memory and needs no ALU dispatch (the interpreter's
// tight loop selects among the three; every other operation takes the general path).
constexpr uint32_t kNoDest = 31;
constexpr uint32_t kRunMax = 1023;
__host__ __device__ constexpr uint32_t pk_op(uint32_t x) { return x & 0x3Fu; }
__host__ __device__ constexpr uint32_t pk_imm(uint32_t x) { return (x >> 6) & 1u; }
__host__ __device__ constexpr uint32_t pk_d(uint32_t x) { return (x >> 7) & 31u; }
__host__ __device__ constexpr uint32_t pk_a(uint32_t x) { return (x >> 12) & 31u; }
__host__ __device__ constexpr uint32_t pk_b(uint32_t x) { return (x >> 17) & 31u; }
__host__ __device__ constexpr uint32_t pk_run(uint32_t x) { return x >> 22; }
__host__ __device__ constexpr uint32_t pk_make(uint32_t op, uint32_t imm, uint32_t d, uint32_t a, uint32_t b,
                                               uint32_t run) {
  return op | imm << 6 | d << 7 | a << 12 | b << 17 | run << 22;
}
__host__ __device__ constexpr bool pk_plain_alu(uint32_t op) {
  return op == SR_OP_MOV || op == SR_OP_ADD || op == SR_OP_MUL;
}
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kMaxBudget = 1u << 26;  // epochs and rounds stay below 2^26
// Polls of an mbarrier that only a CTA's own bulk copy (global -> its shared memory) completes.
// No other agent is involved, so this bound does not follow the caller's spin_limit: a copy that
// has not landed after this many polls is waited for once more, with the same bound, before the
// CTA returns or reuses the buffer, so that no copy is left writing shared memory.
constexpr uint32_t kCopyWaitLimit = 1u << 24;

// Debug build (-DSR_DEBUG_BOUNDS): internal indices are checked before each access; a failed
// check sets `flag_bits` in *flag and the access is skipped (no trap, no fault: the kernel
// goes on and the host reports the failure).  In the default build the check is compiled away.
#if defined(SR_DEBUG_BOUNDS) && defined(__CUDACC__)
__device__ __forceinline__ bool dbg_ok(bool ok, uint32_t* flag, uint32_t flag_bits) {
  if (!ok) atomicOr(flag, flag_bits);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool dbg_ok(bool, uint32_t*, uint32_t) { return true; }
#endif
constexpr uint32_t kErrTimeout = 1, kErrCorrupt = 2, kErrBounds = 4;   // batch error word bits

// thread status of a simulated thread
enum : uint32_t { ST_RUN = 0, ST_WAIT = 1, ST_EXIT = 2, ST_NONE = 3 };
// access kinds inside a log record
enum : uint32_t { K_R = 0, K_W = 1, K_A = 2 };
// per-block flags
enum : uint32_t { BF_OVERFLOW = 1, BF_INTERNAL = 2 };

// Access-log record (8 bytes):
//   bits 63..38 epoch (26) | 37..24 word address (14) | 23..14 tid (10) | 13..12 kind | 11..0 pc
// The high 40 bits (epoch, address) are the sort key of the race check.
__host__ __device__ constexpr uint64_t make_record(uint32_t epoch, uint32_t addr, uint32_t tid,
                                                   uint32_t kind, uint32_t pc) {
  return (uint64_t)epoch << 38 | (uint64_t)addr << 24 | (uint64_t)(tid << 14 | kind << 12 | pc);
}
__host__ __device__ constexpr uint32_t rec_epoch(uint64_t r) { return (uint32_t)(r >> 38); }
__host__ __device__ constexpr uint32_t rec_addr(uint64_t r) { return (uint32_t)(r >> 24) & 0x3FFFu; }
__host__ __device__ constexpr uint32_t rec_tid(uint64_t r) { return (uint32_t)(r >> 14) & 0x3FFu; }
__host__ __device__ constexpr uint32_t rec_kind(uint64_t r) { return (uint32_t)(r >> 12) & 3u; }
__host__ __device__ constexpr uint32_t rec_pc(uint64_t r) { return (uint32_t)r & 0xFFFu; }

// One (program, launch) pair, in canonical order.
struct LaunchDev {
  uint32_t prog, launch, entry, ncode;   // ncode without the EXIT sentinel
  uint32_t code_off, grid, bdim, shw;    // code_off in instructions (even)
  int32_t params[4];
  uint32_t nparams, block_base, log_cap, key_bits;   // log_cap records per block (even)
  uint64_t log_base;                     // record offset of block 0's region
  uint64_t arena_off, arena_words;       // word offset of the program's working arena
  uint32_t groups, group_bytes;          // batched mode: blocks per CTA, smem per block
  uint32_t ir_bytes, nrows;              // smem bytes of the staged code; register rows (zero row last)
  uint32_t check_group, check_item;      // race check: blocks per work item, index of the first item
  uint32_t uninit;                       // 1 = report shared loads of words no thread wrote
  uint32_t fused;                        // 1 = race summaries kept by the interpreter (no log)
  // the launches (batch indices) this one follows: the previous launch of its stream and the
  // one it waits for (kNoDep: none), and its own batch index
  uint32_t dep_prev, dep_wait, index;
  // global-memory race check: global-log records per block (0 = off), the record offset of
  // block 0's region; the program's first launch (batch index) and launch count, and the word
  // offset of its launch-order bit matrix (kNoDep: every pair of its launches is ordered)
  uint32_t glog_cap, first_launch, nl_prog, ord_off;
  uint64_t glog_base;
  // the blocks run are [block_off, block_off + grid) of a grid of gdim blocks (S2R BID and
  // reports add block_off; S2R GDIM reads gdim)
  uint32_t block_off, gdim;
  // batched mode: blocks per work item, a multiple of `groups` (a group that finishes its block
  // claims the item's next one)
  uint32_t item_blocks;
};
constexpr uint32_t kNoDep = 0xFFFFFFFFu;

// Per simulated block, written by the interpreter (n_log, n_misc, flags) and the checker (n_race).
struct BlockRes { uint32_t n_log, n_race, n_misc, flags; };

struct Counters {
  unsigned long long thread_instrs, global_accesses, total_reports, shared_accesses;
  unsigned long long global_records;   // global-log records (global-memory race check)
};

struct RunArgs {
  const LaunchDev* launches;
  uint32_t nlaunches;
  uint32_t budget, check_races, spin_limit;
  const uint2* code;            // packed instructions of all programs
  int32_t* arena;               // working arenas of all programs
  unsigned long long* log;      // access-log pool
  BlockRes* blocks;
  uint32_t* prog_status;        // SR_ST_* bits
  uint32_t* launch_dead;        // per launch: 1 = a block stopped it, or it was skipped
  Counters* counters;
  // batched mode
  const uint2* items;           // (launch index, first block)
  uint32_t nitems;
  uint32_t* queue_head;
  uint32_t* launch_done;        // completed blocks per launch
  // global-memory race check: per-block global-log regions and per-block record counts
  uint4* glog;
  uint32_t* glog_n;
  // batched mode, two CTAs per SM: the wave's block queue of the one-block-per-CTA kernel -
  // its launches in ticket order and the first ticket of each (bq_first[0] = 0), and the
  // ticket counter
  const uint32_t* bq_launch;
  const uint32_t* bq_first;
  uint32_t bq_n;
  uint32_t* bq_head;
};

// Shared-memory footprint of one simulated block in the interpreter.
struct GroupLayout {
  uint32_t regs, sh, clk, rlo, rhi, rsp, park, err, bv, un, wb, tup, rbm, total;
};
// The summary of one shared word in the fused race check: the two smallest distinct tids of
// each access kind (kTupleEmpty none) and the lowest and highest pc, eight planes of this
// many words each, so that the lanes of a warp on consecutive words touch consecutive banks.
constexpr uint32_t kTupleEmpty = 0xFFFFFFFFu;
__host__ __device__ inline uint32_t tuple_plane_words(uint32_t shw) { return (shw + 31u) & ~31u; }
__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }
// The fixed-size arrays come first, at offsets known at compile time; the arrays whose
// size depends on the launch follow.
constexpr uint32_t kGroupClk = 0, kGroupRlo = 128, kGroupRhi = 256, kGroupRsp = 384, kGroupPark = 512,
                   kGroupBv = 512 + 32 * 8 * 4, kGroupFixed = kGroupBv + 64;
// With `uninit`: per-pc counters of loads of unwritten words, and the bitmap of written words.
// With `fused`: the eight summary planes and a bitmap of the interval's racy words.
__host__ __device__ inline GroupLayout group_layout(uint32_t nthr, uint32_t shw, uint32_t ncode, uint32_t nrows,
                                                   uint32_t uninit, uint32_t fused) {
  GroupLayout g;
  g.clk = kGroupClk;
  g.rlo = kGroupRlo;
  g.rhi = kGroupRhi;
  g.rsp = kGroupRsp;
  g.park = kGroupPark;
  g.bv = kGroupBv;
  uint32_t o = kGroupFixed;
  g.regs = o; o += align16(nrows * nthr * 4u);
  g.sh = o;   o += align16(shw * 4u);
  g.err = o;  o += align16(2u * (ncode + 1) * 4u);
  g.un = g.wb = 0;
  if (uninit) {
    g.un = o; o += align16(2u * (ncode + 1) * 4u);
    g.wb = o; o += align16((shw + 31u) / 32u * 4u);
  }
  g.tup = g.rbm = 0;
  if (fused) {
    g.tup = o;     o += 32u * tuple_plane_words(shw);
    g.rbm = o;     o += align16(tuple_plane_words(shw) / 8u);
  }
  g.total = o;
  return g;
}
__host__ __device__ inline uint32_t ir_smem_bytes(uint32_t ncode) {
  return align16(((ncode + 2u) & ~1u) * 8u);   // ncode + EXIT sentinel, even count
}

// kernel launchers (defined in the .cu files); attributes are set once per process
cudaError_t init_kernel_attributes(uint32_t smem_optin);
cudaError_t init_interp_attributes(uint32_t smem_optin);
cudaError_t init_check_attributes(uint32_t smem_optin);
cudaError_t launch_interp_plain(const RunArgs& a, uint32_t li, const LaunchDev& L, uint32_t variant, cudaStream_t s);
// fused: run the instantiation with the fused race check (launches whose `fused` is 0 still
// log their accesses in it); global: the instantiation that logs global accesses (launches
// whose glog_cap is 0 log none in it; it has no fused race check)
cudaError_t launch_interp_batched(const RunArgs& a, uint32_t ctas, uint32_t smem, bool fused, bool global,
                                  cudaStream_t s);
// batched mode, two CTAs per SM: one simulated block per 1024-thread CTA for the wave's block
// queue (a.bq_*), `nblocks` CTAs, `smem` bytes of dynamic shared memory each
cudaError_t launch_interp_blocks(const RunArgs& a, uint32_t nblocks, uint32_t smem, cudaStream_t s);
// dynamic shared memory of one CTA of the one-block-per-CTA kernel that still lets two share an SM
uint32_t interp_blocks_smem_cap(uint32_t smem_optin);

// Global-log record (16 bytes): x = word address in the program's arena, y = epoch (barrier
// interval of the block), z = tid << 16 | kind << 12 | pc (kind 1 = store, 0 = load),
// w = global block index in the batch.  A block's records are in epoch order.
__host__ __device__ inline uint32_t grec_tid(const uint4& r) { return r.z >> 16; }
__host__ __device__ inline uint32_t grec_write(const uint4& r) { return (r.z >> 12) & 1u; }
__host__ __device__ inline uint32_t grec_pc(const uint4& r) { return r.z & 0xFFFu; }
uint32_t interp_plain_smem(const LaunchDev& L);

struct CheckArgs {
  const LaunchDev* launches;
  uint32_t li0, li1;            // launch range of the wave
  uint32_t item0, item1;        // work items of the wave (launch li owns items from check_item on)
  unsigned long long* log;
  BlockRes* blocks;
  uint4* scratch;               // per checker CTA: kScratchWords race entries (intervals with many races)
  uint32_t* work_head;
  uint32_t* error_flag;
  uint32_t spin_limit;
  uint32_t table_words;         // address-table entries: >= every shw of the wave, multiple of 32
  const uint32_t* item_launch;  // launch index of every work item (NULL: found by binary search)
};
// race-check kernel shapes (variant 1..SR_CHECK_VARIANTS; 0 = default)
uint32_t check_default_variant();
uint32_t check_ctas_per_sm(uint32_t variant);
uint32_t check_table_cap(uint32_t variant);
cudaError_t launch_check(const CheckArgs& a, uint32_t variant, uint32_t ctas, cudaStream_t s);
constexpr uint32_t kCheckBins = 12288;         // the largest shared array (words)
constexpr uint32_t kCheckTableCap = 4096;      // shared-memory address table entries at most (per variant)
// per checker CTA in global memory: race entries of an interval staged while its summaries
// take several rounds (at most kCheckBins), then the spill table (kCheckBins words) for the
// intervals that touch words past the shared-memory table
constexpr uint32_t kScratchWords = 1u << 14;
static_assert(kScratchWords >= kCheckBins + kCheckBins / 4, "spill table must fit behind the staged entries");
constexpr uint32_t kCheckItemRecords = 8192;   // log records a check work item aims at
constexpr uint32_t kCheckMaxGroup = 32;        // blocks per check work item at most

// address-table entries for a wave's race check: one per word of its largest shared array,
// and room for the exact summaries (4 entries each) of every word in one round, at most
// `cap` (the kernel shape's), so that small tables keep more CTAs on an SM.  Intervals
// touching words past the table are checked in the CTA's spill table instead.
inline uint32_t check_table_words(const LaunchDev* L, uint32_t li0, uint32_t li1, uint32_t cap) {
  uint32_t m = 8;
  for (uint32_t i = li0; i < li1; ++i) m = L[i].shw > m ? L[i].shw : m;
  m = (4u * m + 31u) & ~31u;
  return m < cap ? m : cap;
}

// blocks per check work item for a launch whose blocks log at most `log_cap` records
__host__ __device__ inline uint32_t check_group_for(uint32_t log_cap) {
  const uint32_t g = (kCheckItemRecords + log_cap - 1) / (log_cap ? log_cap : 1);
  return g < 1 ? 1 : (g > kCheckMaxGroup ? kCheckMaxGroup : g);
}

// Global-memory race check of one wave (gcheck.cu).  Device buffers, all owned by the batch.
struct GcheckArgs {
  const LaunchDev* launches;
  uint32_t li0, li1, gb0, gb1;      // the wave's launches and global blocks
  const uint4* glog;                // per-block regions (LaunchDev::glog_base, glog_cap)
  const uint32_t* glog_n;           // records per global block
  unsigned long long* goff;         // per block of the wave: first record in sort_a
  unsigned long long* gtotal;       // records of the wave
  unsigned long long* partials;     // scan scratch (gcheck_partials)
  uint4* sort_a;                    // rec_cap records each
  uint4* sort_b;
  unsigned long long rec_cap;       // >= the wave's records
  uint32_t addr_passes;             // 8-bit digits of the largest word address of the wave
  unsigned long long* hist;         // 12 x 256 digit counts
  unsigned long long* status;       // gcheck_tiles(max(rec_cap, entry_cap)) x 256 tile states
  uint32_t* tile_ctr;               // 12 tile counters
  uint32_t* err;                    // set when a bounded wait gave up
  uint32_t spin_limit;
  uint32_t sms;
  const uint32_t* ord_bits;         // launch-order matrices of programs with unordered launches
  uint4* entries_a;                 // report entries, 32 bytes each (entry_cap)
  uint4* entries_b;
  unsigned long long entry_cap;
  unsigned long long* gn;           // entries produced in this wave (may exceed entry_cap)
  uint32_t* gcount;                 // per global block: its entries
  unsigned long long* gstart;       // per block of the wave: its first entry in entries_a
  unsigned long long* gn_sorted;    // scratch total
};
cudaError_t init_gcheck_attributes(uint32_t smem_optin);
cudaError_t launch_gcheck(const GcheckArgs& g, uint32_t& kernels, cudaStream_t s);
uint64_t gcheck_tiles(uint64_t records);
uint64_t gcheck_partials(uint32_t nblocks);

struct CompactArgs {
  const LaunchDev* launches;
  uint32_t nlaunches;
  uint32_t gb0, gb1;            // block range of the wave
  unsigned long long* total;    // running report count over waves
  const unsigned long long* log;
  const BlockRes* blocks;
  unsigned long long* offsets;  // nblocks + 1
  unsigned long long* partials; // scan scratch
  sr_report* out;
  unsigned long long out_cap;
  Counters* counters;
  // global-memory race check (NULL when off): per global block its entries, per block of
  // the wave its first entry, and the entries in (block, epoch, kind, word) order
  const uint32_t* gcount;
  const unsigned long long* gstart;
  const uint4* gentries;
  unsigned long long gcap;      // entries the buffer holds (a wave that produced more is run again)
  uint32_t* error_flag;         // debug build: kErrBounds
};
cudaError_t launch_compact_scan(const CompactArgs& a, cudaStream_t s);
cudaError_t launch_compact_emit(const CompactArgs& a, cudaStream_t s);
uint64_t compact_partials_count(uint32_t nblocks);
uint32_t compact_kernels(const CompactArgs& a);   // kernel launches of launch_compact_scan + _emit

}  // namespace sr
