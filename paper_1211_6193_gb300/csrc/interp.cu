// interp.cu - the SIMT interpreter: one real warp per simulated warp.
//
// What it computes (Hathhorn et al., SSV 2012): every thread of every block runs the
// kernel (Sec. 3 "Threads and memory"), blocks own a dynamic shared array (same
// section), __syncthreads() is a block-wide barrier (Sec. 3 "Barrier synchronization"),
// and every shared access is hooked (Sec. 3 "Modularity": the read/write check hook)
// - here the hook appends an 8-byte record to the block's access log for the race
// check of check.cu.  At each barrier the block's waiting threads are examined for
// divergence and deadlock (Sec. 3.1, last paragraph).
//
// GPU design.  A simulated block of B threads runs on ceil(B/32) real warps; simulated
// registers (row-major [reg][tid]) and the simulated shared array live in shared
// memory, the program's code is staged into shared memory with a TMA bulk copy.  The
// canonical schedule is round-lockstep across the block, but warps are NOT barrier-
// synchronised every round: each warp counts its own rounds (within a barrier interval
// a warp executes exactly one instruction per round while it has runnable lanes) and
// publishes a logical clock 4*round + stage in shared memory.  Only memory
// instructions wait, and only for what the round semantics needs:
//   stage 0 (loads)   : every other warp has finished all earlier rounds;
//   stage 1 (stores)  : every other warp has done its loads of this round, and lower
//                       warps with an overlapping store in this round have stored
//                       (highest tid wins; within a warp via __match_any_sync);
//   stage 2 (atomics) : every other warp has done its stores of this round.
// ALU and branch instructions never wait, so warps drift freely between memory
// operations.  A warp whose lanes all wait at a barrier or exited publishes +inf; when
// all warps of the block have parked, warp 0 resolves the barrier.  Every wait is
// bounded (spin_limit) and reports SR_ST_INTERNAL instead of hanging.
#include <climits>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
enum : uint32_t { DEC_RELEASE = 1, DEC_DONE = 2, DEC_STOP = 3 };

struct BlockVars {
  uint32_t cursor;             // log records reserved by the block (stops growing past the log)
  uint32_t n_misc, epoch, k0, flags, decision, err_dirty, status;
  uint32_t bar_np, bar_nw;     // at a release: true predicates, released threads
  uint32_t race_out;           // fused race check: race entries written so far
  uint32_t gcursor;            // global-log records reserved by the block
  uint32_t pad[4];
};
static_assert(sizeof(BlockVars) <= 64, "block vars");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---- TMA bulk copy of the program code into shared memory (mbarrier completion)
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t phase, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Wait for the CTA's own code-staging copy.  Every thread polls; the CTA agrees on the
// outcome (__syncthreads_or), so that no thread takes a named barrier the others skip.  If the
// copy has not landed within kCopyWaitLimit polls it is waited for once more with the same
// bound; `drained` then says whether it has landed (the shared buffer and the mbarrier phase
// may be reused) or is still in flight (the CTA must leave both alone and exit).
__device__ __forceinline__ bool stage_wait(unsigned long long* bar, uint32_t phase, bool& drained) {
  const bool ok = !__syncthreads_or(!mbar_wait(bar, phase, kCopyWaitLimit));
  drained = ok || !__syncthreads_or(!mbar_wait(bar, phase, kCopyWaitLimit));
  return ok;
}

// Shared-memory accesses by 32-bit shared-window address (cheaper address arithmetic than
// generic pointers in the interpreter's tight loops).
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint2 lds_u64(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ void group_sync(uint32_t id, uint32_t nthr) {
  if (nthr == 32)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
}

// int32 ALU of the IR: two's-complement wrap, C division (x/0 and x%0 flagged)
__device__ __forceinline__ int32_t alu(uint32_t op, int32_t x, int32_t y, bool& dz) {
  switch (op) {
    case SR_OP_MOV: return y;
    case SR_OP_ADD: return (int32_t)((uint32_t)x + (uint32_t)y);
    case SR_OP_SUB: return (int32_t)((uint32_t)x - (uint32_t)y);
    case SR_OP_MUL: return (int32_t)((uint32_t)x * (uint32_t)y);
    case SR_OP_DIV:
      if (y == 0) { dz = true; return 0; }
      return y == -1 ? (int32_t)(0u - (uint32_t)x) : x / y;   // -INT_MIN wraps to INT_MIN
    case SR_OP_REM:
      if (y == 0) { dz = true; return 0; }
      return y == -1 ? 0 : x % y;
    case SR_OP_AND: return x & y;
    case SR_OP_OR: return x | y;
    case SR_OP_XOR: return x ^ y;
    case SR_OP_SHL: return (int32_t)((uint32_t)x << (y & 31));
    case SR_OP_SHR: return x >> (y & 31);                        // arithmetic
    case SR_OP_MIN: return min(x, y);
    case SR_OP_MAX: return max(x, y);
    case SR_OP_SLT: return x < y;
    case SR_OP_SLE: return x <= y;
    case SR_OP_SEQ: return x == y;
    default: return x != y;                                      // SNE
  }
}

// Wait until every other warp of the block has published a clock >= need.  With
// `order` (store stage), also wait for lower warps whose store of this same round
// (clock == need) touches an overlapping range of the same memory space.
// `omin` is a lower bound of the other warps' clocks (clocks only grow within a
// barrier interval); when it already decides the wait, no clock is read.
__device__ __forceinline__ bool wait_clocks(const uint32_t* clk, const int32_t* rlo, const int32_t* rhi,
                                            const uint32_t* rsp, uint32_t nw, uint32_t w, uint32_t lane,
                                            uint32_t need, bool order, int32_t lo, int32_t hi, uint32_t sp,
                                            uint32_t limit, uint32_t& omin) {
  if (omin > need || (!order && omin == need)) return true;
  for (uint32_t it = 0; it < limit; ++it) {
    bool ok = true;
    uint32_t c = kInf;
    if (lane < nw && lane != w) {
      c = ld_acquire_cta(clk + lane);
      ok = c >= need;
      if (ok && order && lane < w && c == need) ok = !(rsp[lane] == sp && rlo[lane] <= hi && lo <= rhi[lane]);
    }
    if (__all_sync(FULL, ok)) {
      omin = __reduce_min_sync(FULL, c);
      __syncwarp();
      return true;
    }
    if (it >= 32) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ void note_err(uint32_t* err, BlockVars* bv, uint32_t p, uint32_t w, uint32_t em,
                                         uint32_t lane) {
  if (lane == (uint32_t)(__ffs(em) - 1)) {
    atomicAdd(&err[2 * p], (uint32_t)__popc(em));
    atomicMin(&err[2 * p + 1], w * 32 + lane);
    bv->err_dirty = 1;
  }
}

// The 8-byte access-log record (layout in sr_internal.h) from its parts.
__device__ __forceinline__ unsigned long long rec_of(uint32_t epoch_hi, uint32_t low_bits, uint32_t addr) {
  return (unsigned long long)(epoch_hi | addr >> 8) << 32 | (low_bits | addr << 24);
}

// Append one record per lane with `me` to the block's access log (warp-aggregated:
// one 32-bit shared atomic per warp, consecutive 8-byte slots -> coalesced stores).
// Once the log is full nothing more is reserved, so the cursor cannot wrap.
__device__ __forceinline__ void log_access(BlockVars* bv, unsigned long long* region, uint32_t front_cap,
                                           bool me, unsigned long long rec, uint32_t lane) {
  const uint32_t m = __ballot_sync(FULL, me);
  if (m == 0) return;
  const uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) {
    base = *reinterpret_cast<volatile uint32_t*>(&bv->cursor);
    if (base < front_cap) base = atomicAdd(&bv->cursor, (uint32_t)__popc(m));
  }
  base = __shfl_sync(FULL, base, leader);
  if (me) {
    const uint32_t pos = base + __popc(m & lanemask_lt());
    if (base < front_cap && pos < front_cap)
      region[pos] = rec;
    else
      atomicOr(&bv->flags, BF_OVERFLOW);
  }
}

// Append one 16-byte global-log record per lane with `me` to the block's global log (the
// same warp-aggregated reservation as log_access).
__device__ __forceinline__ void log_global(BlockVars* bv, uint4* region, uint32_t cap, bool me, uint4 rec,
                                           uint32_t lane) {
  const uint32_t m = __ballot_sync(FULL, me);
  if (m == 0) return;
  const uint32_t leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (lane == leader) {
    base = *reinterpret_cast<volatile uint32_t*>(&bv->gcursor);
    if (base < cap) base = atomicAdd(&bv->gcursor, (uint32_t)__popc(m));
  }
  base = __shfl_sync(FULL, base, leader);
  if (me) {
    const uint32_t pos = base + __popc(m & lanemask_lt());
    if (base < cap && pos < cap)
      region[pos] = rec;
    else
      atomicOr(&bv->flags, BF_OVERFLOW);
  }
}

// ---- fused race check (Sec. 3.1: each shared location keeps the accesses made to it since
// the last barrier).  The summary of a word: the two smallest distinct tids per access kind
// and the lowest and highest pc, enough to decide its races exactly.  Plane q of the
// summaries starts at tup + q * tps: planes 2k and 2k+1 hold the smallest and second
// smallest tid of kind k, planes 6 and 7 the pc range.  Every field is updated by one
// atomic min or max, so an access waits on at most one returned value.
//
// Lanes with `inb` add their access to word `addr`.  Inserting tid into (m1, m2): the min
// into m1 returns the old m1, and the larger of the two (unless equal or empty) is the
// candidate for m2; every value that leaves or misses m1 reaches m2, so m2 ends as the
// smallest tid different from m1.
__device__ __forceinline__ void tuple_add(uint32_t* tup, uint32_t tps, bool inb, uint32_t addr, uint32_t tid,
                                          uint32_t kind, uint32_t pc) {
  if (!inb) return;
  uint32_t* T = tup + addr;
  atomicMin(T + 6u * tps, pc);
  atomicMax(T + 7u * tps, pc);
  const uint32_t o = atomicMin(T + 2u * kind * tps, tid);
  if (o != tid && o != kTupleEmpty) atomicMin(T + (2u * kind + 1u) * tps, max(o, tid));
}

// Conflict classes and the smallest conflicting pair of a word from its summary (two threads
// conflict when distinct and write-write, write-read, write-atomic or atomic-read); false when
// the word has no race.
__device__ __forceinline__ bool tuple_race(const uint32_t* T, uint32_t tps, uint32_t& bout, uint32_t& cout) {
  const uint32_t R[2] = {T[0], T[tps]}, W[2] = {T[2u * tps], T[3u * tps]}, A[2] = {T[4u * tps], T[5u * tps]};
  uint32_t cls = 0, best = 0xFFFFFFFFu;
  auto pair = [&](uint32_t x, uint32_t y, uint32_t bit) {
    if (x == kTupleEmpty || y == kTupleEmpty || x == y) return;
    cls |= bit;
    best = min(best, min(x, y) << 16 | max(x, y));
  };
  pair(W[0], W[1], SR_CLS_WW);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      pair(W[i], R[j], SR_CLS_WR);
      pair(W[i], A[j], SR_CLS_WA);
      pair(A[i], R[j], SR_CLS_AR);
    }
  if (!cls) return false;
  bout = best;
  cout = cls << 24 | (T[6u * tps] & 0xFFFu) << 12 | (T[7u * tps] & 0xFFFu);
  return true;
}

__device__ __forceinline__ void tuple_clear(uint32_t* T, uint32_t tps) {
#pragma unroll
  for (uint32_t q = 0; q < 7; ++q) T[q * tps] = kTupleEmpty;
  T[7u * tps] = 0;
}

// End of an interval, every warp of the block: words 32 j .. 32 j + 31 for its share of j.
// A racy word keeps its pair and class|pcs in planes 0 and 1 and is marked in the bitmap;
// every other touched word is cleared for the next interval.
__device__ __forceinline__ void tuples_mark(uint32_t* tup, uint32_t tps, uint32_t* rbm, uint32_t w, uint32_t nw,
                                            uint32_t lane) {
  for (uint32_t j = w; j < tps / 32u; j += nw) {
    uint32_t* T = tup + 32u * j + lane;
    bool racy = false;
    if (T[6u * tps] != kTupleEmpty) {
      uint32_t b, c;
      racy = tuple_race(T, tps, b, c);
      if (racy) {
        T[0] = b;
        T[tps] = c;
      } else {
        tuple_clear(T, tps);
      }
    }
    const uint32_t m = __ballot_sync(FULL, racy);
    if (lane == 0) rbm[j] = m;
  }
}

// Warp 0: race entries of the interval's racy words in address order at the front of the
// block's region (16 bytes each, after the entries of earlier intervals), then the words are
// cleared.  A racy word had at least two accesses, so the entries fit wherever the region is
// sized by the accesses on a path; past `front_cap` record slots (a loop kernel's fixed
// region) entries are dropped and the block is flagged, as the access log would be.
__device__ void tuples_emit(uint32_t* tup, uint32_t tps, const uint32_t* rbm, BlockVars* bv,
                            unsigned long long* region, uint32_t front_cap, uint32_t epoch, uint32_t lane) {
  const uint32_t nbw = tps / 32u;
  const uint32_t cap = front_cap / 2u;           // entries that fit
  uint32_t ro = bv->race_out;
  bool over = false;
  uint4* out = reinterpret_cast<uint4*>(region);
  for (uint32_t base = 0; base < nbw; base += 32) {
    const uint32_t wd = base + lane;
    uint32_t word = wd < nbw ? rbm[wd] : 0u;
    const uint32_t cnt = __popc(word);
    uint32_t inc = cnt;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    uint32_t pos = ro + inc - cnt;
    while (word) {
      const uint32_t a = wd * 32u + (__ffs(word) - 1);
      word &= word - 1;
      uint32_t* T = tup + a;
      if (pos < cap)
        out[pos] = make_uint4(epoch, a, T[0], T[tps]);
      else
        over = true;
      ++pos;
      tuple_clear(T, tps);
    }
    ro += __shfl_sync(FULL, inc, 31);
  }
  ro = min(ro, cap);
  if (__any_sync(FULL, over) && lane == 0) bv->flags |= BF_OVERFLOW;
  __syncwarp();
  if (lane == 0) {
    bv->race_out = ro;
    bv->cursor = 2u * ro;                        // record slots the entries occupy
  }
  __syncwarp();
}

// Barrier/error records grow down from the end of the block's log region (16 B each).
__device__ void push_misc(BlockVars* bv, unsigned long long* region, uint32_t log_cap, uint32_t kind,
                          uint32_t epoch, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t i = bv->n_misc;
  const uint32_t used = bv->cursor < log_cap ? bv->cursor : log_cap;
  if (2ull * (i + 1) + used > log_cap) {
    bv->flags |= BF_OVERFLOW;
    return;
  }
  reinterpret_cast<uint4*>(region)[log_cap / 2 - 1 - i] = make_uint4(kind << 28 | epoch, a, b, c);
  bv->n_misc = i + 1;
}

// Error records of the interval, ordered by (kind, pc); run by one whole warp.
__device__ void flush_errors(BlockVars* bv, uint32_t* err, uint32_t* un, const uint2* ir, uint32_t ncode,
                             unsigned long long* region, uint32_t log_cap, uint32_t epoch, uint32_t lane) {
  const uint32_t last = un ? SR_REP_ERR_UNINIT_SHARED : SR_REP_ERR_DIV0;
  for (uint32_t kind = SR_REP_ERR_OOB_SHARED; kind <= last; ++kind) {
    for (uint32_t base = 0; base < ncode; base += 32) {
      const uint32_t pc = base + lane;
      uint32_t cnt = 0, mt = 0;
      bool hit = false;
      if (pc < ncode && kind == SR_REP_ERR_UNINIT_SHARED) {
        cnt = un[2 * pc];
        hit = cnt != 0;
        mt = un[2 * pc + 1];
      } else if (pc < ncode) {
        cnt = err[2 * pc];
        if (cnt) {
          const uint32_t op = ir[pc].x & 0x3Fu;
          const uint32_t k2 = (op == SR_OP_LDS || op == SR_OP_STS || op == SR_OP_ATOMS) ? SR_REP_ERR_OOB_SHARED
                              : (op == SR_OP_LDG || op == SR_OP_STG)                   ? SR_REP_ERR_OOB_GLOBAL
                                                                                        : SR_REP_ERR_DIV0;
          hit = (k2 == kind);
          mt = err[2 * pc + 1];
        }
      }
      uint32_t hm = __ballot_sync(FULL, hit);
      while (hm) {
        const uint32_t j = __ffs(hm) - 1;
        hm &= hm - 1;
        const uint32_t jc = __shfl_sync(FULL, cnt, j), jm = __shfl_sync(FULL, mt, j);
        if (lane == 0) push_misc(bv, region, log_cap, kind, epoch, base + j, jm, jc);
        __syncwarp();
      }
    }
  }
  for (uint32_t pc = lane; pc <= ncode; pc += 32) {
    err[2 * pc] = 0;
    err[2 * pc + 1] = kInf;
    if (un) {
      un[2 * pc] = 0;
      un[2 * pc + 1] = kInf;
    }
  }
  __syncwarp();
  if (lane == 0) bv->err_dirty = 0;
}

// Run one simulated block on warps [0, nw) of a group (bar_id = its named barrier).  The
// fused race check is compiled in only where Fused is set, and the logging of global
// accesses only where Global is set, so that the default kernels keep their register budget.
template <bool Fused, bool Global>
__device__ void run_block(const RunArgs& A, const LaunchDev* Ls, uint32_t block, const uint2* __restrict__ ir,
                          unsigned char* gsm, uint32_t w, uint32_t nw, uint32_t bar_id) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nthr = nw * 32;
  const uint32_t tid = w * 32 + lane;
  const uint32_t bdim = Ls->bdim, shw = Ls->shw, ncode = Ls->ncode, log_cap = Ls->log_cap, nrows = Ls->nrows;
  const bool uninit = Ls->uninit != 0;
  const bool fused = Fused && Ls->fused != 0 && A.check_races != 0;
  const GroupLayout G = group_layout(nthr, shw, ncode, nrows, Ls->uninit, Ls->fused);
  uint32_t* regs = reinterpret_cast<uint32_t*>(gsm + G.regs);
  int32_t* sh = reinterpret_cast<int32_t*>(gsm + G.sh);
  uint32_t* clk = reinterpret_cast<uint32_t*>(gsm + kGroupClk);
  int32_t* rlo = reinterpret_cast<int32_t*>(gsm + kGroupRlo);
  int32_t* rhi = reinterpret_cast<int32_t*>(gsm + kGroupRhi);
  uint32_t* rsp = reinterpret_cast<uint32_t*>(gsm + kGroupRsp);
  uint32_t* park = reinterpret_cast<uint32_t*>(gsm + kGroupPark);
  uint32_t* err = reinterpret_cast<uint32_t*>(gsm + G.err);
  uint32_t* un = reinterpret_cast<uint32_t*>(gsm + G.un);      // with `uninit` only
  uint32_t* wb = reinterpret_cast<uint32_t*>(gsm + G.wb);      // with `uninit` only
  uint32_t* tup = reinterpret_cast<uint32_t*>(gsm + G.tup);    // with `fused` only
  const uint32_t tps = tuple_plane_words(shw);
  uint32_t* rbm = reinterpret_cast<uint32_t*>(gsm + G.rbm);
  BlockVars* bv = reinterpret_cast<BlockVars*>(gsm + kGroupBv);
  int32_t* arena = A.arena + Ls->arena_off;
  const uint32_t arena_words = (uint32_t)Ls->arena_words;
  unsigned long long* region = A.log + Ls->log_base + (unsigned long long)block * log_cap;
  const bool logging = A.check_races != 0;
  // global log of this block (with Global, for launches whose glog_cap is set)
  const uint32_t gcap = Global ? Ls->glog_cap : 0u;
  const uint32_t gb = Ls->block_base + block;
  uint4* gregion = Global ? A.glog + Ls->glog_base + (unsigned long long)block * gcap : nullptr;
  const uint32_t budget = A.budget, spin = A.spin_limit;
  uint32_t* myregs = regs + tid;                 // row r of this thread: myregs[r * nthr]
  // the same as 32-bit shared-window addresses, for the fast paths
  const uint32_t rs = smem_u32(myregs), rstride = nthr * 4u, shs = smem_u32(sh), irs = smem_u32(ir);

  // ---- block start: registers = params then zeros (the last row stays zero), shared zeroed
  for (uint32_t r = 0; r < nrows; ++r) myregs[r * nthr] = (r < Ls->nparams) ? (uint32_t)Ls->params[r] : 0u;
  for (uint32_t i = tid; i < shw; i += nthr) sh[i] = 0;
  for (uint32_t i = tid; i <= ncode; i += nthr) {
    err[2 * i] = 0;
    err[2 * i + 1] = kInf;
  }
  if (uninit) {
    for (uint32_t i = tid; i <= ncode; i += nthr) {
      un[2 * i] = 0;
      un[2 * i + 1] = kInf;
    }
    for (uint32_t i = tid; i < (shw + 31u) / 32u; i += nthr) wb[i] = 0;
  }
  if (fused) {
    for (uint32_t i = tid; i < 8u * tps; i += nthr) tup[i] = i < 7u * tps ? kTupleEmpty : 0u;
    for (uint32_t i = tid; i < (shw + 31u) / 32u; i += nthr) rbm[i] = 0;
  }
  if (tid == 0) {
    bv->cursor = 0;
    bv->n_misc = 0; bv->epoch = 0; bv->k0 = 0; bv->flags = 0;
    bv->decision = 0; bv->err_dirty = 0; bv->status = 0;
    bv->race_out = 0;
    bv->gcursor = 0;
  }
  if (lane == 0) clk[w] = 0;
  group_sync(bar_id, nthr);

  uint32_t pc = Ls->entry, st = tid < bdim ? ST_RUN : ST_NONE, wpc = 0;
  // at a barrier: destination row | kind << 5 (0 plain, 1 and, 2 or, 3 count) | predicate << 7
  uint32_t bst = 0;
  uint32_t k = 0, epoch = 0, front_cap = log_cap, omin = 0;
  // pn: the pc the warp issues next (the lowest pc of its runnable lanes, kInf if none);
  // while every runnable lane sits at pn (conv) it is advanced without a reduction
  bool conv = true;
  uint32_t pn = Ls->entry;
  uint32_t n_instr = 0, n_gacc = 0;              // per lane: executed instructions, global accesses
  uint32_t n_sacc = 0;                           // per lane, fused race check: shared accesses
  // a log record is built from 32-bit halves: low = addr << 24 | tid << 14 | kind << 12 | pc,
  // high = epoch << 6 | addr >> 8
  const uint32_t lane_rec = tid << 14;
  uint32_t epoch_hi = 0;                         // epoch << 6

  for (;;) {  // barrier intervals
    bool limit = false, timeout = false;
    for (;;) {  // rounds
      const uint32_t p = pn;
      if (p == kInf) break;                      // no runnable lane
      if (k >= budget) { limit = true; break; }
      const bool act = (st == ST_RUN) && (pc == p);
      const uint2 ins = ir[p];
      const uint32_t op = ins.x & 0x3Fu;
      if (conv && pk_run(ins.x)) {
        // Converged warp at a run of MOV / ADD / MUL instructions (the bulk of straight-line code):
        // every runnable lane is at p and the run touches no memory, so its last round can be
        // published at once (other warps wait on a clock only for memory effects), and the
        // run executes in this tight loop, one instruction per round.
        const bool runl = st == ST_RUN;
        const uint32_t len = min(pk_run(ins.x), budget - k);      // (k < budget here)
        if (lane == 0) st_release_cta(&clk[w], 4u * (k + len));
        uint32_t q = p;
        uint2 in = ins;
        bool bad = false;                        // (debug build: an index check failed)
        for (uint32_t i = 0;;) {
          const uint32_t o = pk_op(in.x), dd = pk_d(in.x);
          if (!dbg_ok(q <= ncode && pk_a(in.x) < nrows && pk_b(in.x) < nrows && (dd < nrows || dd == kNoDest),
                      &A.prog_status[Ls->prog], SR_ST_BOUNDS)) {
            bad = true;
            break;
          }
          const uint32_t a = lds_u32(rs + pk_a(in.x) * rstride);
          const uint32_t b = pk_imm(in.x) ? in.y : lds_u32(rs + pk_b(in.x) * rstride);
          const uint32_t r = o == SR_OP_ADD ? a + b : o == SR_OP_MUL ? a * b : b;   // ADD, MUL, MOV
          if (runl && dd != kNoDest) sts_u32(rs + dd * rstride, r);
          ++q;
          if (++i == len) break;
          in = lds_u64(irs + q * 8u);
        }
        if (bad) {                               // stop the block the way a wait that gave up does
          timeout = true;
          break;
        }
        n_instr += runl ? len : 0u;
        if (runl) pc = q;
        pn = q;
        k += len;
        continue;
      }
      const uint32_t d = pk_d(ins.x), ra = pk_a(ins.x), rb = pk_b(ins.x);
      const int32_t imm = (int32_t)ins.y;
      if (!dbg_ok(p <= ncode && ra < nrows && rb < nrows && (d < nrows || d == kNoDest), &A.prog_status[Ls->prog],
                  SR_ST_BOUNDS)) {
        timeout = true;                          // (debug build) stop the block like a failed wait
        break;
      }
      if (conv && (op == SR_OP_LDS || op == SR_OP_STS) && !uninit && !fused) {
        // Converged warp, shared load or store without the optional checks: the general
        // path's steps for this one case (every runnable lane is at p, the next pc is p + 1).
        const bool runl = st == ST_RUN;
        const int32_t addr = (int32_t)(lds_u32(rs + ra * rstride) + (uint32_t)imm);
        const bool inb = runl && (uint32_t)addr < shw;
        uint32_t kind;
        if (op == SR_OP_LDS) {
          kind = K_R;
          if (nw > 1 && !wait_clocks(clk, rlo, rhi, rsp, nw, w, lane, 4u * k, false, 0, 0, 0, spin, omin)) {
            timeout = true;
            break;
          }
          const uint32_t v = inb ? lds_u32(shs + (uint32_t)addr * 4u) : 0u;
          if (runl && d != kNoDest) sts_u32(rs + d * rstride, v);
        } else {
          kind = K_W;
          const uint32_t vb = lds_u32(rs + rb * rstride);
          if (nw > 1) {
            const int32_t lo = __reduce_min_sync(FULL, inb ? addr : INT_MAX);
            const int32_t hi = __reduce_max_sync(FULL, inb ? addr : INT_MIN);
            if (lane == 0) {
              rlo[w] = lo;
              rhi[w] = hi;
              rsp[w] = 1u;
              st_release_cta(&clk[w], 4u * k + 1u);
            }
            if (!wait_clocks(clk, rlo, rhi, rsp, nw, w, lane, 4u * k + 1u, true, lo, hi, 1u, spin, omin)) {
              timeout = true;
              break;
            }
          }
          // several lanes on one word: the highest tid's store is kept (see the general path)
          const uint32_t sm = __ballot_sync(FULL, inb);
          const int32_t off = __shfl_sync(FULL, addr - (int32_t)lane, sm ? __ffs(sm) - 1 : 0);
          bool last = inb;
          if (!__all_sync(FULL, !inb || addr - (int32_t)lane == off)) {
            const uint32_t grp = __match_any_sync(FULL, inb ? (uint32_t)addr : (0x80000000u | lane));
            last = inb && lane == 31u - __clz(grp);
          }
          if (last) sts_u32(shs + (uint32_t)addr * 4u, vb);
        }
        const uint32_t em = __ballot_sync(FULL, runl && !inb);
        if (em) note_err(err, bv, p, w, em, lane);
        if (logging) log_access(bv, region, front_cap, inb, rec_of(epoch_hi, lane_rec | kind << 12 | p, (uint32_t)addr), lane);
        n_instr += runl;
        if (runl) pc = p + 1;
        pn = p + 1;
        ++k;
        __syncwarp();
        if (lane == 0) st_release_cta(&clk[w], 4u * k);
        continue;
      }
      const int32_t va = (int32_t)myregs[ra * nthr];
      const int32_t vb = pk_imm(ins.x) ? imm : (int32_t)myregs[rb * nthr];
      const bool wr = act && d != kNoDest;
      uint32_t npc = p + 1, cn = p + 1;         // cn: the warp's next pc while converged
      bool memop = false;
      n_instr += act;

      if (op <= SR_OP_SNE) {
        bool dz = false;
        const int32_t r = alu(op, va, vb, dz);
        if (wr) myregs[d * nthr] = (uint32_t)r;
        if (op == SR_OP_DIV || op == SR_OP_REM) {
          const uint32_t em = __ballot_sync(FULL, act && dz);
          if (em) note_err(err, bv, p, w, em, lane);
        }
      } else {
        switch (op) {
          case SR_OP_S2R: {
            const uint32_t v = imm == SR_SREG_TID    ? tid
                               : imm == SR_SREG_BID  ? block + Ls->block_off
                               : imm == SR_SREG_BDIM ? bdim
                               : imm == SR_SREG_GDIM ? Ls->gdim
                                                     : 32u;
            if (wr) myregs[d * nthr] = v;
            break;
          }
          case SR_OP_LDS:
          case SR_OP_LDG: {
            memop = true;
            const bool shared = op == SR_OP_LDS;
            const int32_t addr = (int32_t)((uint32_t)va + (uint32_t)imm);
            const bool inb = act && (uint32_t)addr < (shared ? shw : arena_words);
            if (nw > 1 && !wait_clocks(clk, rlo, rhi, rsp, nw, w, lane, 4u * k, false, 0, 0, 0, spin, omin)) {
              timeout = true;
              break;
            }
            int32_t v = 0;
            if (inb) v = shared ? sh[addr] : arena[addr];
            if (wr) myregs[d * nthr] = (uint32_t)v;
            const uint32_t em = __ballot_sync(FULL, act && !inb);
            if (em) note_err(err, bv, p, w, em, lane);
            if (shared && uninit) {                // words no store or atomic of an earlier round wrote
              const uint32_t um = __ballot_sync(FULL, inb && !((wb[addr >> 5] >> (addr & 31)) & 1u));
              if (um) note_err(un, bv, p, w, um, lane);
            }
            if (shared) {
              if (logging) {
                if (fused) {
                  tuple_add(tup, tps, inb, (uint32_t)addr, tid, K_R, p);
                  n_sacc += inb;
                } else {
                  log_access(bv, region, front_cap, inb,
                           rec_of(epoch_hi, lane_rec | K_R << 12 | p, (uint32_t)addr),
                           lane);
                }
              }
            } else {
              n_gacc += act;
              if (Global && gcap)
                log_global(bv, gregion, gcap, inb, make_uint4((uint32_t)addr, epoch, tid << 16 | p, gb), lane);
            }
            break;
          }
          case SR_OP_STS:
          case SR_OP_STG: {
            memop = true;
            const bool shared = op == SR_OP_STS;
            const int32_t addr = (int32_t)((uint32_t)va + (uint32_t)imm);
            const bool inb = act && (uint32_t)addr < (shared ? shw : arena_words);
            if (nw > 1) {
              const int32_t lo = __reduce_min_sync(FULL, inb ? addr : INT_MAX);
              const int32_t hi = __reduce_max_sync(FULL, inb ? addr : INT_MIN);
              if (lane == 0) {
                rlo[w] = lo;
                rhi[w] = hi;
                rsp[w] = shared;
                st_release_cta(&clk[w], 4u * k + 1u);
              }
              if (!wait_clocks(clk, rlo, rhi, rsp, nw, w, lane, 4u * k + 1u, true, lo, hi, shared, spin, omin)) {
                timeout = true;
                break;
              }
            }
            // several lanes of the warp on one word: the highest tid's store is the one kept.
            // Consecutive addresses, one per lane (addr - lane equal across the storing lanes),
            // cannot collide; any other pattern groups the lanes by address.
            const uint32_t sm = __ballot_sync(FULL, inb);
            const int32_t off = __shfl_sync(FULL, addr - (int32_t)lane, sm ? __ffs(sm) - 1 : 0);
            bool last = inb;
            if (!__all_sync(FULL, !inb || addr - (int32_t)lane == off)) {
              const uint32_t grp = __match_any_sync(FULL, inb ? (uint32_t)addr : (0x80000000u | lane));
              last = inb && lane == 31u - __clz(grp);
            }
            if (last) {
              if (shared)
                sh[addr] = vb;
              else
                arena[addr] = vb;
            }
            if (shared && uninit && inb) atomicOr(&wb[addr >> 5], 1u << (addr & 31));
            const uint32_t em = __ballot_sync(FULL, act && !inb);
            if (em) note_err(err, bv, p, w, em, lane);
            if (shared) {
              if (logging) {
                if (fused) {
                  tuple_add(tup, tps, inb, (uint32_t)addr, tid, K_W, p);
                  n_sacc += inb;
                } else {
                  log_access(bv, region, front_cap, inb,
                           rec_of(epoch_hi, lane_rec | K_W << 12 | p, (uint32_t)addr),
                           lane);
                }
              }
            } else {
              n_gacc += act;
              if (Global && gcap)
                log_global(bv, gregion, gcap, inb, make_uint4((uint32_t)addr, epoch, tid << 16 | 1u << 12 | p, gb),
                           lane);
            }
            break;
          }
          case SR_OP_ATOMS: {
            memop = true;
            const int32_t addr = (int32_t)((uint32_t)va + (uint32_t)imm);
            const bool inb = act && (uint32_t)addr < shw;
            if (nw > 1) {
              if (lane == 0) st_release_cta(&clk[w], 4u * k + 2u);
              if (!wait_clocks(clk, rlo, rhi, rsp, nw, w, lane, 4u * k + 2u, false, 0, 0, 0, spin, omin)) {
                timeout = true;
                break;
              }
            }
            if (inb) atomicAdd(&sh[addr], vb);
            if (uninit && inb) atomicOr(&wb[addr >> 5], 1u << (addr & 31));
            const uint32_t em = __ballot_sync(FULL, act && !inb);
            if (em) note_err(err, bv, p, w, em, lane);
            if (logging) {
                if (fused) {
                  tuple_add(tup, tps, inb, (uint32_t)addr, tid, K_A, p);
                  n_sacc += inb;
                } else {
                  log_access(bv, region, front_cap, inb,
                         rec_of(epoch_hi, lane_rec | K_A << 12 | p, (uint32_t)addr),
                         lane);
                }
              }
            break;
          }
          case SR_OP_BRA: npc = cn = (uint32_t)imm; break;
          case SR_OP_BRZ:
          case SR_OP_BRNZ: {
            const bool taken = (va == 0) == (op == SR_OP_BRZ);
            npc = taken ? (uint32_t)imm : p + 1;
            if (conv) {                          // a split branch ends the converged run
              const uint32_t tm = __ballot_sync(FULL, act && taken);
              if (tm != 0 && tm != __ballot_sync(FULL, act)) conv = false;
              if (tm) cn = (uint32_t)imm;
            }
            break;
          }
          case SR_OP_BAR:
          case SR_OP_BARAND:
          case SR_OP_BAROR:
          case SR_OP_BARPOPC:
            // __syncthreads and its reducing forms: wait; a reducing form hands in its
            // predicate and keeps the row its result goes to
            if (act) {
              st = ST_WAIT;
              wpc = p;
              bst = op == SR_OP_BAR ? 0u : (d | (op - SR_OP_BARAND + 1u) << 5 | (va != 0 ? 1u : 0u) << 7);
            }
            conv = false;
            break;
          default:  // EXIT, and the EXIT sentinel after the last instruction
            if (act) st = ST_EXIT;
            conv = false;
            break;
        }
      }
      if (timeout) break;
      if (act) pc = npc;
      ++k;
      if (conv) {
        pn = cn;
      } else {
        pn = __reduce_min_sync(FULL, st == ST_RUN ? pc : kInf);
        conv = __all_sync(FULL, st != ST_RUN || pc == pn);
      }
      // publish progress; after a memory instruction every lane's access must be
      // ordered before the clock (warp barrier, then a release by lane 0)
      if (memop) __syncwarp();
      if (lane == 0) st_release_cta(&clk[w], 4u * k);
    }

    // ---- no runnable lane in this warp: publish its state and park
    // (`uni`: every waiting lane at one barrier pc and none runnable, the usual case: its
    // lanes all resume together after that barrier)
    bool uni = false;
    uint32_t upc = 0;
    {
      const uint32_t wm = __ballot_sync(FULL, st == ST_WAIT);
      const uint32_t xm = __ballot_sync(FULL, st == ST_EXIT);
      const uint32_t rm = __ballot_sync(FULL, st == ST_RUN);
      const uint32_t tm = __ballot_sync(FULL, st == ST_WAIT && (bst >> 7));   // true predicates
      uint32_t pmn = kInf, pmx = 0, rpc = kInf;
      if (wm) {
        upc = __shfl_sync(FULL, wpc, __ffs(wm) - 1);
        uni = rm == 0 && __all_sync(FULL, st != ST_WAIT || wpc == upc);
        if (uni) {
          pmn = pmx = upc;
        } else {
          pmn = __reduce_min_sync(FULL, st == ST_WAIT ? wpc : kInf);
          pmx = __reduce_max_sync(FULL, st == ST_WAIT ? wpc : 0u);
        }
      }
      if (rm) rpc = __reduce_min_sync(FULL, st == ST_RUN ? pc : kInf);
      if (lane == 0) {
        uint32_t* P = park + w * 8;
        P[0] = __popc(wm); P[1] = __popc(xm); P[2] = __popc(rm);
        P[3] = pmn; P[4] = pmx; P[5] = rpc; P[6] = k;
        P[7] = (limit ? 1u : 0u) | (timeout ? 2u : 0u) | (uint32_t)__popc(tm) << 8;
        st_release_cta(&clk[w], kInf);
      }
    }
    group_sync(bar_id, nthr);
    if (fused) {                                 // the interval's touched words, all warps
      tuples_mark(tup, tps, rbm, w, nw, lane);
      group_sync(bar_id, nthr);
    }

    // ---- barrier resolution by warp 0 of the block
    if (w == 0) {
      const bool v = lane < nw;
      const uint4 pa = reinterpret_cast<const uint4*>(park)[2 * lane];      // warp `lane`'s entry
      const uint4 pb = reinterpret_cast<const uint4*>(park)[2 * lane + 1];
      const uint32_t nW = __reduce_add_sync(FULL, v ? pa.x : 0u);
      const uint32_t nX = __reduce_add_sync(FULL, v ? pa.y : 0u);
      const uint32_t nR = __reduce_add_sync(FULL, v ? pa.z : 0u);
      const uint32_t pmn = __reduce_min_sync(FULL, v ? pa.w : kInf);
      const uint32_t pmx = __reduce_max_sync(FULL, v ? pb.x : 0u);
      const uint32_t rpc = __reduce_min_sync(FULL, v ? pb.y : kInf);
      const uint32_t kmax = __reduce_max_sync(FULL, v ? pb.z : 0u);
      const uint32_t fl = __reduce_or_sync(FULL, v ? pb.w & 0xFFu : 0u);
      const uint32_t nP = __reduce_add_sync(FULL, v ? pb.w >> 8 : 0u);
      const uint32_t ep = bv->epoch;
      if (fused) tuples_emit(tup, tps, rbm, bv, region, log_cap - 2u * bv->n_misc, ep, lane);
      uint32_t dec, kind = 0, a = 0, b = 0, c = 0, stbits = 0;
      if (fl & 2u) {
        dec = DEC_STOP;
        if (lane == 0) bv->flags |= BF_INTERNAL;
      } else if (fl & 1u) {            // out of rounds
        dec = DEC_STOP; kind = SR_REP_STEP_LIMIT; a = budget; b = nR; c = rpc; stbits = SR_ST_STEP_LIMIT;
      } else if (nW == 0) {            // every thread exited
        dec = DEC_DONE;
      } else if (nX > 0) {             // some wait at a barrier that exited threads never reach
        dec = DEC_STOP; kind = SR_REP_DEADLOCK; a = pmn; b = pmx; c = nW << 16 | nX; stbits = SR_ST_DEADLOCK;
      } else {                         // all wait: release, flag differing barrier pcs
        dec = DEC_RELEASE;
        if (pmn != pmx) { kind = SR_REP_DIVERGENCE; a = pmn; b = pmx; c = nW << 16; }
      }
      if (lane == 0 && kind) push_misc(bv, region, log_cap, kind, ep, a, b, c);
      __syncwarp();
      if (bv->err_dirty) flush_errors(bv, err, uninit ? un : nullptr, ir, ncode, region, log_cap, ep, lane);
      if (lane == 0) {
        bv->decision = dec;
        bv->status |= stbits;
        if (dec == DEC_RELEASE) {
          bv->epoch = ep + 1;
          bv->k0 = kmax;
          bv->bar_np = nP;
          bv->bar_nw = nW;
        }
      }
      if (dec == DEC_RELEASE && v) clk[lane] = 4u * kmax;
    }
    group_sync(bar_id, nthr);
    if (bv->decision != DEC_RELEASE) break;
    if (st == ST_WAIT) {
      // a reducing barrier's result, over every released thread's predicate
      const uint32_t kind = (bst >> 5) & 3u, row = bst & 31u;
      if (kind && row != kNoDest) {
        const uint32_t np = bv->bar_np;
        myregs[row * nthr] = kind == 1 ? (np == bv->bar_nw ? 1u : 0u) : kind == 2 ? (np ? 1u : 0u) : np;
      }
      st = ST_RUN;
    }
    if (uni) {                                   // every released lane resumes after its barrier
      pn = upc + 1;
      conv = true;
    } else {
      pn = __reduce_min_sync(FULL, st == ST_RUN ? pc : kInf);
      conv = __all_sync(FULL, st != ST_RUN || pc == pn);
    }
    k = bv->k0;
    omin = 4u * k;                               // every clock was reset to 4 * k0
    epoch = bv->epoch;
    epoch_hi = epoch << 6;
    front_cap = log_cap - 2u * bv->n_misc;
  }

  // ---- block finished
  const uint32_t wi = __reduce_add_sync(FULL, n_instr), wg = __reduce_add_sync(FULL, n_gacc);
  const uint32_t ws = __reduce_add_sync(FULL, n_sacc);
  if (lane == 0) {
    atomicAdd(&A.counters->thread_instrs, (unsigned long long)wi);
    if (wg) atomicAdd(&A.counters->global_accesses, (unsigned long long)wg);
    if (ws) atomicAdd(&A.counters->shared_accesses, (unsigned long long)ws);
  }
  if (tid == 0) {
    const uint32_t front = log_cap - 2u * bv->n_misc;
    BlockRes r;
    r.n_log = fused ? 0u : (bv->cursor < front ? bv->cursor : front);   // fused: no records to check
    r.n_race = fused ? bv->race_out : 0u;
    r.n_misc = bv->n_misc;
    r.flags = bv->flags;
    A.blocks[Ls->block_base + block] = r;
    if (Global && gcap) {
      const uint32_t ng = bv->gcursor < gcap ? bv->gcursor : gcap;
      A.glog_n[gb] = ng;
      if (ng) atomicAdd(&A.counters->global_records, (unsigned long long)ng);
    }
    if (r.n_log) atomicAdd(&A.counters->shared_accesses, (unsigned long long)r.n_log);
    const uint32_t bits = bv->status | ((bv->flags & BF_OVERFLOW) ? (uint32_t)SR_ST_LOG_OVERFLOW : 0u) |
                          ((bv->flags & BF_INTERNAL) ? (uint32_t)SR_ST_INTERNAL : 0u);
    if (bits) atomicOr(&A.prog_status[Ls->prog], bits);
    if (bits & (SR_ST_DEADLOCK | SR_ST_STEP_LIMIT | SR_ST_INTERNAL)) atomicOr(&A.launch_dead[Ls->index], 1u);
  }
}

// A launch is skipped when the launch before it in its stream, or the one it waits for,
// stopped or was skipped (Sec. 3, streams and events; Sec. 3.1, the interpreter halts).
__device__ __forceinline__ bool deps_dead(const RunArgs& A, const LaunchDev& L) {
  const volatile uint32_t* dead = A.launch_dead;
  return (L.dep_prev != kNoDep && dead[L.dep_prev]) || (L.dep_wait != kNoDep && dead[L.dep_wait]);
}

// Thread 0 of a CTA, batched mode: wait (bounded) until every block of the launches L follows
// (the previous launch of its stream, the one it waits for) has completed - they hold earlier
// places in the queue, so CTAs that never wait on L's blocks run them - and decide whether L is
// skipped: a wait that gave up marks the program SR_ST_INTERNAL, and a launch that stopped or
// was skipped skips L (deps_dead).  A skipped launch is marked in launch_dead.
__device__ __forceinline__ bool wait_deps(const RunArgs& A, const LaunchDev& L) {
  bool skip = false;
  const uint32_t deps[2] = {L.dep_prev, L.dep_wait};
  for (uint32_t j = 0; j < 2 && !skip; ++j) {
    if (deps[j] == kNoDep) continue;
    const uint32_t need = A.launches[deps[j]].grid;
    bool ok = false;
    for (uint32_t s = 0; s < A.spin_limit; ++s) {
      if (ld_acquire_gpu(&A.launch_done[deps[j]]) >= need) { ok = true; break; }
      __nanosleep(128);
    }
    if (!ok) {
      skip = true;
      atomicOr(&A.prog_status[L.prog], (uint32_t)SR_ST_INTERNAL);
    }
  }
  if (!skip && deps_dead(A, L)) skip = true;
  if (skip) atomicOr(&A.launch_dead[L.index], 1u);
  return skip;
}

// One CTA per simulated block; one kernel launch per (program, launch), in an order that
// respects every stream and wait.  MINB = 2 caps registers so that two 1024-thread CTAs fit
// an SM.
template <int MINB, bool Fused, bool Global>
__global__ void __launch_bounds__(1024, MINB) k_interp_plain(RunArgs A, uint32_t li) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LaunchDev Ls;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t s_skip;
  if (threadIdx.x == 0) {
    Ls = A.launches[li];
    // (the launches before this one have completed: they ran earlier on this CUDA stream)
    s_skip = deps_dead(A, Ls);
    if (s_skip) atomicOr(&A.launch_dead[Ls.index], 1u);
    if (!s_skip) {
      mbar_init(&mbar);
      bulk_load(smem, A.code + Ls.code_off, Ls.ir_bytes, &mbar);
    }
  }
  __syncthreads();
  if (s_skip) return;
  // every thread must take the same branch before the block's named barriers
  bool drained;
  if (!stage_wait(&mbar, 0, drained)) {
    if (threadIdx.x == 0) atomicOr(&A.prog_status[Ls.prog], (uint32_t)SR_ST_INTERNAL);
    return;
  }
  run_block<Fused, Global>(A, &Ls, blockIdx.x, reinterpret_cast<const uint2*>(smem), smem + Ls.ir_bytes,
                           threadIdx.x >> 5, blockDim.x >> 5, 1);
}

// Persistent: CTAs pop (launch, first block) items from a device queue; an item's
// `item_blocks` simulated blocks run `groups` at a time side by side, each group on its own
// warps and named barrier, a group taking the item's next unclaimed block when it finishes one.
// Items are ordered launch-wave by launch-wave, and an item waits (bounded) until every
// block of the launches it follows (the previous launch of its stream, the one it waits
// for) has completed; launches of other streams run meanwhile.
template <int MINB, bool Fused, bool Global>
__global__ void __launch_bounds__(1024, MINB) k_interp_batched(RunArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LaunchDev Ls;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t s_item, s_skip, s_next, s_claim[32];
  uint32_t phase = 0;
  if (threadIdx.x == 0) mbar_init(&mbar);
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(A.queue_head, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= A.nitems) break;
    const uint2 it = A.items[item];
    if (threadIdx.x == 0) {
      Ls = A.launches[it.x];
      const uint32_t skip = wait_deps(A, Ls) ? 1u : 0u;
      if (!skip) bulk_load(smem, A.code + Ls.code_off, Ls.ir_bytes, &mbar);
      s_skip = skip;
      s_next = Ls.groups;
    }
    __syncthreads();
    const uint32_t nblk = min(Ls.item_blocks, Ls.grid - it.y);
    bool drained = true;
    if (!s_skip) {
      const bool ok = stage_wait(&mbar, phase, drained);
      phase ^= 1u;
      const uint32_t nw = (Ls.bdim + 31) >> 5;
      const uint32_t wid = threadIdx.x >> 5, g = wid / nw;
      if (ok && g < Ls.groups) {
        // block j of the item: the first `groups` one per group, the rest claimed in turn; the
        // group barrier after each block also keeps the next block's set-up behind the last
        // reads of this one
        for (uint32_t j = g; j < nblk;) {
          run_block<Fused, Global>(A, &Ls, it.y + j, reinterpret_cast<const uint2*>(smem),
                                   smem + Ls.ir_bytes + g * Ls.group_bytes, wid - g * nw, nw, 1 + g);
          if (wid == g * nw && (threadIdx.x & 31) == 0) s_claim[g] = atomicAdd(&s_next, 1u);
          group_sync(1 + g, nw * 32);
          j = s_claim[g];
        }
      }
      if (!ok && threadIdx.x == 0) atomicOr(&A.prog_status[Ls.prog], (uint32_t)SR_ST_INTERNAL);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&A.launch_done[it.x], nblk);
    }
    // a staging copy still in flight owns the code buffer and the mbarrier: this CTA takes no
    // further item (the others drain the queue)
    if (!drained) break;
  }
}

// Batched mode with two CTAs per SM: the programs whose every launch would take one group per
// persistent CTA (blocks of more than 512 threads, or blocks whose shared memory leaves room for
// one) run here, one simulated block per 1024-thread CTA and two CTAs per SM, the blocks of all
// such launches of a wave in one grid - the occupancy of the plain kernel without a launch per
// (program, launch).  Each CTA takes the next ticket of the wave's queue; tickets follow launch
// level, then launch index, then block, so the launches a block's launch follows hold smaller
// tickets, taken by CTAs that are already running, and the CTA waits for them (bounded) as the
// persistent kernel does.  No loop surrounds the block and its warps are chosen by a warp vote:
// the block then runs with the plain kernel's register allocation (a persistent loop around it,
// or a branch the compiler cannot see to be warp-uniform, costs several times its spills).
__global__ void __launch_bounds__(1024, 2) k_interp_blocks(RunArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ LaunchDev Ls;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t s_skip, s_block, s_li;
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(A.bq_head, 1u);    // one ticket per CTA: t < the grid size
    // the queue entry holding ticket t: the last one whose first ticket is <= t
    uint32_t lo = 0, hi = A.bq_n;
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (A.bq_first[mid] <= t) lo = mid; else hi = mid;
    }
    const uint32_t li = A.bq_launch[lo];
    Ls = A.launches[li];
    s_li = li;
    s_block = t - A.bq_first[lo];
    bool skip = wait_deps(A, Ls);
    if (!skip && s_block >= Ls.grid) {              // (a corrupt queue: never from load_programs)
      skip = true;
      atomicOr(&A.prog_status[Ls.prog], (uint32_t)SR_ST_INTERNAL);
    }
    if (!skip) {
      mbar_init(&mbar);
      bulk_load(smem, A.code + Ls.code_off, Ls.ir_bytes, &mbar);
    }
    s_skip = skip ? 1u : 0u;
  }
  __syncthreads();
  if (!s_skip) {
    bool drained;
    if (!stage_wait(&mbar, 0, drained)) {
      if (threadIdx.x == 0) atomicOr(&A.prog_status[Ls.prog], (uint32_t)SR_ST_INTERNAL);
    } else {
      const uint32_t nw = (Ls.bdim + 31) >> 5;
      if (__all_sync(FULL, (threadIdx.x >> 5) < nw))
        run_block<false, false>(A, &Ls, s_block, reinterpret_cast<const uint2*>(smem), smem + Ls.ir_bytes,
                                threadIdx.x >> 5, nw, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&A.launch_done[s_li], 1u);
  }
}

}  // namespace

uint32_t interp_plain_smem(const LaunchDev& L) {
  const uint32_t nthr = ((L.bdim + 31) / 32) * 32;
  return L.ir_bytes + group_layout(nthr, L.shw, L.ncode, L.nrows, L.uninit, L.fused).total;
}

// dynamic shared memory may use what the kernel's static shared memory leaves of the opt-in limit
template <typename K>
static cudaError_t allow_dynamic_smem(K kernel, uint32_t smem_optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(smem_optin - (uint32_t)fa.sharedSizeBytes));
}

cudaError_t init_interp_attributes(uint32_t smem_optin) {
  cudaError_t e = allow_dynamic_smem(k_interp_plain<1, false, false>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_plain<2, false, false>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_plain<1, true, false>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_plain<2, true, false>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_plain<1, false, true>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_plain<2, false, true>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_batched<1, false, false>, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_blocks, smem_optin);
  // (two CTAs of up to half the SM's shared memory each: the largest shared-memory carveout)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_interp_blocks, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_interp_batched<1, true, false>, smem_optin);
  return e == cudaSuccess ? allow_dynamic_smem(k_interp_batched<1, false, true>, smem_optin) : e;
}

// The plain-mode kernel for one launch: MINB (register budget) x fused race check x global log.
template <int MINB>
static void (*plain_kernel(bool fused, bool global))(RunArgs, uint32_t) {
  if (global) return k_interp_plain<MINB, false, true>;
  return fused ? k_interp_plain<MINB, true, false> : k_interp_plain<MINB, false, false>;
}

// variant: 1 = one CTA per SM budget (no register cap), 2 = two CTAs per SM, 0 = the one
// with more resident warps for this launch (ties: 1)
cudaError_t launch_interp_plain(const RunArgs& a, uint32_t li, const LaunchDev& L, uint32_t variant, cudaStream_t s) {
  const uint32_t threads = ((L.bdim + 31) / 32) * 32;
  const uint32_t smem = interp_plain_smem(L);
  const bool global = L.glog_cap != 0;
  const bool fused = L.fused != 0 && !global;
  if (variant == 0) {
    int b1 = 0, b2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, plain_kernel<1>(fused, global), (int)threads, smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, plain_kernel<2>(fused, global), (int)threads, smem);
    variant = b2 > b1 ? 2 : 1;
  }
  if (variant == 2)
    plain_kernel<2>(fused, global)<<<L.grid, threads, smem, s>>>(a, li);
  else
    plain_kernel<1>(fused, global)<<<L.grid, threads, smem, s>>>(a, li);
  return cudaGetLastError();
}

cudaError_t launch_interp_batched(const RunArgs& a, uint32_t ctas, uint32_t smem, bool fused, bool global,
                                  cudaStream_t s) {
  auto k = global ? k_interp_batched<1, false, true>
           : fused ? k_interp_batched<1, true, false> : k_interp_batched<1, false, false>;
  k<<<ctas, 1024, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_interp_blocks(const RunArgs& a, uint32_t nblocks, uint32_t smem, cudaStream_t s) {
  k_interp_blocks<<<nblocks, 1024, smem, s>>>(a);
  return cudaGetLastError();
}

// Two CTAs per SM: each may use half the SM's shared memory, less the 1 KB the hardware reserves
// per CTA and the kernel's static shared memory.
uint32_t interp_blocks_smem_cap(uint32_t smem_per_sm) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_interp_blocks) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const uint32_t half = smem_per_sm / 2u, fixed = 1024u + (uint32_t)fa.sharedSizeBytes;
  return half > fixed ? half - fixed : 0u;
}

}  // namespace sr
