// check.cu - race check of the access logs.
//
// Sec. 3.1 of the paper: a race is two threads accessing the same shared location
// with no synchronisation point in between, at least one access writing; the access
// history is cleared at every __syncthreads().  The interpreter wrote one 8-byte
// record per shared access into a per-block log region, the records of a barrier
// interval contiguous and the intervals in order.
//
// Grouping the records of an interval by word address is a counting sort whose one
// digit is the whole 14-bit address, so the groups are never materialised: a table in
// shared memory holds one 32-bit word per shared word,
//     tag:18 | first tid:10 | second-tid flag:1 | access kinds:3,
// updated by one compare-and-swap per record.  Those bits decide whether an address
// races (two distinct tids, and a write or both a read and an atomic), so a race-free
// interval is dropped by advancing the tag.  An interval with a racy address is read a
// second time from the log: each racy address gets an exact summary (the two smallest
// distinct tids per access kind, and the pc range), from which the conflict classes and
// the lexicographically smallest conflicting pair follow exactly (such a pair always
// uses one of the two smallest tids of each kind involved).  Race entries (epoch, addr,
// pair, class|pcs; 16 bytes) are written in address order at the front of the block's
// region; every entry consumes at least two records of its interval, so the writes
// never reach records not yet read.
//
// The table is sized to the wave's shared arrays but capped per kernel shape, because a
// CTA checks one simulated block at a time and the speed follows the blocks in flight
// per SM; an interval that touches a word past the table is read again into a larger
// table the CTA keeps in global memory (the spill table) and closed the same way.
//
// Two families of kernels share the per-stage logic (stage_pass):
//   k_check      one producer warp per CTA claims groups of blocks and streams their
//                records into a ring of shared-memory stages with TMA bulk copies
//                (cp.async.bulk + mbarrier); every wait is bounded: a wait that gives up
//                sets the error flag, and the producer drains its copies before exiting;
//   k_check_reg  every thread loads its own records of the next stage into registers,
//                with the blocks' first stages pulled into L2 ahead of time; no flag is
//                waited on.  The one-warp form runs sixteen CTAs per SM.
// In both, the consumers meet at a named barrier only where an interval ends.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFu;
constexpr uint32_t NB = kCheckBins;
constexpr uint32_t NBW = NB / 32;              // words of the racy-address bitmap
constexpr uint32_t END = 0xFFFFFFFFu;

// table word: tag << 14 | tid << 4 | MULTI | kind bits (1 << K_R, 1 << K_W, 1 << K_A)
constexpr uint32_t TAG_MOD = 1u << 18;
constexpr uint32_t MULTI = 8u;
constexpr uint32_t KB_R = 1u << K_R, KB_W = 1u << K_W, KB_A = 1u << K_A;

__device__ __forceinline__ bool entry_racy(uint32_t x) {
  return (x & MULTI) && ((x & KB_W) || (x & (KB_R | KB_A)) == (KB_R | KB_A));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- summaries
// r/w/a: two smallest distinct tids of that kind (low 16 bits smallest, NONE = absent);
// pc: low 16 bits lowest pc, high 16 bits highest pc.
struct Summ { uint32_t r, w, a, pc; };

__device__ __forceinline__ uint32_t min2_add(uint32_t m, uint32_t t) {
  const uint32_t m1 = m & 0xFFFFu, m2 = m >> 16;
  if (t == m1 || t == m2) return m;
  if (t < m1) return m1 << 16 | t;
  if (t < m2) return t << 16 | m1;
  return m;
}

// Conflict classes (write-write, write-read, write-atomic, atomic-read between
// distinct threads) and the smallest conflicting pair, from the summary alone.
__device__ __forceinline__ bool summ_race(const Summ& s, uint32_t& bout, uint32_t& cout) {
  const uint32_t R[2] = {s.r & 0xFFFFu, s.r >> 16}, W[2] = {s.w & 0xFFFFu, s.w >> 16};
  const uint32_t A[2] = {s.a & 0xFFFFu, s.a >> 16};
  uint32_t cls = 0, best = 0xFFFFFFFFu;
  auto cand = [&](uint32_t x, uint32_t y, uint32_t bit) {
    if (x == NONE || y == NONE || x == y) return;
    cls |= bit;
    best = min(best, min(x, y) << 16 | max(x, y));
  };
  cand(W[0], W[1], SR_CLS_WW);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      cand(W[i], R[j], SR_CLS_WR);
      cand(W[i], A[j], SR_CLS_WA);
      cand(A[i], R[j], SR_CLS_AR);
    }
  if (!cls) return false;
  bout = best;
  cout = cls << 24 | (s.pc & 0xFFFu) << 12 | ((s.pc >> 16) & 0xFFFu);
  return true;
}

// ---------------------------------------------------------------- TMA staging
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Pull [p, p + bytes) into L2 (no destination; p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_init_count(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// non-blocking test of phase completion (a bounded spin loop calls it)
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{ .reg .pred p; mbarrier.test_wait.parity.shared.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}

// Bounded wait for a phase: polls with a growing sleep so that a waiting warp leaves
// the issue slots and the shared-memory pipe to the warps doing work.  Gives up after
// `limit` polls, or as soon as *abort is set.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t phase, uint32_t limit,
                                          const volatile uint32_t* abort) {
  uint32_t ns = 32;
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_test(bar, phase)) return true;
    if (*abort) return false;
    __nanosleep(ns);
    ns = min(ns * 2u, 256u);
  }
  return false;
}

// ---------------------------------------------------------------- consumer barriers
// Named barrier 1 joins the NC consumer threads; the producer warp never takes part.
template <uint32_t NC>
__device__ __forceinline__ void cbar() {
  asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
}
template <uint32_t NC>
__device__ __forceinline__ bool cbar_or(bool p) {
  uint32_t r;
  asm volatile(
      "{ .reg .pred a, b; setp.ne.u32 a, %1, 0; bar.red.or.pred b, 1, %2, a; selp.u32 %0, 1, 0, b; }"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(NC)
      : "memory");
  return r != 0;
}

// Exclusive prefix of the popcounts of bm[0..nw) into pre[]; returns the total.  Ends
// with the consumers synchronised.
template <uint32_t NC>
__device__ uint32_t scan_bitmap(const uint32_t* bm, uint32_t* pre, uint32_t nw, uint32_t* wtot) {
  constexpr uint32_t Q = (NBW + NC - 1) / NC, NCW = NC / 32;
  const uint32_t c = threadIdx.x, lane = c & 31u, w = c >> 5;
  uint32_t v[Q], s = 0;
#pragma unroll
  for (uint32_t q = 0; q < Q; ++q) {
    const uint32_t i = c * Q + q;
    v[q] = i < nw ? __popc(bm[i]) : 0u;
    s += v[q];
  }
  uint32_t x = s;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[w] = x;
  cbar<NC>();
  if (w == 0) {
    const uint32_t t = lane < NCW ? wtot[lane] : 0u;
    uint32_t z = t;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, z, o);
      if (lane >= o) z += y;
    }
    if (lane < NCW) wtot[lane] = z - t;
    if (lane == 31) wtot[NCW] = z;
  }
  cbar<NC>();
  uint32_t base = wtot[w] + x - s;
#pragma unroll
  for (uint32_t q = 0; q < Q; ++q) {
    const uint32_t i = c * Q + q;
    if (i < nw) pre[i] = base;
    base += v[q];
  }
  const uint32_t total = wtot[NCW];
  cbar<NC>();
  return total;
}

// One record (low and high words) into the address table, the tag in the high bits of
// tagw.  An entry that becomes racy marks the interval in *racy; an address past the table
// sets `oor` and is left out.
__device__ __forceinline__ void table_add(uint32_t* tab, uint32_t ntab, uint32_t lo, uint32_t hi, uint32_t tagw,
                                          uint32_t tag, volatile uint32_t* racy, bool& oor) {
  const uint32_t a = __funnelshift_r(lo, hi, 24) & 0x3FFFu;   // record bits 24..37
  if (a >= ntab) {
    oor = true;
    return;
  }
  const uint32_t t4 = (lo >> 10) & 0x3FF0u;                   // tid << 4
  const uint32_t kb = 1u << ((lo >> 12) & 3u);
  uint32_t old = *(volatile uint32_t*)(tab + a);
  for (;;) {
    const uint32_t nw = (old & ~0x3FFFu) != tagw ? (tagw | t4 | kb)
                                                 : (old | kb | ((old & 0x3FF0u) != t4 ? MULTI : 0u));
    if (nw == old) return;
    const uint32_t prev = atomicCAS(tab + a, old, nw);
    if (prev == old) {
      if ((nw & MULTI) && entry_racy(nw)) *racy = tag;
      return;
    }
    old = prev;
  }
}

// The records of mask `m` (bit j: record j) into the table at once: all entries are
// read, all new values computed, and all compare-and-swaps issued before any result is
// needed.  A swap that lost a race (another thread, or an earlier record of this same
// thread, wrote the entry) is redone by table_add.
template <uint32_t P>
__device__ __forceinline__ void table_add_set(uint32_t* tab, uint32_t ntab, const uint32_t (&lo)[P],
                                              const uint32_t (&hi)[P], uint32_t m, uint32_t tagw, uint32_t tag,
                                              volatile uint32_t* racy, bool& oor) {
  uint32_t a[P], x[P], o[P], n[P];
#pragma unroll
  for (uint32_t j = 0; j < P; ++j) {
    a[j] = __funnelshift_r(lo[j], hi[j], 24) & 0x3FFFu;
    if (((m >> j) & 1u) && a[j] >= ntab) {
      oor = true;
      m &= ~(1u << j);
    }
    x[j] = ((lo[j] >> 10) & 0x3FF0u) | 1u << ((lo[j] >> 12) & 3u);
  }
#pragma unroll
  for (uint32_t j = 0; j < P; ++j) o[j] = ((m >> j) & 1u) ? *(volatile uint32_t*)(tab + a[j]) : 0u;
#pragma unroll
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t t4 = x[j] & 0x3FF0u, kb = x[j] & 7u;
    n[j] = (o[j] & ~0x3FFFu) != tagw ? (tagw | x[j]) : (o[j] | kb | ((o[j] & 0x3FF0u) != t4 ? MULTI : 0u));
  }
  uint32_t retry = 0, hit = 0;
#pragma unroll
  for (uint32_t j = 0; j < P; ++j) {
    if (((m >> j) & 1u) && n[j] != o[j]) {
      const uint32_t prev = atomicCAS(tab + a[j], o[j], n[j]);
      if (prev != o[j]) retry |= 1u << j;
      else if ((n[j] & MULTI) && entry_racy(n[j])) hit = 1;
    }
  }
  if (hit) *racy = tag;
  if (retry) {
#pragma unroll
    for (uint32_t j = 0; j < P; ++j)
      if ((retry >> j) & 1u) table_add(tab, ntab, lo[j], hi[j], tagw, tag, racy, oor);
  }
}

// One record into an exact summary held in four table words {r, w, a, pc}.
__device__ __forceinline__ void slot_add(uint32_t* sl, unsigned long long r) {
  const uint32_t t = rec_tid(r), pc = rec_pc(r);
  uint32_t* m = sl + rec_kind(r);                 // K_R, K_W, K_A index r, w, a
  uint32_t old = *(volatile uint32_t*)m;
  for (;;) {
    const uint32_t nw = min2_add(old, t);
    if (nw == old) break;
    const uint32_t prev = atomicCAS(m, old, nw);
    if (prev == old) break;
    old = prev;
  }
  old = *(volatile uint32_t*)(sl + 3);
  for (;;) {
    const uint32_t nw = max(old >> 16, pc) << 16 | min(old & 0xFFFFu, pc);
    if (nw == old) break;
    const uint32_t prev = atomicCAS(sl + 3, old, nw);
    if (prev == old) break;
    old = prev;
  }
}

// Exact pass over a racy interval [s, e) of the block whose region is `region` (the
// consumers are synchronised on entry and on return).  Returns the number of race
// entries written at region (as 16-byte entries) + race_out.  Inlined: as a call, the
// registers live across the call site were spilled in the main loop.
template <uint32_t NC>
__device__ __forceinline__ uint32_t racy_interval(uint32_t* tab, uint32_t ntab, uint32_t* bm, uint32_t* pre,
                                               uint32_t* wtot, uint4* stage_out, unsigned long long* region,
                                               uint32_t race_out, uint32_t shw, uint32_t tagw, uint32_t epoch,
                                               uint32_t s, uint32_t e) {
  const uint32_t DS = ntab / 4;                   // exact summaries per round (4 table words each)
  constexpr uint32_t NCW = NC / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const uint32_t lim = min(shw, ntab);            // every address of the interval is below both
  const uint32_t nw = (lim + 31u) >> 5;
  for (uint32_t wd = warp; wd < nw; wd += NCW) {
    const uint32_t a = wd * 32u + lane;
    const uint32_t x = a < lim ? tab[a] : 0u;
    const uint32_t bits = __ballot_sync(FULL, a < lim && (x & ~0x3FFFu) == tagw && entry_racy(x));
    if (lane == 0) bm[wd] = bits;
  }
  cbar<NC>();
  const uint32_t M = scan_bitmap<NC>(bm, pre, nw, wtot);
  uint4* const dst = M <= DS ? reinterpret_cast<uint4*>(region) + race_out : stage_out;
  for (uint32_t r0 = 0; r0 < M; r0 += DS) {
    const uint32_t nr = min(DS, M - r0);
    for (uint32_t j = tid; j < 4u * nr; j += NC) tab[j] = (j & 3u) == 3u ? NONE : 0xFFFFFFFFu;
    cbar<NC>();
    for (uint32_t i = s + tid; i < e; i += NC) {
      const unsigned long long r = region[i];
      const uint32_t a = rec_addr(r);
      if (a >= lim) continue;                     // (a logged address is always below lim)
      const uint32_t word = bm[a >> 5], bit = 1u << (a & 31u);
      if (!(word & bit)) continue;
      const uint32_t rank = pre[a >> 5] + __popc(word & (bit - 1u)) - r0;
      if (rank < nr) slot_add(tab + 4u * rank, r);
    }
    cbar<NC>();
    for (uint32_t wd = warp; wd < nw; wd += NCW) {
      const uint32_t word = bm[wd];
      if (!((word >> lane) & 1u)) continue;
      const uint32_t rank = pre[wd] + __popc(word & ((1u << lane) - 1u)) - r0;
      if (rank >= nr) continue;
      const uint32_t* sl = tab + 4u * rank;
      uint32_t b = 0, c = 0;
      summ_race(Summ{sl[0], sl[1], sl[2], sl[3]}, b, c);
      dst[r0 + rank] = make_uint4(epoch, wd * 32u + lane, b, c);
    }
    cbar<NC>();
  }
  if (M > DS) {                                   // entries were staged: place them now
    uint4* out = reinterpret_cast<uint4*>(region) + race_out;
    for (uint32_t i = tid; i < M; i += NC) out[i] = __ldcg(stage_out + i);
  }
  for (uint32_t j = tid; j < 4u * min(M, DS); j += NC) tab[j] = 0;
  cbar<NC>();
  return M;
}

// An interval with an address past the shared-memory table (a launch whose shared array is
// larger than the table): its records, still intact in the log, go into the CTA's spill
// table in global memory (kCheckBins entries, zeroed on first use), under the same tag.  An
// address past the shared array there is a corrupt record.  Consumers synchronised on
// entry and on return.
template <uint32_t NC>
__device__ __forceinline__ void spill_interval(uint32_t* gtab, uint32_t shw, const unsigned long long* region,
                                            uint32_t s, uint32_t e, uint32_t tagw, uint32_t tag,
                                            volatile uint32_t* racy, bool& bad, bool& g_ready) {
  if (!g_ready) {
    for (uint32_t i = threadIdx.x; i < kCheckBins; i += NC) gtab[i] = 0;
    g_ready = true;
    cbar<NC>();
  }
  for (uint32_t i = s + threadIdx.x; i < e; i += NC) {
    const unsigned long long r = region[i];
    table_add(gtab, shw, (uint32_t)r, (uint32_t)(r >> 32), tagw, tag, racy, bad);
  }
  cbar<NC>();
}

// End of the interval [s, e) with epoch `epoch` (consumers synchronised): races of a
// racy interval, from the spill table if the interval went there, then the next tag and
// parity.
template <uint32_t NC>
__device__ __forceinline__ void close_interval(uint32_t* tab, uint32_t ntab, uint32_t* gtab, bool spilled,
                                               bool& g_ready, uint32_t* bm, uint32_t* pre,
                                               uint32_t* wtot, uint4* stage_out, volatile uint32_t* s_racy,
                                               unsigned long long* region, uint32_t& race_out, uint32_t shw,
                                               uint32_t& iv, uint32_t& par, uint32_t& tag, uint32_t& tagw,
                                               uint32_t epoch, uint32_t s, uint32_t e) {
  if (s_racy[par] == tag)
    race_out += racy_interval<NC>(spilled ? gtab : tab, spilled ? kCheckBins : ntab, bm, pre, wtot, stage_out, region,
                                  race_out, shw, tagw, epoch, s, e);
  par ^= 1u;
  if (++iv % TAG_MOD == 0) {                      // tags wrap: forget every entry
    cbar<NC>();                                   // everyone has read s_racy
    for (uint32_t i = threadIdx.x; i < ntab; i += NC) tab[i] = 0;
    if (threadIdx.x < 2) s_racy[threadIdx.x] = 0;
    g_ready = false;                              // the spill table is zeroed again before its next use
    cbar<NC>();
    ++iv;
  }
  tag = iv % TAG_MOD;
  tagw = tag << 14;
}

// The records of one stage (this thread's PER records, as low/high words, nval valid;
// e0 / elast the epochs of the stage's first and last records, ebefore that of the record
// before this thread's first), applied interval by interval.  Intervals end here at the
// stage start (1), inside the stage (2) or at the block end (3); `release` is called once
// the stage's records have all been read.  Returns the last reason handled (2 if a corrupt
// log stopped the pass before the release).
template <uint32_t NC, uint32_t PER, class Release>
__device__ __forceinline__ uint32_t stage_pass(
    uint32_t* tab, uint32_t ntab, uint32_t* bm, uint32_t* pre, uint32_t* wtot, uint4* stage_out,
    volatile uint32_t* s_racy,
    volatile uint32_t* s_npos, volatile uint32_t* s_nep, BlockRes* blocks, const uint32_t (&lo)[PER],
    const uint32_t (&hi)[PER], uint32_t nval, uint32_t cbase, uint32_t e0, uint32_t ebefore, uint32_t elast,
    bool first, bool last, uint32_t pos, uint32_t cnt, uint32_t n, uint32_t gb, unsigned long long* region,
    uint32_t shw, uint32_t& race_out, uint32_t& ep, uint32_t& ivs, uint32_t& iv, uint32_t& par, uint32_t& tag,
    uint32_t& tagw, bool& bad, uint32_t* gtab, bool& ovf, bool& g_ready, Release release) {
  uint32_t why = (!first && e0 != ep) ? 1u : 0u;
  for (;;) {
    if (why) {
      const bool spill = cbar_or<NC>(ovf);        // some record of the interval was past the table
      ovf = false;
      uint32_t end = n, nep = ep;
      if (why == 1) {
        end = pos;
        nep = e0;
      } else if (why == 2) {
        const uint32_t np = s_npos[par];
        nep = s_nep[par];
        if (nep <= ep || np >= cnt) {             // epochs out of order: a corrupt log
          bad = true;
          return 2;
        }
        end = pos + np;
      }
      if (spill) spill_interval<NC>(gtab, shw, region, ivs, end, tagw, tag, s_racy + par, bad, g_ready);
      close_interval<NC>(tab, ntab, gtab, spill, g_ready, bm, pre, wtot, stage_out, s_racy, region, race_out, shw, iv,
                         par, tag, tagw, ep, ivs, end);
      if (why == 3) {
        if (threadIdx.x == 0) blocks[gb].n_race = race_out;
        return 3;
      }
      ep = nep;
      ivs = end;
      why = 0;
    }
    uint32_t m = (1u << nval) - 1u;               // this thread's records of interval `ep`
    if (!(e0 == ep && elast == ep)) {             // the stage holds more than interval `ep`
      m = 0;
#pragma unroll
      for (uint32_t j = 0; j < PER; ++j) {
        const uint32_t e = hi[j] >> 6;
        const uint32_t pe = j ? hi[j ? j - 1 : 0] >> 6 : ebefore;
        if (j < nval && e == ep) m |= 1u << j;
        // the record whose predecessor is older notes where the next interval starts
        if (j < nval && e > ep && pe <= ep && cbase + j > 0) {
          s_npos[par] = cbase + j;
          s_nep[par] = e;
        }
      }
    }
    if (__any_sync(FULL, m != 0)) table_add_set<PER>(tab, ntab, lo, hi, m, tagw, tag, s_racy + par, ovf);
    if (elast != ep) {
      why = 2;
      continue;
    }
    release();
    if (!last) return 0;
    why = 3;
  }
}

// A stage of the ring: where its records come from.
struct Desc {
  unsigned long long* region;   // the block's log region
  uint32_t gb, pos, cnt, n;     // block, first record of the stage, records staged, records of the block
  uint32_t shw, flags;          // the launch's shared words; 1 = first stage of the block, 2 = last
};

template <uint32_t NC, uint32_t T, uint32_t NBUF>
struct CheckCfg {
  static constexpr uint32_t NT = NC + 32;       // consumers + one producer warp
  static constexpr uint32_t NCW = NC / 32;
  static constexpr uint32_t PER = T / NC;       // records per consumer thread and stage
  static_assert(PER >= 2 && PER % 2 == 0 && PER * NC == T, "stage must split into pairs of records");
  static constexpr uint32_t TILE_BYTES = T * 8;
  static constexpr uint32_t O_TABLE = NBUF * TILE_BYTES;
  static constexpr uint32_t O_BM = O_TABLE + NB * 4;
  static constexpr uint32_t O_PRE = O_BM + NBW * 4;
  static constexpr uint32_t O_DESC = O_PRE + NBW * 4;
  static constexpr uint32_t O_MISC = O_DESC + NBUF * (uint32_t)sizeof(Desc);
  static constexpr uint32_t MISC_WORDS = 8 + NCW + 1;
  static constexpr uint32_t SMEM = O_MISC + MISC_WORDS * 4;
};

template <uint32_t NC, uint32_t T, uint32_t NBUF, uint32_t MINB>
__global__ void __launch_bounds__(NC + 32, MINB) k_check(CheckArgs A) {
  using C = CheckCfg<NC, T, NBUF>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[NBUF], empty[NBUF];
  const unsigned long long* tiles = reinterpret_cast<const unsigned long long*>(smem);
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + C::O_TABLE);
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem + C::O_BM);
  uint32_t* pre = reinterpret_cast<uint32_t*>(smem + C::O_PRE);
  Desc* desc = reinterpret_cast<Desc*>(smem + C::O_DESC);
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + C::O_MISC);
  volatile uint32_t* s_racy = misc;              // [2] tag of the racy interval, by interval parity
  volatile uint32_t* s_npos = misc + 2;          // [2] first record of the next interval in the stage
  volatile uint32_t* s_nep = misc + 4;           // [2] its epoch
  volatile uint32_t* s_fail = misc + 6;
  uint32_t* wtot = misc + 8;
  const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;

  for (uint32_t i = tid; i < NB; i += C::NT) tab[i] = 0;
  if (tid < 8) misc[tid] = 0;
  if (tid == 0) {
    for (uint32_t b = 0; b < NBUF; ++b) {
      mbar_init_count(&full[b], 1);
      mbar_init_count(&empty[b], C::NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == C::NCW) {
    // ------------------------------------------------------------ producer warp
    uint32_t k = 0;
    bool failed = false;
    auto claim = [&]() {
      uint32_t v = 0;
      if (lane == 0) v = A.item0 + atomicAdd(A.work_head, 1u);
      return __shfl_sync(FULL, v, 0);
    };
    // wait until stage buffer `buf` is free for the chunk numbered k
    auto acquire = [&](uint32_t buf) {
      bool ok = true;
      if (lane == 0 && k >= NBUF) {
        const uint32_t ph = ((k / NBUF) & 1u) ^ 1u;
        ok = mbar_wait(&empty[buf], ph, A.spin_limit, s_fail);
      }
      return __shfl_sync(FULL, (uint32_t)ok, 0) != 0;
    };
    uint32_t item = claim();
    while (item < A.item1 && !failed) {
      uint32_t lo = A.li0, hi = A.li1 - 1;       // launch owning the item
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (A.launches[mid].check_item <= item) lo = mid; else hi = mid - 1;
      }
      const LaunchDev* L = A.launches + lo;
      const uint32_t first = L->block_base + (item - L->check_item) * L->check_group;
      const uint32_t nb = min(L->check_group, L->block_base + L->grid - first);
      const uint32_t n_l = lane < nb ? A.blocks[first + lane].n_log : 0u;
      const unsigned long long* log0 = A.log + L->log_base;
      const uint32_t cap = L->log_cap, base = L->block_base, shw = L->shw;
      const uint32_t next = claim();               // in flight while this item streams
      for (uint32_t b = 0; b < nb && !failed; ++b) {
        const uint32_t n = __shfl_sync(FULL, n_l, b);
        if (!n) continue;
        unsigned long long* region = const_cast<unsigned long long*>(log0) + (unsigned long long)(first + b - base) * cap;
        for (uint32_t pos = 0; pos < n; pos += T) {
          const uint32_t buf = k % NBUF;
          if (!acquire(buf)) { failed = true; break; }
          if (lane == 0) {
            const uint32_t cnt = min(T, n - pos);
            Desc& d = desc[buf];
            d.region = region;
            d.gb = first + b;
            d.pos = pos;
            d.cnt = cnt;
            d.n = n;
            d.shw = shw;
            d.flags = (pos == 0 ? 1u : 0u) | (pos + cnt == n ? 2u : 0u);
            bulk_load(const_cast<unsigned long long*>(tiles) + (size_t)buf * T, region + pos, ((cnt + 1u) & ~1u) * 8u,
                      &full[buf]);
          }
          __syncwarp();
          ++k;
        }
      }
      item = next;
    }
    if (!failed) {
      const uint32_t buf = k % NBUF;
      if (acquire(buf)) {
        if (lane == 0) {
          desc[buf].gb = END;
          mbar_arrive(&full[buf]);
        }
      } else {
        failed = true;
      }
    }
    if (failed) {
      if (lane == 0) {
        *s_fail = 1;
        atomicOr(A.error_flag, 1u);
        // every copy issued must land before the CTA may exit
        for (uint32_t b = 0; b < NBUF && b < k; ++b) {
          const uint32_t last = b + ((k - 1 - b) / NBUF) * NBUF;
          const uint32_t never = 0;
          mbar_wait(&full[b], (last / NBUF) & 1u, kCopyWaitLimit, &never);
        }
      }
      __syncwarp();
    }
    return;
  }

  // -------------------------------------------------------------- consumer warps
  const uint32_t cbase = tid * C::PER;
  uint4* const stage_out = A.scratch + (size_t)blockIdx.x * kScratchWords;
  uint32_t* const gtab = reinterpret_cast<uint32_t*>(stage_out + kCheckBins);
  bool ovf = false, g_ready = false;
  uint32_t iv = 1, par = 0, tag = 1, tagw = 1u << 14;
  // per block
  unsigned long long* region = nullptr;
  uint32_t gb = 0, race_out = 0, ep = 0, ivs = 0, shw = 0;

  for (uint32_t k = 0;; ++k) {
    const uint32_t buf = k % NBUF;
    const bool ok = mbar_wait(&full[buf], (k / NBUF) & 1u, A.spin_limit, s_fail);
    if (cbar_or<NC>(!ok)) {
      if (tid == 0) {
        *s_fail = 1;
        atomicOr(A.error_flag, 1u);
      }
      return;
    }
    const Desc& d = desc[buf];
    const uint32_t d_gb = d.gb;
    if (d_gb == END) break;
    const uint32_t d_pos = d.pos, d_cnt = d.cnt, d_n = d.n, d_flags = d.flags;
    const unsigned long long* tile = tiles + (size_t)buf * T;
    const uint32_t e0 = rec_epoch(tile[0]);
    if (d_flags & 1u) {
      region = d.region;
      gb = d_gb;
      shw = d.shw;
      race_out = 0;
      ep = e0;
      ivs = 0;
    }
    // this thread's records as (low, high) words; the epoch is the high word >> 6
    uint32_t lo[C::PER], hi[C::PER];
#pragma unroll
    for (uint32_t j = 0; j < C::PER; j += 2) {
      const uint4 v = *reinterpret_cast<const uint4*>(tile + cbase + j);
      lo[j] = v.x;
      hi[j] = v.y;
      lo[j + 1] = v.z;
      hi[j + 1] = v.w;
    }
    const uint32_t nval = d_cnt > cbase ? min(C::PER, d_cnt - cbase) : 0u;
    const uint32_t ebefore = cbase ? rec_epoch(tile[min(cbase, d_cnt) - 1]) : 0u;
    const uint32_t elast = rec_epoch(tile[d_cnt - 1]);
    bool bad = false;
    const uint32_t why = stage_pass<NC, C::PER>(
        tab, NB, bm, pre, wtot, stage_out, s_racy, s_npos, s_nep, A.blocks, lo, hi, nval, cbase, e0, ebefore, elast,
        d_flags & 1u, d_flags & 2u, d_pos, d_cnt, d_n, gb, region, shw, race_out, ep, ivs, iv, par, tag, tagw, bad,
        gtab, ovf, g_ready, [&]() {
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[buf]);   // the stage may be refilled
        });
    if (bad) {
      atomicOr(A.error_flag, 2u);
      if (why == 2) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[buf]);
      }
    }
  }
}

// ---------------------------------------------------------------- register-staged form
// The same check without the shared-memory ring: every thread loads its records of a
// stage straight from the log into registers (16-byte loads, coalesced across the warp),
// the next stage's loads in flight while the current one is processed, and the CTA meets
// only where an interval ends and between work items.  Nothing waits on a flag here, and
// all the shared memory goes to the address table, so more CTAs fit on an SM.
template <uint32_t NC>
struct RegCfg {
  static constexpr uint32_t NCW = NC / 32;
  static constexpr uint32_t O_BM = 0;
  static constexpr uint32_t O_PRE = O_BM + NBW * 4;
  static constexpr uint32_t O_ITEM = O_PRE + NBW * 4;          // [2] x {item, launch, n[32]}
  static constexpr uint32_t ITEM_WORDS = 2 + kCheckMaxGroup;
  static constexpr uint32_t O_MISC = O_ITEM + 2 * ITEM_WORDS * 4;
  static constexpr uint32_t MISC_WORDS = 8 + NCW + 1;
  static constexpr uint32_t O_TABLE = (O_MISC + MISC_WORDS * 4 + 15u) & ~15u;   // table_words entries
  static constexpr uint32_t smem(uint32_t table_words) { return O_TABLE + table_words * 4; }
};

// Records [0, nval) of a stage from src (16-byte aligned); the pair that holds the last
// record may read one record past it, which is still inside the block's region.
template <uint32_t PER>
__device__ __forceinline__ void load_records(const unsigned long long* src, uint32_t nval, uint32_t (&lo)[PER],
                                             uint32_t (&hi)[PER]) {
#pragma unroll
  for (uint32_t j = 0; j < PER; j += 2) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (j < nval) v = *reinterpret_cast<const uint4*>(src + j);
    lo[j] = v.x;
    hi[j] = v.y;
    lo[j + 1] = v.z;
    hi[j + 1] = v.w;
  }
}

constexpr uint32_t kAheadStages = 8;             // L2 prefetch distance inside a block

// Warp 0: resolve work item `item` into sh = {item, launch, n_log of each of its blocks}
// and pull the first stages of every block into L2.
__device__ __forceinline__ void item_setup(const CheckArgs& A, uint32_t item, volatile uint32_t* sh,
                                           uint32_t ahead_records) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t li = 0, nb = 0, first = 0;
  if (item < A.item1) {
    uint32_t lo = A.li0, hi = A.li1 - 1;
    if (A.item_launch) {
      lo = A.item_launch[item];
    } else {
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (A.launches[mid].check_item <= item) lo = mid; else hi = mid - 1;
      }
    }
    const LaunchDev* L = A.launches + lo;
    li = lo;
    first = L->block_base + (item - L->check_item) * L->check_group;
    nb = min(L->check_group, L->block_base + L->grid - first);
    if (lane < nb) {
      const uint32_t n = A.blocks[first + lane].n_log;
      sh[2 + lane] = n;
      if (n) {
        const unsigned long long* region =
            A.log + L->log_base + (unsigned long long)(first + lane - L->block_base) * L->log_cap;
        prefetch_l2(region, ((min(n, ahead_records) + 1u) & ~1u) * 8u);
      }
    }
  }
  if (lane == 0) {
    sh[0] = item;
    sh[1] = li;
  }
}

template <uint32_t NC, uint32_t PER, uint32_t MINB>
__global__ void __launch_bounds__(NC, MINB) k_check_reg(CheckArgs A) {
  using C = RegCfg<NC>;
  constexpr uint32_t T = NC * PER;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + C::O_TABLE);
  const uint32_t ntab = A.table_words;           // >= every shared array of the wave
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem + C::O_BM);
  uint32_t* pre = reinterpret_cast<uint32_t*>(smem + C::O_PRE);
  volatile uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + C::O_ITEM);
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + C::O_MISC);
  volatile uint32_t* s_racy = misc;              // [2] tag of the racy interval, by interval parity
  volatile uint32_t* s_npos = misc + 2;          // [2] first record of the next interval in the stage
  volatile uint32_t* s_nep = misc + 4;           // [2] its epoch
  uint32_t* wtot = misc + 8;
  const uint32_t tid = threadIdx.x, cbase = tid * PER;
  uint4* const stage_out = A.scratch + (size_t)blockIdx.x * kScratchWords;
  uint32_t* const gtab = reinterpret_cast<uint32_t*>(stage_out + kCheckBins);
  bool ovf = false, g_ready = false;

  for (uint32_t i = tid; i < ntab; i += NC) tab[i] = 0;
  if (tid < 8) misc[tid] = 0;
  if (tid < 32) {
    uint32_t item = 0;
    if (tid == 0) item = A.item0 + atomicAdd(A.work_head, 1u);
    item_setup(A, __shfl_sync(FULL, item, 0), s_items, kAheadStages * T);
  }
  __syncthreads();
  uint32_t ipar = 0;
  uint32_t iv = 1, par = 0, tag = 1, tagw = 1u << 14;
  bool bad = false, stop = false;                // bad: this thread saw a corrupt record; stop: all did
  for (;;) {
    volatile uint32_t* sh = s_items + ipar * C::ITEM_WORDS;
    const uint32_t item = sh[0];
    if (item >= A.item1) break;
    uint32_t next = 0;
    if (tid == 0) next = A.item0 + atomicAdd(A.work_head, 1u);   // in flight during this item
    const LaunchDev* L = A.launches + sh[1];
    const uint32_t first = L->block_base + (item - L->check_item) * L->check_group;
    const uint32_t nb = min(L->check_group, L->block_base + L->grid - first);
    unsigned long long* const log0 = A.log + L->log_base;
    const uint32_t cap = L->log_cap, base = L->block_base, shw = L->shw;
    for (uint32_t b = 0; b < nb; ++b) {
      const uint32_t gb = first + b;
      const uint32_t n = sh[2 + b];
      if (!n) continue;
      // (debug build: the block's records lie inside its region)
      if (!dbg_ok(n <= cap && gb - base < L->grid, A.error_flag, kErrBounds)) continue;
      unsigned long long* const region = log0 + (unsigned long long)(gb - base) * cap;
      uint32_t race_out = 0, ep = 0, ivs = 0;
      // a stage: this thread's records plus three epochs (the stage's first and last
      // records, and the record before this thread's first), loaded one stage ahead
      const uint32_t* const hw = reinterpret_cast<const uint32_t*>(region) + 1;   // high word of record i: hw[2i]
      uint32_t clo[PER], chi[PER], ce0, celast, cebefore;
      {
        const uint32_t cnt = min(T, n);
        load_records<PER>(region + cbase, cnt > cbase ? min(PER, cnt - cbase) : 0u, clo, chi);
        ce0 = hw[0];
        celast = hw[2u * (cnt - 1u)];
        cebefore = cbase ? hw[2u * (min(cbase, cnt) - 1u)] : 0u;
      }
      for (uint32_t pos = 0; pos < n; pos += T) {
        const uint32_t cnt = min(T, n - pos);
        const uint32_t nval = cnt > cbase ? min(PER, cnt - cbase) : 0u;
        const bool last = pos + T >= n;
        uint32_t nlo[PER], nhi[PER], ne0 = 0, nelast = 0, nebefore = 0;
        if (!last) {                              // the next stage's loads go out first
          const uint32_t npos = pos + T, ncnt = min(T, n - npos);
          load_records<PER>(region + npos + cbase, ncnt > cbase ? min(PER, ncnt - cbase) : 0u, nlo, nhi);
          ne0 = hw[2u * npos];
          nelast = hw[2u * (npos + ncnt - 1u)];
          nebefore = cbase ? hw[2u * (npos + min(cbase, ncnt) - 1u)] : 0u;
          const uint32_t far = pos + kAheadStages * T;
          if (tid == 0 && far < n) prefetch_l2(region + far, ((min(T, n - far) + 1u) & ~1u) * 8u);
        }
        const uint32_t e0 = ce0 >> 6, elast = celast >> 6, ebefore = cebefore >> 6;
        if (pos == 0) ep = e0;
        const uint32_t how =
            stage_pass<NC, PER>(tab, ntab, bm, pre, wtot, stage_out, s_racy, s_npos, s_nep, A.blocks, clo, chi, nval,
                                cbase, e0, ebefore, elast, pos == 0, last, pos, cnt, n, gb, region, shw, race_out, ep,
                                ivs, iv, par, tag, tagw, bad, gtab, ovf, g_ready, []() {});
        if (how == 2) {                           // (uniform) epochs out of order: give up
          stop = true;
          break;
        }
        if (!last) {
#pragma unroll
          for (uint32_t j = 0; j < PER; ++j) {
            clo[j] = nlo[j];
            chi[j] = nhi[j];
          }
          ce0 = ne0;
          celast = nelast;
          cebefore = nebefore;
        }
      }
      if (stop) break;
    }
    if (stop) break;
    // warp 0 prepares the next item (its blocks' records start moving into L2) while
    // the other warps finish this one
    if (tid < 32) item_setup(A, __shfl_sync(FULL, next, 0), s_items + (ipar ^ 1u) * C::ITEM_WORDS, kAheadStages * T);
    __syncthreads();
    ipar ^= 1u;
  }
  if (bad || stop) atomicOr(A.error_flag, kErrCorrupt);
}

// ---------------------------------------------------------------- lean one-warp form
// One warp per CTA and one simulated block at a time, as in the one-warp register-staged form,
// with a leaner main loop: a chunk is 32 x R records, lane l holding records base + 32 j + l
// (one coalesced 8-byte load per j), the next chunk's loads in flight while this one is
// applied.  A chunk whose first and last records belong to the open interval - most of them -
// goes to the table with no per-record interval work; only a chunk in which intervals end is
// taken apart interval by interval.  Intervals are closed, spilled and checked exactly by the
// same code as in the other forms.
template <uint32_t R>
__device__ __forceinline__ void lean_load(const unsigned long long* region, uint32_t base, uint32_t n, uint32_t lane,
                                          uint32_t (&lo)[R], uint32_t (&hi)[R]) {
#pragma unroll
  for (uint32_t j = 0; j < R; ++j) {
    const uint32_t i = base + 32u * j + lane;
    unsigned long long v = 0;
    if (i < n) v = __ldcs(region + i);           // streamed once (the exact pass re-reads from L2 or HBM)
    lo[j] = (uint32_t)v;
    hi[j] = (uint32_t)(v >> 32);
  }
}

template <uint32_t R>
__global__ void __launch_bounds__(32, 20) k_check_lean(CheckArgs A) {
  using C = RegCfg<32>;
  constexpr uint32_t T = 32u * R;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* tab = reinterpret_cast<uint32_t*>(smem + C::O_TABLE);
  const uint32_t ntab = A.table_words;
  uint32_t* bm = reinterpret_cast<uint32_t*>(smem + C::O_BM);
  uint32_t* pre = reinterpret_cast<uint32_t*>(smem + C::O_PRE);
  volatile uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + C::O_ITEM);
  uint32_t* misc = reinterpret_cast<uint32_t*>(smem + C::O_MISC);
  volatile uint32_t* s_racy = misc;              // [2] tag of the racy interval, by interval parity
  uint32_t* wtot = misc + 8;
  const uint32_t lane = threadIdx.x;
  uint4* const stage_out = A.scratch + (size_t)blockIdx.x * kScratchWords;
  uint32_t* const gtab = reinterpret_cast<uint32_t*>(stage_out + kCheckBins);
  bool g_ready = false, bad = false;

  for (uint32_t i = lane; i < ntab; i += 32) tab[i] = 0;
  if (lane < 8) misc[lane] = 0;
  {
    uint32_t item = 0;
    if (lane == 0) item = A.item0 + atomicAdd(A.work_head, 1u);
    item_setup(A, __shfl_sync(FULL, item, 0), s_items, kAheadStages * T);
  }
  __syncwarp();
  uint32_t ipar = 0;
  uint32_t iv = 1, par = 0, tag = 1, tagw = 1u << 14;
  for (;;) {
    volatile uint32_t* sh = s_items + ipar * C::ITEM_WORDS;
    const uint32_t item = sh[0];
    if (item >= A.item1) break;
    const LaunchDev* L = A.launches + sh[1];
    const uint32_t first = L->block_base + (item - L->check_item) * L->check_group;
    const uint32_t nb = min(L->check_group, L->block_base + L->grid - first);
    unsigned long long* const log0 = A.log + L->log_base;
    const uint32_t cap = L->log_cap, base0 = L->block_base, shw = L->shw;
    for (uint32_t b = 0; b < nb && !bad; ++b) {
      const uint32_t gb = first + b;
      const uint32_t n = sh[2 + b];
      if (!n) continue;
      if (!dbg_ok(n <= cap && gb - base0 < L->grid, A.error_flag, kErrBounds)) continue;
      unsigned long long* const region = log0 + (unsigned long long)(gb - base0) * cap;
      const uint32_t* const hw = reinterpret_cast<const uint32_t*>(region) + 1;   // high word of record i: hw[2i]
      uint32_t race_out = 0, ivs = 0;            // race entries written, start of the open interval
      uint32_t cur = hw[0] >> 6;                 // its epoch
      bool ovf = false;                          // some record of the open interval is past the table
      // close the open interval at record `end`
      auto close = [&](uint32_t end) {
        const bool spill = __any_sync(FULL, ovf);
        ovf = false;
        if (spill) spill_interval<32>(gtab, shw, region, ivs, end, tagw, tag, s_racy + par, bad, g_ready);
        close_interval<32>(tab, ntab, gtab, spill, g_ready, bm, pre, wtot, stage_out, s_racy, region, race_out, shw,
                           iv, par, tag, tagw, cur, ivs, end);
      };
      uint32_t clo[R], chi[R];
      lean_load<R>(region, 0, n, lane, clo, chi);
      for (uint32_t base = 0; base < n; base += T) {
        const uint32_t e = min(n, base + T);
        uint32_t nlo[R], nhi[R];
        const bool more = e < n;
        if (more) {                              // the next chunk's loads go out first
          lean_load<R>(region, e, n, lane, nlo, nhi);
          const uint32_t far = base + kAheadStages * T;
          if (lane == 0 && far < n) prefetch_l2(region + far, ((min(T, n - far) + 1u) & ~1u) * 8u);
        }
        // the epoch of the chunk's last record, from the register that holds it
        uint32_t last_ep;
        {
          const uint32_t t = e - 1u - base, jl = t >> 5;
          uint32_t h = chi[0];
#pragma unroll
          for (uint32_t j = 1; j < R; ++j) h = jl == j ? chi[j] : h;
          last_ep = __shfl_sync(FULL, h, t & 31u) >> 6;
        }
        uint32_t valid = 0;
#pragma unroll
        for (uint32_t j = 0; j < R; ++j) valid |= (base + 32u * j + lane < e ? 1u : 0u) << j;
        if (last_ep == cur) {
          // the whole chunk lies in the open interval
          if (__any_sync(FULL, valid != 0)) table_add_set<R>(tab, ntab, clo, chi, valid, tagw, tag, s_racy + par, ovf);
        } else {
          // intervals end in this chunk: apply it interval by interval (epochs ascend)
          uint32_t pending = valid;              // this lane's records not applied yet
          for (;;) {
            uint32_t m = 0, later = kInf;
#pragma unroll
            for (uint32_t j = 0; j < R; ++j) {
              const uint32_t ep = chi[j] >> 6;
              if ((pending >> j) & 1u) {
                if (ep == cur) m |= 1u << j;
                else if (ep > cur) later = min(later, base + 32u * j + lane);
                else bad = true;                 // epochs out of order: a corrupt log
              }
            }
            pending &= ~m;
            if (__any_sync(FULL, m != 0)) table_add_set<R>(tab, ntab, clo, chi, m, tagw, tag, s_racy + par, ovf);
            later = __reduce_min_sync(FULL, later);
            if (later == kInf || __any_sync(FULL, bad)) break;   // the open interval goes on
            close(later);
            ivs = later;
            cur = hw[2u * later] >> 6;
          }
          if (__any_sync(FULL, bad)) {
            bad = true;
            break;
          }
        }
        if (more) {
#pragma unroll
          for (uint32_t j = 0; j < R; ++j) {
            clo[j] = nlo[j];
            chi[j] = nhi[j];
          }
        }
      }
      if (bad) break;
      close(n);
      if (lane == 0) A.blocks[gb].n_race = race_out;
    }
    if (bad) break;
    uint32_t next = 0;
    if (lane == 0) next = A.item0 + atomicAdd(A.work_head, 1u);
    ipar ^= 1u;
    item_setup(A, __shfl_sync(FULL, next, 0), s_items + ipar * C::ITEM_WORDS, kAheadStages * T);
    __syncwarp();
  }
  if (bad) atomicOr(A.error_flag, kErrCorrupt);
}

template <uint32_t R>
struct LeanVariant {
  static constexpr uint32_t smem(uint32_t table_words) { return RegCfg<32>::smem(table_words); }
  static cudaError_t init(uint32_t optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_check_lean<R>);
    if (e != cudaSuccess) return e;
    if (smem(NB) + fa.sharedSizeBytes > optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_check_lean<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem(NB));
  }
  static cudaError_t launch(const CheckArgs& a, uint32_t ctas, cudaStream_t s) {
    k_check_lean<R><<<ctas, 32, smem(a.table_words), s>>>(a);
    return cudaGetLastError();
  }
};

template <uint32_t NC, uint32_t PER, uint32_t MINB>
struct RegVariant {
  static constexpr uint32_t smem(uint32_t table_words) { return RegCfg<NC>::smem(table_words); }
  static cudaError_t init(uint32_t optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_check_reg<NC, PER, MINB>);
    if (e != cudaSuccess) return e;
    if (smem(NB) + fa.sharedSizeBytes > optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_check_reg<NC, PER, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem(NB));
  }
  static cudaError_t launch(const CheckArgs& a, uint32_t ctas, cudaStream_t s) {
    k_check_reg<NC, PER, MINB><<<ctas, NC, smem(a.table_words), s>>>(a);
    return cudaGetLastError();
  }
};

// Checker variants (consumer threads, records per stage, stages, CTAs per SM).
template <uint32_t NC, uint32_t T, uint32_t NBUF, uint32_t MINB>
struct CheckVariant {
  static constexpr uint32_t smem() { return CheckCfg<NC, T, NBUF>::SMEM; }
  static cudaError_t init(uint32_t optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_check<NC, T, NBUF, MINB>);
    if (e != cudaSuccess) return e;
    if (smem() + fa.sharedSizeBytes > optin) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_check<NC, T, NBUF, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
  }
  static cudaError_t launch(const CheckArgs& a, uint32_t ctas, cudaStream_t s) {
    k_check<NC, T, NBUF, MINB><<<ctas, NC + 32, smem(), s>>>(a);
    return cudaGetLastError();
  }
};

struct VariantEntry {
  cudaError_t (*init)(uint32_t);
  cudaError_t (*launch)(const CheckArgs&, uint32_t, cudaStream_t);
  uint32_t ctas_per_sm;
  uint32_t table_cap;           // shared-memory address table entries at most
};
template <class V, uint32_t MINB, uint32_t CAP>
constexpr VariantEntry entry() { return VariantEntry{&V::init, &V::launch, MINB, CAP}; }

// The TMA-ring kernels always hold the whole table.  The register-staged ones size it to
// the wave; one-warp CTAs take a smaller cap so that sixteen fit an SM, each checking its
// own simulated block.
const VariantEntry kVariants[SR_CHECK_VARIANTS] = {
    entry<CheckVariant<256, 1024, 3, 2>, 2, kCheckBins>(),
    entry<CheckVariant<128, 512, 4, 3>, 3, kCheckBins>(),
    entry<RegVariant<128, 4, 4>, 4, kCheckTableCap>(),
    entry<RegVariant<64, 4, 8>, 8, kCheckTableCap>(),
    entry<RegVariant<32, 4, 16>, 16, kCheckTableCap / 2>(),
    entry<LeanVariant<4>, 20, kCheckTableCap / 2>(),
    entry<LeanVariant<8>, 20, kCheckTableCap / 2>(),
};
constexpr uint32_t kDefaultVariant = 4;

const VariantEntry& variant_entry(uint32_t v) {
  return kVariants[(v >= 1 && v <= SR_CHECK_VARIANTS ? v : kDefaultVariant) - 1];
}

}  // namespace

uint32_t check_default_variant() { return kDefaultVariant; }
uint32_t check_ctas_per_sm(uint32_t variant) { return variant_entry(variant).ctas_per_sm; }
uint32_t check_table_cap(uint32_t variant) { return variant_entry(variant).table_cap; }

cudaError_t init_check_attributes(uint32_t smem_optin) {
  for (const VariantEntry& v : kVariants) {
    const cudaError_t e = v.init(smem_optin);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t init_kernel_attributes(uint32_t smem_optin) {
  cudaError_t e = init_interp_attributes(smem_optin);
  if (e == cudaSuccess) e = init_check_attributes(smem_optin);
  return e == cudaSuccess ? init_gcheck_attributes(smem_optin) : e;
}

cudaError_t launch_check(const CheckArgs& a, uint32_t variant, uint32_t ctas, cudaStream_t s) {
  return variant_entry(variant).launch(a, ctas, s);
}

}  // namespace sr
