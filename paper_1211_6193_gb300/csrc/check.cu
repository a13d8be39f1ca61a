// check.cu - race check of the access logs (segmented sort + run scan).
//
// Sec. 3.1 of the paper: a race is two threads accessing the same shared location
// with no synchronisation point in between, at least one access writing; the access
// history is cleared at every __syncthreads().  The interpreter wrote one 8-byte
// record per shared access into a per-block log region, records of a barrier interval
// contiguous and intervals in order.  This kernel groups each interval's records by
// word address (a counting sort of the interval staged in shared memory, or a warp
// __match_any_sync for intervals of at most 32 records) and reduces every group to a
// summary: the two smallest distinct tids per access kind, and the pc range.  Those
// summaries decide the conflict classes and the smallest conflicting pair exactly (a
// lexicographically smallest conflicting pair always uses one of the two smallest tids
// of each kind involved).  Race entries (epoch, addr, pair, class|pcs; 16 bytes) are
// written back in address order at the front of the block's region; every entry
// consumes at least two records, so the writes never reach records not yet read.
//
// Records are staged with TMA bulk copies (cp.async.bulk + mbarrier).  Intervals
// larger than one tile are folded chunk by chunk into a per-CTA summary table in
// global memory indexed by address.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t NT = kCheckThreads;
constexpr uint32_t T = kCheckTile;
constexpr uint32_t NB = kCheckBins;
constexpr uint32_t NBUF = kCheckBuffers;
constexpr uint32_t NONE = 0xFFFFu;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- summaries
// r/w/a: two smallest distinct tids of that kind (low 16 bits smallest, NONE = absent);
// pc: low 16 bits lowest pc, high 16 bits highest pc.
struct Summ { uint32_t r, w, a, pc; };

__device__ __forceinline__ Summ summ_empty() { return Summ{0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, NONE}; }

__device__ __forceinline__ uint32_t min2_add(uint32_t m, uint32_t t) {
  const uint32_t m1 = m & 0xFFFFu, m2 = m >> 16;
  if (t == m1 || t == m2) return m;
  if (t < m1) return m1 << 16 | t;
  if (t < m2) return t << 16 | m1;
  return m;
}
__device__ __forceinline__ uint32_t min2_merge(uint32_t m, uint32_t o) {
  if ((o & 0xFFFFu) != NONE) m = min2_add(m, o & 0xFFFFu);
  if ((o >> 16) != NONE) m = min2_add(m, o >> 16);
  return m;
}
__device__ __forceinline__ void summ_add(Summ& s, unsigned long long rec) {
  const uint32_t t = rec_tid(rec), k = rec_kind(rec), pc = rec_pc(rec);
  if (k == K_R) s.r = min2_add(s.r, t);
  else if (k == K_W) s.w = min2_add(s.w, t);
  else s.a = min2_add(s.a, t);
  const uint32_t lo = min(s.pc & 0xFFFFu, pc), hi = max(s.pc >> 16, pc);
  s.pc = hi << 16 | lo;
}
__device__ __forceinline__ void summ_merge(Summ& s, const Summ& o) {
  s.r = min2_merge(s.r, o.r);
  s.w = min2_merge(s.w, o.w);
  s.a = min2_merge(s.a, o.a);
  const uint32_t lo = min(s.pc & 0xFFFFu, o.pc & 0xFFFFu), hi = max(s.pc >> 16, o.pc >> 16);
  s.pc = hi << 16 | lo;
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

// ---------------------------------------------------------------- CTA scans
// Exclusive scan of one value per thread over the CTA; returns the prefix, total in *tot.
__device__ uint32_t cta_scan_value(uint32_t v, uint32_t* wtot, uint32_t* tot) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += y;
  }
  if (lane == 31) wtot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t x0 = lane < NT / 32 ? wtot[lane] : 0u;
    uint32_t x = x0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane < NT / 32) wtot[lane] = x - x0;
    if (lane == 31) wtot[32] = x;
  }
  __syncthreads();
  const uint32_t r = wtot[wid] + inc - v;
  *tot = wtot[32];
  __syncthreads();
  return r;
}

// In-place exclusive scan of a[0..len) (shared memory); returns the total.
__device__ uint32_t cta_exclusive_scan(uint32_t* a, uint32_t len, uint32_t* wtot) {
  const uint32_t per = (len + NT - 1) / NT;
  const uint32_t b0 = min(len, threadIdx.x * per), b1 = min(len, b0 + per);
  uint32_t sum = 0;
  for (uint32_t i = b0; i < b1; ++i) sum += a[i];
  uint32_t total;
  uint32_t run = cta_scan_value(sum, wtot, &total);
  for (uint32_t i = b0; i < b1; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  __syncthreads();
  return total;
}

constexpr uint32_t MAXSEG = 256;   // barrier intervals handled per staged tile

struct Smem {
  unsigned long long* tile[2];  // T + 2 staged records each (NBUF buffers)
  unsigned long long* sorted;   // T
  uint16_t* sbin;               // T: bin of sorted[i]
  uint32_t* bins;               // NB
  uint32_t* flags;              // 2T
  uint16_t* segidx;             // T: interval of each tile record
  uint32_t* seg_start;          // MAXSEG + 1 (record index of each interval of the tile)
  uint32_t* seg_lo;             // MAXSEG: lowest address of the interval
  uint32_t* seg_hi;             // MAXSEG
  uint32_t* seg_off;            // MAXSEG: first bin of the interval
  uint32_t* touched;            // NB / 32 + 1 bitmap (large intervals)
  uint32_t* wtot;               // 36 scan words
  uint32_t* misc;               // broadcast words
};

// Counting sort of records rec[0..m) (intervals s0..s0+nseg-1 of the tile, starting at
// record seg_start[s0]) by (interval, address): each interval owns the bins of its own
// address range, so the sorted order is exactly (epoch, address).  Returns the number
// of intervals that fit the bin budget (at least one).  Afterwards sorted/sbin hold the
// records and their bins, bins[b] is the end of bin b's run.
__device__ uint32_t sort_intervals(const Smem& S, const unsigned long long* tile, uint32_t s0, uint32_t nseg,
                                   uint32_t& m_out) {
  const uint32_t tid = threadIdx.x;
  const uint32_t base = S.seg_start[s0], end = S.seg_start[s0 + nseg];
  for (uint32_t i = tid; i < nseg; i += NT) { S.seg_lo[s0 + i] = 0xFFFFFFFFu; S.seg_hi[s0 + i] = 0; }
  __syncthreads();
  // per-interval address range: a warp whose 32 records share one interval reduces them
  // first (one atomic pair per warp instead of per record)
  for (uint32_t i0 = base + (tid & ~31u); i0 < end; i0 += NT) {
    const uint32_t i = i0 + (tid & 31u);
    const bool valid = i < end;
    uint32_t sg = 0, a = 0;
    if (valid) {
      sg = S.segidx[i];
      a = rec_addr(tile[i]);
    }
    const uint32_t sg0 = __shfl_sync(FULL, sg, 0);
    if (__all_sync(FULL, !valid || sg == sg0)) {
      const uint32_t mn = __reduce_min_sync(FULL, valid ? a : 0xFFFFFFFFu);
      const uint32_t mx = __reduce_max_sync(FULL, valid ? a : 0u);
      if ((tid & 31u) == 0) {
        atomicMin(&S.seg_lo[sg0], mn);
        atomicMax(&S.seg_hi[sg0], mx);
      }
    } else if (valid) {
      atomicMin(&S.seg_lo[sg], a);
      atomicMax(&S.seg_hi[sg], a);
    }
  }
  __syncthreads();
  // bin offsets: a prefix of the intervals whose ranges fit NB bins together (one warp);
  // a single range never exceeds NB, so at least one interval is always kept
  if (tid < 32) {
    uint32_t run = 0, kept = 0;
    for (uint32_t c = 0; c < nseg; c += 32) {
      const uint32_t i = c + tid;
      const uint32_t r = i < nseg ? S.seg_hi[s0 + i] - S.seg_lo[s0 + i] + 1 : 0u;
      uint32_t inc = r;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (tid >= (uint32_t)o) inc += y;
      }
      const bool fits = i < nseg && run + inc <= NB;   // a prefix of the lanes (inc grows)
      const uint32_t nf = __popc(__ballot_sync(FULL, fits));
      if (fits) S.seg_off[s0 + i] = run + inc - r;
      if (nf) run += __shfl_sync(FULL, inc, nf - 1);
      kept += nf;
      if (nf < 32) break;
    }
    if (tid == 0) { S.misc[0] = kept; S.misc[1] = run; }
  }
  __syncthreads();
  const uint32_t kept = S.misc[0], nb = S.misc[1];
  const uint32_t mend = S.seg_start[s0 + kept];
  const uint32_t m = mend - base;
  for (uint32_t b = tid; b < nb; b += NT) S.bins[b] = 0;
  __syncthreads();
  for (uint32_t i = base + tid; i < mend; i += NT) {
    const uint32_t sg = S.segidx[i];
    const uint32_t b = S.seg_off[sg] + rec_addr(tile[i]) - S.seg_lo[sg];
    S.flags[T + (i - base)] = b;
    atomicAdd(&S.bins[b], 1u);
  }
  __syncthreads();
  cta_exclusive_scan(S.bins, nb, S.wtot);
  for (uint32_t i = tid; i < m; i += NT) {
    const uint32_t b = S.flags[T + i];
    const uint32_t pos = atomicAdd(&S.bins[b], 1u);
    S.sorted[pos] = tile[base + i];
    S.sbin[pos] = (uint16_t)b;
  }
  __syncthreads();
  m_out = m;
  return kept;
}

__device__ __forceinline__ Summ run_summary(const Smem& S, uint32_t i, uint32_t end) {
  Summ s = summ_empty();
  for (uint32_t j = i; j < end; ++j) summ_add(s, S.sorted[j]);
  return s;
}

// Race entries of sorted intervals, in (epoch, address) order, at out[race_out ...].
__device__ void emit_races(const Smem& S, uint32_t m, uint4* out, uint32_t& race_out) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < m; i += NT) {
    uint32_t f = 0;
    if (i == 0 || S.sbin[i] != S.sbin[i - 1]) {
      // cheap pass: one thread only, or reads only / atomics only, cannot race
      const uint32_t end = S.bins[S.sbin[i]];
      uint32_t tmin = 0xFFFFu, tmax = 0, kinds = 0;
      for (uint32_t j = i; j < end; ++j) {
        const unsigned long long r = S.sorted[j];
        const uint32_t t = rec_tid(r);
        tmin = min(tmin, t);
        tmax = max(tmax, t);
        kinds |= 1u << rec_kind(r);
      }
      const bool maybe = tmin != tmax && ((kinds & (1u << K_W)) || kinds == ((1u << K_R) | (1u << K_A)));
      if (maybe) {
        uint32_t b, c;
        f = summ_race(run_summary(S, i, end), b, c);
      }
    }
    S.flags[i] = f;
    S.flags[T + i] = f;
  }
  __syncthreads();
  const uint32_t total = cta_exclusive_scan(S.flags, m, S.wtot);
  for (uint32_t i = tid; i < m; i += NT) {
    if (!S.flags[T + i]) continue;
    const unsigned long long r = S.sorted[i];
    uint32_t b = 0, c = 0;
    summ_race(run_summary(S, i, S.bins[S.sbin[i]]), b, c);
    out[race_out + S.flags[i]] = make_uint4(rec_epoch(r), rec_addr(r), b, c);
  }
  race_out += total;
  __syncthreads();
}

// A chunk of an interval larger than a tile: fold run summaries into the per-CTA table.
__device__ void fold_sorted(const Smem& S, uint32_t m, uint4* table) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < m; i += NT) {
    if (i != 0 && S.sbin[i] == S.sbin[i - 1]) continue;
    Summ s = run_summary(S, i, S.bins[S.sbin[i]]);
    const uint32_t a = rec_addr(S.sorted[i]);
    const uint32_t bit = 1u << (a & 31);
    if (atomicOr(&S.touched[a >> 5], bit) & bit) {
      const uint4 o = table[a];
      summ_merge(s, Summ{o.x, o.y, o.z, o.w});
    }
    table[a] = make_uint4(s.r, s.w, s.a, s.pc);
  }
  __threadfence_block();
  __syncthreads();
}

// End of a large interval: races of every touched address, in address order.
__device__ void finish_large(const Smem& S, uint32_t epoch, uint4* table, uint4* out, uint32_t& race_out) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t a = tid; a < NB; a += NT) {
    uint32_t f = 0;
    if (S.touched[a >> 5] & (1u << (a & 31))) {
      const uint4 o = table[a];
      uint32_t b, c;
      f = summ_race(Summ{o.x, o.y, o.z, o.w}, b, c);
    }
    S.bins[a] = f;
  }
  __syncthreads();
  const uint32_t total = cta_exclusive_scan(S.bins, NB, S.wtot);
  for (uint32_t a = tid; a < NB; a += NT) {          // racy flags re-derived from the table
    if (!(S.touched[a >> 5] & (1u << (a & 31)))) continue;
    const uint4 o = table[a];
    uint32_t b = 0, c = 0;
    if (summ_race(Summ{o.x, o.y, o.z, o.w}, b, c)) out[race_out + S.bins[a]] = make_uint4(epoch, a, b, c);
  }
  __syncthreads();
  race_out += total;
  for (uint32_t i = tid; i < NB / 32 + 1; i += NT) S.touched[i] = 0;
  __syncthreads();
}

// Interval starts of tile[0..cnt) (records are in interval order): at most MAXSEG are
// kept; returns their number and sets cnt_eff to the end of the last kept interval.
__device__ uint32_t find_intervals(const Smem& S, const unsigned long long* tile, uint32_t cnt, uint32_t& cnt_eff) {
  constexpr uint32_t PER = (T + NT - 1) / NT;
  const uint32_t i0 = threadIdx.x * PER;
  uint32_t f = 0, c = 0;
  for (uint32_t j = 0; j < PER; ++j) {
    const uint32_t i = i0 + j;
    const bool st = i < cnt && (i == 0 || rec_epoch(tile[i]) != rec_epoch(tile[i - 1]));
    f |= (uint32_t)st << j;
    c += st;
  }
  uint32_t total;
  uint32_t o = cta_scan_value(c, S.wtot, &total);
  for (uint32_t j = 0; j < PER; ++j) {
    if (f >> j & 1u) {
      if (o <= MAXSEG) S.seg_start[o] = i0 + j;
      ++o;
    }
    if (i0 + j < cnt) S.segidx[i0 + j] = (uint16_t)min(o - 1, 0xFFFFu);   // interval of record i0 + j
  }
  __syncthreads();
  const uint32_t nseg = min(total, MAXSEG);
  if (total <= MAXSEG && threadIdx.x == 0) S.seg_start[nseg] = cnt;
  __syncthreads();
  cnt_eff = S.seg_start[nseg];
  return nseg;
}

__global__ void __launch_bounds__(NT, kCheckCtasPerSm) k_check(CheckArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t s_next;
  Smem S;
  unsigned char* p = smem;
  S.tile[0] = reinterpret_cast<unsigned long long*>(p); p += (T + 2) * 8;
  S.tile[1] = NBUF == 2 ? reinterpret_cast<unsigned long long*>(p) : S.tile[0];
  p += (NBUF - 1) * (T + 2) * 8;
  S.sorted = reinterpret_cast<unsigned long long*>(p); p += T * 8;
  S.sbin = reinterpret_cast<uint16_t*>(p); p += T * 2;
  S.bins = reinterpret_cast<uint32_t*>(p); p += NB * 4;
  S.flags = reinterpret_cast<uint32_t*>(p); p += 2 * T * 4;
  S.segidx = reinterpret_cast<uint16_t*>(p); p += T * 2;
  S.seg_start = reinterpret_cast<uint32_t*>(p); p += (MAXSEG + 4) * 4;
  S.seg_lo = reinterpret_cast<uint32_t*>(p); p += MAXSEG * 4;
  S.seg_hi = reinterpret_cast<uint32_t*>(p); p += MAXSEG * 4;
  S.seg_off = reinterpret_cast<uint32_t*>(p); p += MAXSEG * 4;
  S.touched = reinterpret_cast<uint32_t*>(p); p += (NB / 32 + 1) * 4;
  S.wtot = reinterpret_cast<uint32_t*>(p); p += 36 * 4;
  S.misc = reinterpret_cast<uint32_t*>(p);
  uint4* table = A.scratch + (size_t)blockIdx.x * kScratchWords;
  const uint32_t tid = threadIdx.x;
  uint32_t phases = 0;                           // bit b: mbarrier parity of buffer b
  if (tid == 0) { mbar_init(&mbar[0]); mbar_init(&mbar[1]); }
  for (uint32_t i = tid; i < NB / 32 + 1; i += NT) S.touched[i] = 0;

  // next block with a non-empty log, and the start of its staging into buffer `buf`
  auto claim = [&](uint32_t buf) {
    if (tid == 0) {
      uint32_t gb;
      for (;;) {
        gb = A.gb0 + atomicAdd(A.work_head, 1u);
        if (gb >= A.gb1 || A.blocks[gb].n_log) break;
      }
      if (gb < A.gb1) {
        uint32_t lo = 0, hi = A.nlaunches - 1;
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (A.launches[mid].block_base <= gb) lo = mid; else hi = mid - 1;
        }
        const LaunchDev* L = A.launches + lo;
        const unsigned long long* region = A.log + L->log_base + (unsigned long long)(gb - L->block_base) * L->log_cap;
        const uint32_t n = A.blocks[gb].n_log, cnt = min(T, n);
        bulk_load(S.tile[buf], region, ((cnt + 1u) & ~1u) * 8u, &mbar[buf]);
        S.misc[8] = lo;
      }
      s_next = gb;
    }
    __syncthreads();
    return s_next;
  };

  uint32_t cur = 0;
  uint32_t gb = claim(cur);
  while (gb < A.gb1) {
    const LaunchDev* L = A.launches + S.misc[8];
    unsigned long long* region = A.log + L->log_base + (unsigned long long)(gb - L->block_base) * L->log_cap;
    uint4* out = reinterpret_cast<uint4*>(region);
    const uint32_t n = A.blocks[gb].n_log;
    uint32_t pos = 0, race_out = 0, large_epoch = 0, next_gb = A.gb1;
    bool large = false, failed = false, prefetched = false;
    while (pos < n) {
      const bool ok = mbar_wait(&mbar[cur], (phases >> cur) & 1u, A.spin_limit);
      phases ^= 1u << cur;
      if (__syncthreads_or(!ok)) { failed = true; break; }
      const uint32_t off = pos & 1u, cnt = min(T, n - pos);
      const unsigned long long* tile = S.tile[cur] + off;
      const bool last_tile = pos + cnt == n;
      if (NBUF == 2 && last_tile && !prefetched) {   // stage the next block while this one is checked
        next_gb = claim(cur ^ 1u);
        prefetched = true;
      }
      uint32_t cnt_eff;
      const uint32_t nseg = find_intervals(S, tile, cnt, cnt_eff);
      // the last interval of a tile may continue in the next tile unless the block ends here
      const bool tail_open = !last_tile && cnt_eff == cnt;
      uint32_t sidx = 0, consumed = 0;
      if (large && rec_epoch(tile[0]) != large_epoch) {   // it ended exactly at the last tile boundary
        finish_large(S, large_epoch, table, out, race_out);
        large = false;
      }
      if (large) {                               // the first interval continues the large one
        uint32_t m;
        sort_intervals(S, tile, 0, 1, m);
        fold_sorted(S, m, table);
        if (!(nseg == 1 && tail_open)) {
          finish_large(S, large_epoch, table, out, race_out);
          large = false;
        }
        sidx = 1;
        consumed = S.seg_start[1];
      }
      const uint32_t ncomplete = tail_open ? nseg - 1 : nseg;
      while (!large && sidx < ncomplete) {
        uint32_t m;
        const uint32_t kept = sort_intervals(S, tile, sidx, ncomplete - sidx, m);
        emit_races(S, m, out, race_out);
        sidx += kept;
        consumed = S.seg_start[sidx];
      }
      if (!large && sidx == 0 && tail_open) {     // one interval fills the whole tile
        large = true;
        large_epoch = rec_epoch(tile[0]);
        uint32_t m;
        sort_intervals(S, tile, 0, 1, m);
        fold_sorted(S, m, table);
        consumed = cnt;
      }
      pos += consumed;
      if (pos < n) {                             // restage the rest of this block
        if (tid == 0) {
          const uint32_t o2 = pos & 1u, c2 = min(T, n - pos);
          bulk_load(S.tile[cur], region + (pos - o2), ((c2 + o2 + 1u) & ~1u) * 8u, &mbar[cur]);
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      A.blocks[gb].n_race = race_out;
      if (failed) atomicOr(A.error_flag, 1u);
    }
    if (failed) break;
    if (!prefetched) next_gb = claim(NBUF == 2 ? cur ^ 1u : 0u);
    gb = next_gb;
    if (NBUF == 2) cur ^= 1u;
    __syncthreads();
  }
}

}  // namespace

uint32_t check_smem_bytes() {
  return NBUF * (T + 2) * 8 + T * 8 + T * 2 + NB * 4 + 2 * T * 4 + T * 2 + (MAXSEG + 4) * 4 + 3 * MAXSEG * 4 +
         (NB / 32 + 1) * 4 + 36 * 4 + 64;
}

cudaError_t init_check_attributes(uint32_t smem_optin) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_check);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_check, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(smem_optin - (uint32_t)fa.sharedSizeBytes));
}

cudaError_t init_kernel_attributes(uint32_t smem_optin) {
  cudaError_t e = init_interp_attributes(smem_optin);
  return e == cudaSuccess ? init_check_attributes(smem_optin) : e;
}

cudaError_t launch_check(const CheckArgs& a, uint32_t ctas, cudaStream_t s) {
  k_check<<<ctas, NT, check_smem_bytes(), s>>>(a);
  return cudaGetLastError();
}

}  // namespace sr
