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

// ---------------------------------------------------------------- CTA scan
// In-place exclusive scan of a[0..len) (shared memory) by all NT threads; returns the total.
__device__ uint32_t cta_exclusive_scan(uint32_t* a, uint32_t len, uint32_t* wtot) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t per = (len + NT - 1) / NT;
  const uint32_t b0 = min(len, tid * per), b1 = min(len, b0 + per);
  uint32_t sum = 0;
  for (uint32_t i = b0; i < b1; ++i) sum += a[i];
  uint32_t inc = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(FULL, inc, o);
    if (lane >= (uint32_t)o) inc += v;
  }
  if (lane == 31) wtot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const uint32_t v = lane < NT / 32 ? wtot[lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane < NT / 32) wtot[lane] = x - v;     // exclusive warp offsets
    if (lane == 31) wtot[32] = x;               // total
  }
  __syncthreads();
  uint32_t run = wtot[wid] + inc - sum;
  for (uint32_t i = b0; i < b1; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  const uint32_t total = wtot[32];
  __syncthreads();
  return total;
}

struct Smem {
  unsigned long long* tile;     // T + 2 staged records
  unsigned long long* sorted;   // T
  uint32_t* bins;               // 1 << max key bits
  uint32_t* flags;              // T (or bins) entries for the scans
  uint32_t* touched;            // bitmap over addresses (large-interval path)
  uint32_t* wtot;               // 33 scan words
  uint32_t* misc;               // small broadcast words
};

// Sort the m records rec[0..m) by address into S.sorted; afterwards S.bins[x] is the end
// (exclusive) of address x's run.
__device__ void counting_sort(const Smem& S, const unsigned long long* rec, uint32_t m, uint32_t nb) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t i = tid; i < nb; i += NT) S.bins[i] = 0;
  __syncthreads();
  for (uint32_t i = tid; i < m; i += NT) atomicAdd(&S.bins[rec_addr(rec[i])], 1u);
  __syncthreads();
  cta_exclusive_scan(S.bins, nb, S.wtot);
  for (uint32_t i = tid; i < m; i += NT) {
    const unsigned long long r = rec[i];
    S.sorted[atomicAdd(&S.bins[rec_addr(r)], 1u)] = r;
  }
  __syncthreads();
}

// One complete barrier interval held in shared memory: emit its race entries in
// address order at out[*race_out ...].
__device__ void check_interval(const Smem& S, const unsigned long long* rec, uint32_t m, uint32_t epoch,
                               uint32_t nb, uint4* out, uint32_t& race_out) {
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  if (m <= 32) {
    // warp path: group equal addresses with __match_any_sync
    if (tid < 32) {
      const bool valid = lane < m;
      const unsigned long long r = valid ? rec[lane] : 0ull;
      const uint32_t addr = valid ? rec_addr(r) : 0u;
      const uint32_t grp = __match_any_sync(FULL, valid ? addr : (0x80000000u | lane));
      const bool leader = valid && lane == (uint32_t)(__ffs(grp) - 1);
      bool racy = false;
      uint32_t b = 0, c = 0;
      if (leader) {
        Summ s = summ_empty();
        for (uint32_t g = grp; g; g &= g - 1) summ_add(s, rec[__ffs(g) - 1]);
        racy = summ_race(s, b, c);
      }
      const uint32_t rm = __ballot_sync(FULL, racy);
      uint32_t rank = 0;
      for (uint32_t g = rm; g; g &= g - 1) {
        const uint32_t aj = __shfl_sync(FULL, addr, __ffs(g) - 1);
        rank += aj < addr;
      }
      if (racy) out[race_out + rank] = make_uint4(epoch, addr, b, c);
      race_out += __popc(rm);
      if (tid == 0) S.misc[0] = race_out;
    }
    __syncthreads();
    race_out = S.misc[0];
    __syncthreads();
    return;
  }
  counting_sort(S, rec, m, nb);
  // run heads: summary of [i, end of run) -> racy flag
  for (uint32_t i = tid; i < m; i += NT) {
    const unsigned long long r = S.sorted[i];
    const uint32_t a = rec_addr(r);
    uint32_t f = 0;
    if (i == 0 || rec_addr(S.sorted[i - 1]) != a) {
      Summ s = summ_empty();
      const uint32_t end = S.bins[a];
      for (uint32_t j = i; j < end; ++j) summ_add(s, S.sorted[j]);
      uint32_t b, c;
      f = summ_race(s, b, c);
    }
    S.flags[i] = f;
  }
  __syncthreads();
  // keep the flags: the scan below turns them into output positions
  for (uint32_t i = tid; i < m; i += NT) S.flags[T + i] = S.flags[i];
  __syncthreads();
  const uint32_t total = cta_exclusive_scan(S.flags, m, S.wtot);
  for (uint32_t i = tid; i < m; i += NT) {
    if (!S.flags[T + i]) continue;
    const uint32_t a = rec_addr(S.sorted[i]);
    Summ s = summ_empty();
    const uint32_t end = S.bins[a];
    for (uint32_t j = i; j < end; ++j) summ_add(s, S.sorted[j]);
    uint32_t b = 0, c = 0;
    summ_race(s, b, c);
    out[race_out + S.flags[i]] = make_uint4(epoch, a, b, c);
  }
  race_out += total;
  __syncthreads();
}

// Part of an interval that does not fit one tile: fold its run summaries into the
// per-CTA table (each address once per chunk, so no atomics on the table itself).
__device__ void fold_chunk(const Smem& S, const unsigned long long* rec, uint32_t m, uint32_t nb, uint4* table) {
  const uint32_t tid = threadIdx.x;
  counting_sort(S, rec, m, nb);
  for (uint32_t i = tid; i < m; i += NT) {
    const unsigned long long r = S.sorted[i];
    const uint32_t a = rec_addr(r);
    if (i != 0 && rec_addr(S.sorted[i - 1]) == a) continue;
    Summ s = summ_empty();
    const uint32_t end = S.bins[a];
    for (uint32_t j = i; j < end; ++j) summ_add(s, S.sorted[j]);
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
__device__ void finish_large(const Smem& S, uint32_t epoch, uint32_t nb, uint4* table, uint4* out,
                             uint32_t& race_out) {
  const uint32_t tid = threadIdx.x;
  for (uint32_t a = tid; a < nb; a += NT) {
    uint32_t f = 0;
    if (S.touched[a >> 5] & (1u << (a & 31))) {
      const uint4 o = table[a];
      uint32_t b, c;
      f = summ_race(Summ{o.x, o.y, o.z, o.w}, b, c);
    }
    S.flags[a] = f;
  }
  __syncthreads();
  const uint32_t total = cta_exclusive_scan(S.flags, nb, S.wtot);
  for (uint32_t a = tid; a < nb; a += NT) {          // racy flags re-derived from the table
    if (!(S.touched[a >> 5] & (1u << (a & 31)))) continue;
    const uint4 o = table[a];
    uint32_t b = 0, c = 0;
    if (summ_race(Summ{o.x, o.y, o.z, o.w}, b, c)) out[race_out + S.flags[a]] = make_uint4(epoch, a, b, c);
  }
  __syncthreads();
  race_out += total;
  for (uint32_t i = tid; i < nb / 32 + 1; i += NT) S.touched[i] = 0;
  __syncthreads();
}

__global__ void __launch_bounds__(NT) k_check(CheckArgs A, uint32_t max_bits) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t s_gb, s_li;
  const uint32_t maxnb = 1u << max_bits;
  Smem S;
  unsigned char* p = smem;
  S.tile = reinterpret_cast<unsigned long long*>(p); p += (T + 2) * 8;
  S.sorted = reinterpret_cast<unsigned long long*>(p); p += T * 8;
  S.bins = reinterpret_cast<uint32_t*>(p); p += maxnb * 4;
  S.flags = reinterpret_cast<uint32_t*>(p); p += max(2 * T, maxnb) * 4;
  S.touched = reinterpret_cast<uint32_t*>(p); p += (maxnb / 32 + 1) * 4;
  S.wtot = reinterpret_cast<uint32_t*>(p); p += 36 * 4;
  S.misc = reinterpret_cast<uint32_t*>(p);
  uint4* table = A.scratch + (size_t)blockIdx.x * kScratchWords;
  const uint32_t tid = threadIdx.x;
  uint32_t phase = 0;
  if (tid == 0) mbar_init(&mbar);
  for (uint32_t i = tid; i < maxnb / 32 + 1; i += NT) S.touched[i] = 0;
  __syncthreads();

  for (;;) {
    __syncthreads();                                 // every thread is done with s_gb / s_li
    if (tid == 0) {
      const uint32_t gb = A.gb0 + atomicAdd(A.work_head, 1u);
      s_gb = gb;
      if (gb < A.gb1) {
        uint32_t lo = 0, hi = A.nlaunches - 1;     // last launch with block_base <= gb
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (A.launches[mid].block_base <= gb) lo = mid; else hi = mid - 1;
        }
        s_li = lo;
      }
    }
    __syncthreads();
    const uint32_t gb = s_gb;
    if (gb >= A.gb1) break;
    const uint32_t n = A.blocks[gb].n_log;
    if (n == 0) continue;
    const LaunchDev* L = A.launches + s_li;
    const uint32_t nb = 1u << L->key_bits;
    unsigned long long* region = A.log + L->log_base + (unsigned long long)(gb - L->block_base) * L->log_cap;
    uint4* out = reinterpret_cast<uint4*>(region);
    uint32_t race_out = 0, pos = 0;
    bool large = false;
    uint32_t large_epoch = 0;
    bool failed = false;
    while (pos < n && !failed) {
      const uint32_t off = pos & 1u, cnt = min(T, n - pos);
      const uint32_t nload = (cnt + off + 1u) & ~1u;
      if (tid == 0) bulk_load(S.tile, region + (pos - off), nload * 8u, &mbar);
      const bool ok = mbar_wait(&mbar, phase, A.spin_limit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {                   // agree on a (bounded) wait that gave up
        failed = true;
        break;
      }
      const unsigned long long* rec = S.tile + off;
      uint32_t s = 0;
      while (s < cnt) {
        const uint32_t e = rec_epoch(rec[s]);
        uint32_t lo = s, hi = cnt;                   // first index with a later epoch
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (rec_epoch(rec[mid]) <= e) lo = mid + 1; else hi = mid;
        }
        const uint32_t t_end = lo;
        const bool complete = t_end < cnt || pos + cnt == n;
        if (large && e == large_epoch) {
          fold_chunk(S, rec + s, t_end - s, nb, table);
          if (complete) {
            finish_large(S, e, nb, table, out, race_out);
            large = false;
          }
          s = t_end;
          continue;
        }
        if (!complete) {
          if (s > 0) break;                          // restage from the start of this interval
          large = true;                              // interval larger than a tile
          large_epoch = e;
          fold_chunk(S, rec, t_end, nb, table);
          s = t_end;
          continue;
        }
        check_interval(S, rec + s, t_end - s, e, nb, out, race_out);
        s = t_end;
      }
      pos += s;
      __syncthreads();                               // tile fully consumed before it is restaged
    }
    if (tid == 0) {
      A.blocks[gb].n_race = race_out;
      if (failed) atomicOr(A.error_flag, 1u);
    }
    if (failed) break;
  }
}

}  // namespace

uint32_t check_smem_bytes_bits(uint32_t max_bits) {
  const uint32_t maxnb = 1u << max_bits;
  return (T + 2) * 8 + T * 8 + maxnb * 4 + (2 * T > maxnb ? 2 * T : maxnb) * 4 + (maxnb / 32 + 1) * 4 + 36 * 4 + 16;
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
  k_check<<<ctas, NT, check_smem_bytes_bits(a.max_key_bits), s>>>(a, a.max_key_bits);
  return cudaGetLastError();
}

}  // namespace sr
