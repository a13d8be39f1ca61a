// gcheck.cu - race check of global memory (optional, sr_opts.check_global).
//
// Sec. 3.1 defines a race as two threads touching one location with no synchronisation
// point between them, at least one writing; the paper applies it to shared memory.  Applied
// to global words it gives three kinds of race, all decided here from one grouping of the
// global accesses by word:
//   - inside a block's barrier interval (like the shared check)      -> SR_REP_GLOBAL_RACE;
//   - between blocks of one launch: nothing but the end of the kernel call orders them
//     (Sec. 2), so any two accesses from different blocks, one writing -> SR_REP_GLOBAL_BLOCKS;
//   - between launches that no stream order or event wait orders (Sec. 3, streams and
//     events)                                                          -> SR_REP_GLOBAL_LAUNCHES.
//
// The interpreter appends a 16-byte record per in-bounds global load or store to its
// block's region (epoch order inside a block).  Per wave:
//   1. gather   the blocks' records into one array, blocks in (program, launch, block) order;
//   2. sort     stably by word address: an LSD radix sort with 8-bit digits, onesweep style -
//               one upsweep pass builds the digit histograms of every pass, then each pass
//               is one kernel in which a CTA ranks a tile staged in shared memory by a TMA
//               bulk copy, learns the tile's offsets from its predecessors by decoupled
//               look-back (bounded waits), and writes the tile out digit by digit.  Stable,
//               so the records of one word keep (program, launch, block, epoch) order;
//   3. scan     each run of one (program, word) in one pass: sub-runs of one (block, epoch)
//               give the interval check, of one launch the check between blocks, and the
//               run's launches the check between unordered launches.  Every word keeps the
//               two smallest distinct tids (blocks) of each access kind and the pc range,
//               which decide the classes and the smallest conflicting pair exactly;
//   4. order    the report entries by (block, epoch, kind, word) with the same radix sort,
//               for the canonical merge in compact.cu.
#include <algorithm>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t RS_T = 256;                       // threads of a sort CTA
constexpr uint32_t RS_WARPS = RS_T / 32;
constexpr uint32_t RS_ITEMS = 8;                     // records per thread and tile
constexpr uint32_t RS_TILE = RS_T * RS_ITEMS;        // 2048 records per tile
constexpr uint32_t RADIX = 256;
constexpr uint32_t MAX_PASSES = 12;
constexpr unsigned long long ST_AGG = 1ull << 62;    // tile status: its own count is known
constexpr unsigned long long ST_INC = 1ull << 63;    // tile status: its inclusive prefix is known
constexpr unsigned long long ST_VAL = ST_AGG - 1;
constexpr uint32_t NONE16 = 0xFFFFu;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
// A look-back status word carries its whole payload (flag and count), and nothing else is
// read on the strength of it, so relaxed GPU-scope accesses suffice.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
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

// ---------------------------------------------------------------- record types and digits
struct Rec16 { uint4 a; };                 // a global-log record
struct Rec32 { uint4 a, b; };              // a report entry (see GrunArgs)

// global-log records: by word address (x), low byte first
struct AddrDigit {
  __device__ __forceinline__ uint32_t operator()(const Rec16& r, uint32_t pass) const {
    return (r.a.x >> (8u * pass)) & 0xFFu;
  }
};
// report entries: by (block, epoch << 2 | kind - 9, word), least significant word first
struct EntryDigit {
  __device__ __forceinline__ uint32_t operator()(const Rec32& r, uint32_t pass) const {
    const uint32_t w = pass < 4 ? r.a.z : pass < 8 ? r.a.y : r.a.x;
    return (w >> (8u * (pass & 3u))) & 0xFFu;
  }
};

// ---------------------------------------------------------------- exclusive scan of counts
// Per-block counts c[gb0 .. gb1) -> offsets off[gb - gb0] (from 0) and the total, in three
// kernels: chunk sums, one CTA over the chunk sums, offsets.
constexpr uint32_t SC_T = 1024, SC_PER = 4, SC_CHUNK = SC_T * SC_PER;

__device__ unsigned long long cta_inclusive(unsigned long long v, unsigned long long* wsum) {
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, v, o);
    if (lane >= (uint32_t)o) v += y;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long x = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  const unsigned long long r = v + (wid ? wsum[wid - 1] : 0ull);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SC_T) k_count_chunks(const uint32_t* c, uint32_t gb0, uint32_t gb1,
                                                       unsigned long long* partials) {
  __shared__ unsigned long long wsum[32];
  const uint32_t base = gb0 + blockIdx.x * SC_CHUNK + threadIdx.x * SC_PER;
  unsigned long long s = 0;
  for (uint32_t i = 0; i < SC_PER; ++i)
    if (base + i < gb1) s += c[base + i];
  const unsigned long long inc = cta_inclusive(s, wsum);
  if (threadIdx.x == SC_T - 1) partials[blockIdx.x] = inc;
}

__global__ void __launch_bounds__(SC_T) k_count_scan(unsigned long long* partials, uint32_t nchunks,
                                                     unsigned long long* total) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long s_tot;
  unsigned long long carry = 0;
  for (uint32_t b = 0; b < nchunks; b += SC_T) {
    const uint32_t i = b + threadIdx.x;
    const unsigned long long v = i < nchunks ? partials[i] : 0ull;
    const unsigned long long inc = cta_inclusive(v, wsum);
    if (i < nchunks) partials[i] = carry + inc - v;
    if (threadIdx.x == SC_T - 1) s_tot = inc;
    __syncthreads();
    carry += s_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(SC_T) k_count_offsets(const uint32_t* c, uint32_t gb0, uint32_t gb1,
                                                        const unsigned long long* partials,
                                                        unsigned long long* off) {
  __shared__ unsigned long long wsum[32];
  const uint32_t base = gb0 + blockIdx.x * SC_CHUNK + threadIdx.x * SC_PER;
  uint32_t v[SC_PER];
  unsigned long long s = 0;
  for (uint32_t i = 0; i < SC_PER; ++i) {
    v[i] = base + i < gb1 ? c[base + i] : 0u;
    s += v[i];
  }
  unsigned long long run = cta_inclusive(s, wsum) - s + partials[blockIdx.x];
  for (uint32_t i = 0; i < SC_PER; ++i) {
    if (base + i < gb1) off[base + i - gb0] = run;
    run += v[i];
  }
}

// ---------------------------------------------------------------- 1. gather
// One warp per block: its records from its region to their place in the wave's array.
__global__ void __launch_bounds__(256) k_ggather(const LaunchDev* launches, uint32_t li0, uint32_t li1,
                                                 uint32_t gb0, uint32_t gb1, const uint4* glog,
                                                 const uint32_t* glog_n, const unsigned long long* off,
                                                 uint4* out, unsigned long long cap, uint32_t* err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t gb = gb0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gb < gb1; gb += nwarps) {
    const uint32_t n = glog_n[gb];
    if (!n) continue;
    uint32_t lo = li0, hi = li1 - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (launches[mid].block_base <= gb) lo = mid; else hi = mid - 1;
    }
    const LaunchDev& L = launches[lo];
    // (debug build: the block's records fit its region and the gathered array)
    if (!dbg_ok(n <= L.glog_cap && off[gb - gb0] + n <= cap, err, kErrBounds)) continue;
    const uint4* src = glog + L.glog_base + (unsigned long long)(gb - L.block_base) * L.glog_cap;
    uint4* dst = out + off[gb - gb0];
    for (uint32_t i = lane; i < n; i += 32) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------- 2. radix sort
// Digit histograms of every pass in one read of the records.  Each warp reads UP_ITEMS rows
// of 32 consecutive records; per pass and row, a digit that all 32 lanes share (the upper
// digits of nearly sorted input) is counted by one shared atomic, other rows by one atomic
// per lane.
constexpr uint32_t UP_ITEMS = 8;
template <class Rec, class Digit>
__global__ void __launch_bounds__(RS_T) k_rs_upsweep(const Rec* in, const unsigned long long* n_ptr,
                                                     unsigned long long cap, uint32_t npasses,
                                                     unsigned long long* hist) {
  __shared__ uint32_t h[MAX_PASSES * RADIX];
  for (uint32_t i = threadIdx.x; i < npasses * RADIX; i += RS_T) h[i] = 0;
  __syncthreads();
  const unsigned long long n = min(*n_ptr, cap);
  const uint32_t lane = threadIdx.x & 31;
  constexpr uint32_t CHUNK = RS_T * UP_ITEMS;
  const unsigned long long stride = (unsigned long long)gridDim.x * CHUNK;
  for (unsigned long long base = (unsigned long long)blockIdx.x * CHUNK + (threadIdx.x >> 5) * (32 * UP_ITEMS);
       base < n; base += stride) {
    Rec r[UP_ITEMS];
#pragma unroll
    for (uint32_t j = 0; j < UP_ITEMS; ++j) {
      const unsigned long long i = base + 32u * j + lane;
      r[j] = i < n ? in[i] : Rec{};
    }
    for (uint32_t p = 0; p < npasses; ++p) {
#pragma unroll
      for (uint32_t j = 0; j < UP_ITEMS; ++j) {
        const unsigned long long i0 = base + 32u * j;
        if (i0 >= n) break;                                  // (warp-uniform)
        const bool valid = i0 + lane < n;
        const uint32_t d = Digit()(r[j], p);
        const uint32_t lo = __reduce_min_sync(FULL, valid ? d : RADIX);
        const uint32_t hi = __reduce_max_sync(FULL, valid ? d : 0u);
        if (lo == hi) {
          if (lane == 0) atomicAdd(&h[p * RADIX + lo], (uint32_t)min(32ull, n - i0));
        } else if (valid) {
          atomicAdd(&h[p * RADIX + d], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < npasses * RADIX; i += RS_T)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// Per pass, digit counts -> exclusive digit offsets (one CTA of RADIX threads).
__global__ void __launch_bounds__(RADIX) k_rs_bins(unsigned long long* hist, uint32_t npasses) {
  __shared__ unsigned long long wsum[RADIX / 32];
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint32_t p = 0; p < npasses; ++p) {
    const unsigned long long v = hist[p * RADIX + threadIdx.x];
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (uint32_t w = 0; w < wid; ++w) before += wsum[w];
    hist[p * RADIX + threadIdx.x] = before + x - v;
    __syncthreads();
  }
}

// One pass of the stable LSD radix sort (onesweep): persistent CTAs claim tiles in order from
// a counter, so every tile's predecessors are claimed by running CTAs and the look-back ends
// (a CTA also holds the tile it prefetches, but that one comes after its current tile, so the
// lowest unfinished tile is always some CTA's current tile).
// status[tile * RADIX + d] holds ST_AGG | the tile's count of digit d, then ST_INC | the count
// of digit d in tiles 0..tile (zero: not yet known); it is cleared before every pass.
// Two tile buffers: while a tile is ranked, placed and written from one, the CTA's next tile
// streams into the other by a TMA bulk copy.  The tile's records are held in registers after
// ranking, so it is placed in digit order in its own buffer.
// (one thread) claim the next tile, and start its copy into `dst` if it exists
template <class Rec>
__device__ __forceinline__ void claim_tile(const Rec* in, Rec* dst, unsigned long long n, unsigned long long ntiles,
                                           uint32_t* tile_ctr, uint32_t* s_tile, unsigned long long* bar) {
  const uint32_t t = atomicAdd(tile_ctr, 1u);
  *s_tile = t;
  if (t < ntiles) {
    const unsigned long long t0 = (unsigned long long)t * RS_TILE;
    const uint32_t tn = (uint32_t)min((unsigned long long)RS_TILE, n - t0);
    // generic-proxy accesses to the buffer (its last write-out) before the async-proxy copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bulk_load(dst, in + t0, tn * (uint32_t)sizeof(Rec), bar);
  }
}

template <class Rec, class Digit>
__global__ void __launch_bounds__(RS_T, sizeof(Rec) == 16 ? 3 : 1)
    k_rs_pass(const Rec* __restrict__ in, Rec* __restrict__ out, const unsigned long long* n_ptr,
              unsigned long long cap, uint32_t pass, const unsigned long long* bins, unsigned long long* status,
              uint32_t* tile_ctr, uint32_t* err, uint32_t spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  Rec* const buf0 = reinterpret_cast<Rec*>(smem);
  __shared__ uint16_t whist[RS_WARPS][RADIX];                // per warp and digit: count, then offset
  __shared__ uint16_t tstart[RADIX];                         // tile-local start of each digit
  __shared__ uint32_t thist[RADIX];                          // the tile's count of each digit
  __shared__ unsigned long long gdst[RADIX];                 // output index of tile position 0 per digit
  __shared__ uint32_t wsum[RS_WARPS];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t s_tile[2];
  const uint32_t tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
  const unsigned long long n = min(*n_ptr, cap);
  const unsigned long long ntiles = (n + RS_TILE - 1) / RS_TILE;
  if (tid == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    claim_tile(in, buf0, n, ntiles, tile_ctr, &s_tile[0], &mbar[0]);
  }
  __syncthreads();
  uint32_t cur = 0, phases = 0;                              // bit b: buffer b's mbarrier parity
  for (;;) {
    const unsigned long long tile = s_tile[cur];
    if (tile >= ntiles) break;
    Rec* const stage = buf0 + cur * RS_TILE;
    if (tid == 0)                                            // the next tile streams in meanwhile
      claim_tile(in, buf0 + (cur ^ 1u) * RS_TILE, n, ntiles, tile_ctr, &s_tile[cur ^ 1u], &mbar[cur ^ 1u]);
    for (uint32_t i = tid; i < RS_WARPS * RADIX; i += RS_T) (&whist[0][0])[i] = 0;
    thist[tid] = 0;                                          // (RS_T == RADIX)
    const unsigned long long t0 = tile * RS_TILE;
    const uint32_t tn = (uint32_t)min((unsigned long long)RS_TILE, n - t0);
    // the CTA's own copies: bounded independently of spin_limit; on a timeout both buffers'
    // copies are drained before the CTA stops taking tiles
    const bool ok = !__syncthreads_or(!mbar_wait(&mbar[cur], (phases >> cur) & 1u, kCopyWaitLimit));
    if (!ok) {
      if (tid == 0) atomicOr(err, 1u);
      __syncthreads_or(!mbar_wait(&mbar[cur], (phases >> cur) & 1u, kCopyWaitLimit));
      if (s_tile[cur ^ 1u] < ntiles)
        __syncthreads_or(!mbar_wait(&mbar[cur ^ 1u], (phases >> (cur ^ 1u)) & 1u, kCopyWaitLimit));
      break;
    }
    phases ^= 1u << cur;

    // the tile's digit counts, published before the tile is ranked, so that tiles reaching
    // their look-back meanwhile find them (a warp whose 32 records share a digit adds once);
    // the look-back itself comes after the ranking, which gives the predecessors time to
    // publish their inclusive prefixes
#pragma unroll
    for (uint32_t s2 = 0; s2 < RS_ITEMS; ++s2) {
      const uint32_t i = w * (RS_ITEMS * 32) + s2 * 32 + lane;
      const bool valid = i < tn;
      const uint32_t dd = valid ? Digit()(stage[i], pass) : 0u;
      const uint32_t lo = __reduce_min_sync(FULL, valid ? dd : RADIX);
      const uint32_t hi = __reduce_max_sync(FULL, valid ? dd : 0u);
      const uint32_t vm = __ballot_sync(FULL, valid);
      if (lo == hi) {
        if (lane == 0 && vm) atomicAdd(&thist[lo], (uint32_t)__popc(vm));
      } else if (valid) {
        atomicAdd(&thist[dd], 1u);
      }
    }
    __syncthreads();
    st_relaxed_u64(status + tile * RADIX + tid, (tile == 0 ? ST_INC : ST_AGG) | thist[tid]);   // digit tid

    // rank: warp w takes records [256 w, 256 w + 256) in 8 steps of 32 consecutive records;
    // a group of lanes with one digit adds itself to the warp's count in one step, in lane
    // order, so ranks follow the input order (stability)
    Rec rec[RS_ITEMS];
    uint32_t pk[RS_ITEMS];                                   // rank in the warp's digit group << 8 | digit
#pragma unroll
    for (uint32_t s2 = 0; s2 < RS_ITEMS; ++s2) {
      const uint32_t i = w * (RS_ITEMS * 32) + s2 * 32 + lane;
      const bool valid = i < tn;
      if (valid) rec[s2] = stage[i];
      const uint32_t d = valid ? Digit()(rec[s2], pass) : 0u;
      // one digit across the valid lanes (upper digits of nearly sorted input): no match needed
      const uint32_t lo = __reduce_min_sync(FULL, valid ? d : RADIX);
      const uint32_t hi = __reduce_max_sync(FULL, valid ? d : 0u);
      const uint32_t vm = __ballot_sync(FULL, valid);
      const uint32_t peers = lo == hi ? (valid ? vm : 1u << lane)
                                      : __match_any_sync(FULL, valid ? d : 0x100u | lane);
      const uint32_t leader = __ffs(peers) - 1;
      uint32_t base = 0;
      if (valid && lane == leader) {
        base = whist[w][d];
        whist[w][d] = (uint16_t)(base + __popc(peers));
      }
      base = __shfl_sync(FULL, base, leader);
      pk[s2] = (base + __popc(peers & lanemask_lt())) << 8 | d;
      __syncwarp();
    }
    __syncthreads();
    // digit d = tid: per-warp offsets and the tile's count
    const uint32_t d = tid;
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t ww = 0; ww < RS_WARPS; ++ww) {
      const uint32_t c = whist[ww][d];
      whist[ww][d] = (uint16_t)cnt;
      cnt += c;
    }
    // tile-local start of each digit: exclusive scan of the counts over the digits
    uint32_t x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    // decoupled look-back for digit d: add the predecessors' counts until one whose inclusive
    // prefix is known, publish the inclusive prefix
    unsigned long long* st = status + tile * RADIX + d;
    unsigned long long excl = 0;
    if (tile != 0) {                 // (the tile's count went out before the ranking)
      // the predecessors' words for digit d, LB tiles at a time (independent loads in flight
      // together), then summed in order until one whose inclusive prefix is known; a word not
      // yet published is polled (bounded)
      constexpr uint32_t LB = 4;
      bool waited_out = false, found = false;
      for (unsigned long long top = tile; top > 0 && !found && !waited_out;) {
        const uint32_t k = (uint32_t)min((unsigned long long)LB, top);
        unsigned long long v[LB];
#pragma unroll
        for (uint32_t q = 0; q < LB; ++q)
          if (q < k) v[q] = ld_relaxed_u64(status + (top - 1 - q) * RADIX + d);
#pragma unroll
        for (uint32_t q = 0; q < LB; ++q) {
          if (q >= k || found || waited_out) break;
          const unsigned long long* sp = status + (top - 1 - q) * RADIX + d;
          unsigned long long y = v[q];
          for (uint32_t it = 0; !(y & (ST_AGG | ST_INC)); ++it) {
            if (it >= spin_limit) {
              waited_out = true;
              break;
            }
            __nanosleep(64);
            y = ld_relaxed_u64(sp);
          }
          if (waited_out) break;
          excl += y & ST_VAL;
          found = (y & ST_INC) != 0;
        }
        top -= k;
      }
      if (waited_out) atomicOr(err, 1u);
      st_relaxed_u64(st, ST_INC | (excl + cnt));
    }
    __syncthreads();
    uint32_t before = 0;
    for (uint32_t ww = 0; ww < w; ++ww) before += wsum[ww];
    tstart[d] = (uint16_t)(before + x - cnt);
    gdst[d] = bins[d] + excl - (before + x - cnt);     // output index = gdst[d] + tile position
    __syncthreads();
    // the tile in digit order, in its own buffer (every record was read above), then out:
    // consecutive positions of one digit go to consecutive output records
#pragma unroll
    for (uint32_t s2 = 0; s2 < RS_ITEMS; ++s2) {
      const uint32_t i = w * (RS_ITEMS * 32) + s2 * 32 + lane;
      const uint32_t dd = pk[s2] & 0xFFu;
      if (i < tn) stage[tstart[dd] + whist[w][dd] + (pk[s2] >> 8)] = rec[s2];
    }
    __syncthreads();
    for (uint32_t i = tid; i < tn; i += RS_T) {
      const Rec r = stage[i];
      const unsigned long long o = gdst[Digit()(r, pass)] + i;
      if (o < n) out[o] = r;        // (only a look-back that gave up can miss: the error flag is set)
    }
    __syncthreads();                 // the buffer is free for the copy issued next iteration
    cur ^= 1u;
  }
}

// ---------------------------------------------------------------- 3. run scan
struct GrunArgs {
  const uint4* rec;                 // sorted global-log records
  const unsigned long long* n_ptr;  // their number
  const LaunchDev* launches;
  uint32_t li0, li1;                // the wave's launches
  const uint32_t* ord_bits;         // launch-order matrices (LaunchDev::ord_off)
  uint4* gout;                      // report entries, two uint4 each:
                                    //   {block, epoch << 2 | kind - 9, word, b}, {c, 0, 0, 0}
  unsigned long long gcap;          // entries that fit
  unsigned long long* gn;           // entries produced (may exceed gcap: the run is repeated)
  uint32_t* gcount;                 // per global block: its entries
};

__device__ __forceinline__ uint32_t find_launch(const GrunArgs& A, uint32_t gb) {
  uint32_t lo = A.li0, hi = A.li1 - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (A.launches[mid].block_base <= gb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// the two smallest distinct values (16-bit; low half the smallest, NONE16 = absent)
__device__ __forceinline__ uint32_t min2_16(uint32_t m, uint32_t t) {
  const uint32_t m1 = m & 0xFFFFu, m2 = m >> 16;
  if (t == m1 || t == m2) return m;
  if (t < m1) return m1 << 16 | t;
  if (t < m2) return t << 16 | m1;
  return m;
}
// the same for 32-bit values (block indices), kInf = absent
__device__ __forceinline__ void min2_32(uint32_t& m1, uint32_t& m2, uint32_t t) {
  if (t == m1 || t == m2) return;
  if (t < m1) {
    m2 = m1;
    m1 = t;
  } else if (t < m2) {
    m2 = t;
  }
}

// classes and smallest conflicting pair from the two smallest writers W and readers R
// (absent = `none`): write-write between distinct writers, write-read between a writer and a
// distinct reader
__device__ __forceinline__ uint32_t pair_classes(const uint32_t (&W)[2], const uint32_t (&R)[2], uint32_t none,
                                                 uint32_t& p1, uint32_t& p2) {
  uint32_t cls = 0;
  p1 = p2 = kInf;
  auto cand = [&](uint32_t x, uint32_t y, uint32_t bit) {
    if (x == none || y == none || x == y) return;
    cls |= bit;
    const uint32_t lo = min(x, y), hi = max(x, y);
    if (lo < p1 || (lo == p1 && hi < p2)) {
      p1 = lo;
      p2 = hi;
    }
  };
  cand(W[0], W[1], SR_CLS_WW);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) cand(W[i], R[j], SR_CLS_WR);
  return cls;
}

__device__ __forceinline__ void emit_entry(const GrunArgs& A, uint32_t gbp, uint32_t ek, uint32_t word, uint32_t b,
                                           uint32_t c) {
  const unsigned long long e = atomicAdd(A.gn, 1ull);
  if (e < A.gcap) {
    A.gout[2 * e] = make_uint4(gbp, ek, word, b);
    A.gout[2 * e + 1] = make_uint4(c, 0u, 0u, 0u);
  }
  atomicAdd(&A.gcount[gbp], 1u);
}

// 1 when launch m (program-local) precedes launch l in the program's order matrix
__device__ __forceinline__ bool ordered(const GrunArgs& A, const LaunchDev& P0, uint32_t m, uint32_t l) {
  const unsigned long long bit = (unsigned long long)l * P0.nl_prog + m;
  return (A.ord_bits[P0.ord_off + (bit >> 5)] >> (bit & 31u)) & 1u;
}

// One thread per run of equal (program, word); records of a run are in (launch, block, epoch)
// order.  A thread looks at record i, and takes the run that starts there.
__global__ void __launch_bounds__(256) k_grun(GrunArgs A) {
  const unsigned long long n = *A.n_ptr;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 r0 = A.rec[i];
    uint32_t li = find_launch(A, r0.w);
    const uint32_t prog = A.launches[li].prog;
    if (i > 0) {
      const uint4 q = A.rec[i - 1];
      if (q.x == r0.x && A.launches[find_launch(A, q.w)].prog == prog) continue;   // not a run start
    }
    // a run of one record holds no pair: nothing to decide
    if (i + 1 >= n) continue;
    {
      const uint4 q = A.rec[i + 1];
      if (q.x != r0.x || A.launches[find_launch(A, q.w)].prog != prog) continue;
    }
    const uint32_t word = r0.x;
    const LaunchDev& P0 = A.launches[A.launches[li].first_launch];    // the program's launch 0
    const bool pairs = P0.ord_off != kNoDep;                          // unordered launches exist
    // interval summary: the two smallest distinct reader and writer tids, pc range
    uint32_t igb = kInf, iep = 0, iR = NONE16 << 16 | NONE16, iW = NONE16 << 16 | NONE16, ipl = kInf, iph = 0;
    // launch summary: the two smallest distinct reader and writer blocks, pc range
    uint32_t lcur = kInf, lR[2] = {kInf, kInf}, lW[2] = {kInf, kInf}, lpl = kInf, lph = 0;
    // launch pairs: kinds of the current launch, start of its sub-run, best pair and classes
    uint32_t lk = 0, b1 = kInf, b2 = kInf, pcls = 0;
    unsigned long long lstart = i;
    for (unsigned long long j = i;; ++j) {
      bool end = j >= n;
      uint4 q = make_uint4(0, 0, 0, 0);
      uint32_t qli = li;
      if (!end) {
        q = A.rec[j];
        const LaunchDev& Lc = A.launches[li];
        qli = (q.w >= Lc.block_base && q.w - Lc.block_base < Lc.grid) ? li : find_launch(A, q.w);
        end = q.x != word || A.launches[qli].prog != prog;
      }
      // interval boundary: (block, epoch) changes
      if (igb != kInf && (end || q.w != igb || q.y != iep)) {
        const uint32_t W[2] = {iW & 0xFFFFu, iW >> 16}, R[2] = {iR & 0xFFFFu, iR >> 16};
        uint32_t t1, t2;
        const uint32_t cls = pair_classes(W, R, NONE16, t1, t2);
        if (cls) emit_entry(A, igb, iep << 2, word, t1 << 16 | t2, cls << 24 | (ipl & 0xFFFu) << 12 | (iph & 0xFFFu));
        igb = kInf;
      }
      // launch boundary
      if (lcur != kInf && (end || qli != lcur)) {
        const LaunchDev& L = A.launches[lcur];
        uint32_t p1, p2;
        const uint32_t cls = pair_classes(lW, lR, kInf, p1, p2);
        if (cls)
          emit_entry(A, L.block_base + p1, 1u, word, p2 + L.block_off,
                     cls << 24 | (lpl & 0xFFFu) << 12 | (lph & 0xFFFu));
        if (pairs) {
          // this launch against every earlier launch of the run that nothing orders before it
          const uint32_t l = L.launch;
          unsigned long long k = i;
          while (k < lstart) {
            const uint32_t mli = find_launch(A, A.rec[k].w);
            const LaunchDev& M = A.launches[mli];
            uint32_t mk = 1u << grec_write(A.rec[k]);      // (the first record is M's: progress)
            for (++k; k < lstart && A.rec[k].w >= M.block_base && A.rec[k].w - M.block_base < M.grid; ++k)
              mk |= 1u << grec_write(A.rec[k]);
            const uint32_t m = M.launch;
            if (ordered(A, P0, m, l)) continue;
            uint32_t c = 0;
            if ((mk & 2u) && (lk & 2u)) c |= SR_CLS_WW;
            if (((mk & 2u) && (lk & 1u)) || ((mk & 1u) && (lk & 2u))) c |= SR_CLS_WR;
            if (!c) continue;
            pcls |= c;
            if (m < b1 || (m == b1 && l < b2)) {
              b1 = m;
              b2 = l;
            }
          }
        }
        lcur = kInf;
      }
      if (end) break;
      // accumulate record q
      const uint32_t t = grec_tid(q), wr = grec_write(q), pc = grec_pc(q);
      if (igb == kInf) {
        igb = q.w;
        iep = q.y;
        iR = iW = NONE16 << 16 | NONE16;
        ipl = kInf;
        iph = 0;
      }
      if (wr) iW = min2_16(iW, t); else iR = min2_16(iR, t);
      ipl = min(ipl, pc);
      iph = max(iph, pc);
      if (lcur == kInf) {
        lcur = qli;
        lR[0] = lR[1] = lW[0] = lW[1] = kInf;
        lpl = kInf;
        lph = 0;
        lk = 0;
        lstart = j;
      }
      const uint32_t blk = q.w - A.launches[qli].block_base;
      if (wr) min2_32(lW[0], lW[1], blk); else min2_32(lR[0], lR[1], blk);
      lpl = min(lpl, pc);
      lph = max(lph, pc);
      lk |= 1u << wr;
      li = qli;
    }
    if (pcls) emit_entry(A, A.launches[P0.first_launch + b1].block_base, 2u, word, b2, pcls << 24);
  }
}

uint32_t g_pass_ctas16 = 0, g_pass_ctas32 = 0;

}  // namespace

// ---------------------------------------------------------------- host side
cudaError_t init_gcheck_attributes(uint32_t smem_optin) {
  (void)smem_optin;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rs_pass<Rec16, AddrDigit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * RS_TILE * sizeof(Rec16)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_rs_pass<Rec32, EntryDigit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * RS_TILE * sizeof(Rec32)));
  int b16 = 0, b32 = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b16, k_rs_pass<Rec16, AddrDigit>, RS_T,
                                                      2 * RS_TILE * sizeof(Rec16));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_rs_pass<Rec32, EntryDigit>, RS_T,
                                                      2 * RS_TILE * sizeof(Rec32));
  g_pass_ctas16 = (uint32_t)std::max(1, b16) * (uint32_t)sms;
  g_pass_ctas32 = (uint32_t)std::max(1, b32) * (uint32_t)sms;
  return e;
}

uint64_t gcheck_tiles(uint64_t records) { return (records + RS_TILE - 1) / RS_TILE; }
uint64_t gcheck_partials(uint32_t nblocks) { return (nblocks + SC_CHUNK - 1) / SC_CHUNK + 1; }

// exclusive scan of per-block counts c[gb0 .. gb1) into off[0 .. gb1 - gb0) and *total
static cudaError_t count_scan(const uint32_t* c, uint32_t gb0, uint32_t gb1, unsigned long long* partials,
                              unsigned long long* off, unsigned long long* total, uint32_t& kernels,
                              cudaStream_t s) {
  const uint32_t nchunks = (gb1 - gb0 + SC_CHUNK - 1) / SC_CHUNK;
  if (nchunks) k_count_chunks<<<nchunks, SC_T, 0, s>>>(c, gb0, gb1, partials);
  k_count_scan<<<1, SC_T, 0, s>>>(partials, nchunks, total);
  if (nchunks) k_count_offsets<<<nchunks, SC_T, 0, s>>>(c, gb0, gb1, partials, off);
  kernels += nchunks ? 3 : 1;
  return cudaGetLastError();
}

// sort n (device count, at most cap) records of `in` by `npasses` digits; returns the buffer
// holding the result (in or tmp)
template <class Rec, class Digit>
static cudaError_t radix_sort(Rec* in, Rec* tmp, const unsigned long long* n_ptr, unsigned long long cap,
                              uint32_t npasses, const GcheckArgs& G, uint32_t ctas, Rec** result,
                              uint32_t& kernels, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(G.hist, 0, MAX_PASSES * RADIX * 8, s);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = gcheck_tiles(cap);
  const uint32_t up = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, (cap + RS_T - 1) / RS_T), 8ull * G.sms);
  k_rs_upsweep<Rec, Digit><<<up, RS_T, 0, s>>>(in, n_ptr, cap, npasses, G.hist);
  k_rs_bins<<<1, RADIX, 0, s>>>(G.hist, npasses);
  kernels += 2;
  Rec* a = in;
  Rec* b = tmp;
  const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(tiles, ctas));
  for (uint32_t p = 0; p < npasses; ++p) {
    e = cudaMemsetAsync(G.status, 0, std::max<uint64_t>(1, tiles) * RADIX * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(G.tile_ctr + p, 0, 4, s);
    if (e != cudaSuccess) return e;
    k_rs_pass<Rec, Digit><<<grid, RS_T, 2 * RS_TILE * sizeof(Rec), s>>>(a, b, n_ptr, cap, p, G.hist + p * RADIX,
                                                                       G.status, G.tile_ctr + p, G.err,
                                                                       G.spin_limit);
    ++kernels;
    Rec* t = a;
    a = b;
    b = t;
  }
  *result = a;
  return cudaGetLastError();
}

cudaError_t launch_gcheck(const GcheckArgs& G, uint32_t& kernels, cudaStream_t s) {
  // 1. gather the wave's records
  cudaError_t e = count_scan(G.glog_n, G.gb0, G.gb1, G.partials, G.goff, G.gtotal, kernels, s);
  if (e != cudaSuccess) return e;
  {
    const uint32_t want = (G.gb1 - G.gb0 + 7) / 8;
    const uint32_t ctas = std::max(1u, std::min(want, 8u * G.sms));
    k_ggather<<<ctas, 256, 0, s>>>(G.launches, G.li0, G.li1, G.gb0, G.gb1, G.glog, G.glog_n, G.goff, G.sort_a,
                                   G.rec_cap, G.err);
    ++kernels;
  }
  // 2. sort by word address
  Rec16* sorted = nullptr;
  e = radix_sort<Rec16, AddrDigit>(reinterpret_cast<Rec16*>(G.sort_a), reinterpret_cast<Rec16*>(G.sort_b),
                                   G.gtotal, G.rec_cap, G.addr_passes, G, g_pass_ctas16, &sorted, kernels, s);
  if (e != cudaSuccess) return e;
  // 3. the run scan
  e = cudaMemsetAsync(G.gn, 0, 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.gcount + G.gb0, 0, (size_t)(G.gb1 - G.gb0) * 4, s);
  if (e != cudaSuccess) return e;
  GrunArgs R{};
  R.rec = reinterpret_cast<const uint4*>(sorted);
  R.n_ptr = G.gtotal;
  R.launches = G.launches;
  R.li0 = G.li0;
  R.li1 = G.li1;
  R.ord_bits = G.ord_bits;
  R.gout = G.entries_a;
  R.gcap = G.entry_cap;
  R.gn = G.gn;
  R.gcount = G.gcount;
  {
    const uint32_t ctas = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((G.rec_cap + 255) / 256, 16ull * G.sms));
    k_grun<<<ctas, 256, 0, s>>>(R);
    ++kernels;
  }
  // 4. the entries in (block, epoch, kind, word) order, and each block's first entry
  Rec32* ordered_entries = nullptr;
  e = radix_sort<Rec32, EntryDigit>(reinterpret_cast<Rec32*>(G.entries_a), reinterpret_cast<Rec32*>(G.entries_b),
                                    G.gn, G.entry_cap, MAX_PASSES, G, g_pass_ctas32, &ordered_entries, kernels, s);
  if (e != cudaSuccess) return e;
  // (12 passes: the result is back in entries_a)
  return count_scan(G.gcount, G.gb0, G.gb1, G.partials, G.gstart, G.gn_sorted, kernels, s);
}

}  // namespace sr
