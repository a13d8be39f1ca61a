// compact.cu - canonical report order (the diagnostics of Sec. 3.2's cudak runs).
//
// Work is done per wave, a range [gb0, gb1) of global block indices whose access logs
// are resident together; the reports of a wave follow those of earlier waves.
// Reports are ordered by (prog, launch, block, epoch, kind, a, b, c).  Global block
// indices already follow (prog, launch, block), so an exclusive scan of the per-block
// report counts gives every block its output range.  Inside a block, race entries
// (kind 1, address order per interval) and barrier/error entries (kinds 2..7, kind and
// pc order per interval) are both sorted by interval; a merge by interval places them:
// races of an interval come before its other records.  With the global-memory race check a
// third list per block (kinds 9..11, ordered by (epoch, kind, word) in gcheck.cu) is merged
// the same way: its records of an interval follow the interval's races and other records.
#include "sr_internal.h"

namespace sr {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t SCAN_T = 1024;
constexpr uint32_t SCAN_PER = 4;
constexpr uint32_t CHUNK = SCAN_T * SCAN_PER;

__device__ __forceinline__ uint32_t block_count(const CompactArgs& A, uint32_t gb) {
  const BlockRes& r = A.blocks[gb];
  return r.n_race + r.n_misc + (A.gcount ? A.gcount[gb] : 0u);
}

// inclusive scan of one value per thread across a CTA of SCAN_T threads
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

__global__ void __launch_bounds__(SCAN_T) k_chunk_sums(CompactArgs A) {
  __shared__ unsigned long long wsum[32];
  const uint32_t base = A.gb0 + blockIdx.x * CHUNK + threadIdx.x * SCAN_PER;
  unsigned long long s = 0;
  for (uint32_t i = 0; i < SCAN_PER; ++i)
    if (base + i < A.gb1) s += block_count(A, base + i);
  const unsigned long long inc = cta_inclusive(s, wsum);
  if (threadIdx.x == SCAN_T - 1) A.partials[blockIdx.x] = inc;
}

// single CTA: chunk sums -> exclusive chunk offsets (plus the running total of earlier
// waves); advances the running total by this wave's reports
__global__ void __launch_bounds__(SCAN_T) k_scan_chunks(CompactArgs A, uint32_t nchunks) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long s_tot;
  unsigned long long carry = *A.total;
  for (uint32_t b = 0; b < nchunks; b += SCAN_T) {
    const uint32_t i = b + threadIdx.x;
    const unsigned long long v = i < nchunks ? A.partials[i] : 0ull;
    const unsigned long long inc = cta_inclusive(v, wsum);
    if (i < nchunks) A.partials[i] = carry + inc - v;
    if (threadIdx.x == SCAN_T - 1) s_tot = inc;
    __syncthreads();
    carry += s_tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *A.total = carry;
    A.counters->total_reports = carry;
  }
}

__global__ void __launch_bounds__(SCAN_T) k_block_offsets(CompactArgs A) {
  __shared__ unsigned long long wsum[32];
  const uint32_t base = A.gb0 + blockIdx.x * CHUNK + threadIdx.x * SCAN_PER;
  uint32_t c[SCAN_PER];
  unsigned long long s = 0;
  for (uint32_t i = 0; i < SCAN_PER; ++i) {
    c[i] = base + i < A.gb1 ? block_count(A, base + i) : 0u;
    s += c[i];
  }
  unsigned long long run = cta_inclusive(s, wsum) - s + A.partials[blockIdx.x];
  for (uint32_t i = 0; i < SCAN_PER; ++i) {
    if (base + i < A.gb1) A.offsets[base + i] = run;
    run += c[i];
  }
}

// entries [0, n) of the block's global list whose epoch is below `ep` (the list is in epoch order)
__device__ __forceinline__ uint32_t global_before(const uint4* ge, uint32_t n, uint32_t ep) {
  uint32_t a = 0, b = n;
  while (a < b) {
    const uint32_t m = (a + b) >> 1;
    if ((ge[2 * m].y >> 2) < ep) a = m + 1; else b = m;
  }
  return a;
}

// one warp per simulated block
__global__ void __launch_bounds__(256) k_emit(CompactArgs A) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t gb = A.gb0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gb < A.gb1; gb += nwarps) {
    const BlockRes r = A.blocks[gb];
    const uint32_t nr = r.n_race, nm = r.n_misc;
    uint32_t ng = A.gcount ? A.gcount[gb] : 0u;
    if (nr + nm + ng == 0) continue;
    // entries past the buffer (the wave produced more than it holds and is run again before
    // any report is read) are left out
    if (ng && A.gstart[gb - A.gb0] + ng > A.gcap) ng = 0;
    uint32_t lo = 0, hi = A.nlaunches - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (A.launches[mid].block_base <= gb) lo = mid; else hi = mid - 1;
    }
    const LaunchDev* L = A.launches + lo;
    const uint32_t lb = gb - L->block_base;            // the block's place in this batch's share
    const uint32_t block = lb + L->block_off;          // its index in the grid (reports)
    const uint4* reg4 = reinterpret_cast<const uint4*>(A.log + L->log_base + (unsigned long long)lb * L->log_cap);
    const uint32_t top = L->log_cap / 2 - 1;        // misc entry j lives at reg4[top - j]
    const uint4* ge = ng ? A.gentries + 2 * A.gstart[gb - A.gb0] : nullptr;   // the block's global list
    // (debug build: both lists lie inside the block's region)
    if (!dbg_ok(2ull * (nr + nm) <= L->log_cap, A.error_flag, kErrBounds)) continue;
    const unsigned long long base = A.offsets[gb];
    // misc entries (epoch order) with epoch below / at most `ep`
    auto misc_below = [&](uint32_t ep, bool at_most) {
      uint32_t a = 0, b = nm;
      while (a < b) {
        const uint32_t m = (a + b) >> 1;
        const uint32_t e = reg4[top - m].x & 0x0FFFFFFFu;
        if (e < ep || (at_most && e == ep)) a = m + 1; else b = m;
      }
      return a;
    };
    // race entries (epoch order) with epoch at most `ep`
    auto races_upto = [&](uint32_t ep) {
      uint32_t a = 0, b = nr;
      while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (reg4[m].x <= ep) a = m + 1; else b = m;
      }
      return a;
    };
    for (uint32_t i = lane; i < nr; i += 32) {
      const uint4 e = reg4[i];
      // misc and global entries of earlier intervals
      const uint32_t before = (nm ? misc_below(e.x, false) : 0u) + (ng ? global_before(ge, ng, e.x) : 0u);
      const unsigned long long o = base + i + before;
      if (o < A.out_cap) A.out[o] = sr_report{SR_REP_RACE, L->prog, L->launch, block, e.x, e.y, e.z, e.w};
    }
    for (uint32_t j = lane; j < nm; j += 32) {
      const uint4 e = reg4[top - j];
      const uint32_t ep = e.x & 0x0FFFFFFFu;
      // races of this or earlier intervals, global entries of earlier intervals
      const unsigned long long o = base + j + races_upto(ep) + (ng ? global_before(ge, ng, ep) : 0u);
      if (o < A.out_cap) A.out[o] = sr_report{e.x >> 28, L->prog, L->launch, block, ep, e.y, e.z, e.w};
    }
    for (uint32_t k = lane; k < ng; k += 32) {
      const uint4 e = ge[2 * k], f = ge[2 * k + 1];
      const uint32_t ep = e.y >> 2;
      // races and other records of this or earlier intervals
      const unsigned long long o = base + k + races_upto(ep) + (nm ? misc_below(ep, true) : 0u);
      if (o < A.out_cap)
        A.out[o] = sr_report{SR_REP_GLOBAL_RACE + (e.y & 3u), L->prog, L->launch, block, ep, e.z, e.w, f.x};
    }
  }
}

}  // namespace

uint64_t compact_partials_count(uint32_t nblocks) { return (nblocks + CHUNK - 1) / CHUNK + 1; }

uint32_t compact_kernels(const CompactArgs& a) {
  const uint32_t nchunks = (a.gb1 - a.gb0 + CHUNK - 1) / CHUNK;
  return (nchunks ? 3u : 1u) + 1u;
}

cudaError_t launch_compact_scan(const CompactArgs& a, cudaStream_t s) {
  const uint32_t nchunks = (a.gb1 - a.gb0 + CHUNK - 1) / CHUNK;
  if (nchunks) {
    k_chunk_sums<<<nchunks, SCAN_T, 0, s>>>(a);
  }
  k_scan_chunks<<<1, SCAN_T, 0, s>>>(a, nchunks);
  if (nchunks) k_block_offsets<<<nchunks, SCAN_T, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_compact_emit(const CompactArgs& a, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint32_t want = (a.gb1 - a.gb0 + 7) / 8;
  const uint32_t ctas = want < (uint32_t)sms * 8 ? (want ? want : 1) : (uint32_t)sms * 8;
  k_emit<<<ctas, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sr
