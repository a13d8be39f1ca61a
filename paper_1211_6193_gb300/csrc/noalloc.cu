// noalloc.cu - sr_check_program_noalloc: the whole check of one program without any
// device (or host heap) allocation.
//
// Some callers cannot allocate: code inside a framework that owns every byte of device
// memory through its own allocator, or in a process that forbids cudaMalloc after
// start-up.  This entry point runs the same kernels as
// load_programs + run_and_check, but every intermediate buffer (packed code, launch
// table, access logs, per-block results, scan and checker scratch) lives in one
// file-scope __device__ array of SR_NOALLOC_SCRATCH_BYTES.  The caller passes the inputs
// (program descriptors in host memory, the global arena on the device) and the outputs
// (the arena, updated in place, and a device report buffer).
#include <algorithm>
#include <mutex>

#include "host_prep.h"
#include "sr_internal.h"

namespace {

// The scratch: every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr uint32_t kMaxLaunches = 256;
constexpr uint32_t kMaxWaves = 256;
constexpr uint32_t kCheckCtas = 8;          // checker CTAs (each owns 256 KB of race-entry staging)

// Device address of the array and the result of the one-time set-up, per device.  The
// set-up runs once per device under std::call_once, also when several host threads make
// their first call at the same time.
void* g_scratch_addr[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];
std::once_flag g_setup_once[kMaxDevices];

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocWave {
  uint32_t li0, li1, gb0, gb1;
};

// Host staging of one call (~150 KB): thread-local, so that a call needs neither heap
// memory nor a large stack (callers on threads with small stacks).
struct HostStaging {
  uint2 code[SR_MAX_CODE + 2];
  uint8_t colour[SR_MAX_CODE + 1];
  uint32_t acc[SR_MAX_CODE + 1], bar[SR_MAX_CODE + 1], spc[SR_MAX_CODE + 1], snx[SR_MAX_CODE + 1];
  uint32_t gacc[SR_MAX_CODE + 1];
  sr::LaunchDev L[kMaxLaunches];
  NoallocWave waves[kMaxWaves];
};
thread_local HostStaging t_staging;

}  // namespace

using namespace sr::host;

extern "C" int sr_check_program_noalloc(const sr_program* prog, int32_t* d_arena, sr_report* d_reports,
                                        uint64_t report_cap, uint64_t* n_reports, uint32_t* status,
                                        void* stream) {
  if (!prog || (prog->global_words && !d_arena) || (report_cap && !d_reports) || !n_reports || !status)
    return SR_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  char msg[256];
  // validation reads only the code and launches; the arena is the caller's device buffer
  sr_program pv = *prog;
  static const int32_t one_word = 0;
  pv.global_init = &one_word;
  if (validate(&pv, msg, sizeof msg) != SR_OK) return SR_E_INVAL;
  if (prog->nlaunches > kMaxLaunches) return SR_E_RANGE;
  // on a stream that is being captured the copies and the synchronisation below would fail
  // and invalidate the caller's capture: refuse before touching the stream
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return SR_E_INVAL;
  }
  if (cap != cudaStreamCaptureStatusNone) return SR_E_INVAL;

  // ---- once per device: the array's device address and the kernels' attributes
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDevices) return SR_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return SR_E_CUDA;
  std::call_once(g_setup_once[dev], [dev, optin]() {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = sr::init_kernel_attributes((uint32_t)optin);
    if (e != cudaSuccess) cudaGetLastError();
    g_setup_err[dev] = e;
    g_scratch_addr[dev] = e == cudaSuccess ? ptr : nullptr;
  });
  if (g_setup_err[dev] != cudaSuccess || !g_scratch_addr[dev]) return SR_E_CUDA;
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);

  // ---- pack code and launch table (thread-local host staging)
  HostStaging& T = t_staging;
  const uint32_t ncode = prog->ncode;
  uint2* code = T.code;
  const RegMap rm = map_registers(*prog);
  for (uint32_t pc = 0; pc < ncode; ++pc) code[pc] = pack(prog->code[pc], rm);
  code[ncode] = exit_sentinel(rm);
  set_run_lengths(code, ncode + 1);
  uint32_t npacked = ncode + 1;
  if (npacked & 1) code[npacked++] = exit_sentinel(rm);

  const BoundScratch ws{T.colour, T.acc, T.bar, T.spc, T.snx, T.gacc};
  sr::LaunchDev* L = T.L;
  uint64_t nblocks = 0, check_items = 0;
  for (uint32_t l = 0; l < prog->nlaunches; ++l) {
    const sr_launch& pl = prog->launches[l];
    const KernelBound k = bound_kernel(prog->code, ncode, prog->kernel_entry[pl.kernel], ws);
    sr::LaunchDev d{};
    d.prog = 0;
    d.launch = l;
    d.index = l;
    launch_deps(prog->launches, l, sr::kNoDep, d.dep_prev, d.dep_wait);
    d.entry = prog->kernel_entry[pl.kernel];
    d.ncode = ncode;
    d.code_off = 0;
    d.grid = pl.block_count ? pl.block_count : pl.grid;
    d.gdim = pl.grid;
    d.block_off = pl.block_begin;
    d.bdim = pl.block_dim;
    d.shw = pl.shmem_words;
    d.nparams = pl.nparams;
    for (uint32_t q = 0; q < 4; ++q) d.params[q] = q < pl.nparams ? pl.params[q] : 0;
    d.block_base = (uint32_t)nblocks;
    d.key_bits = key_bits_for(std::max(1u, pl.shmem_words));
    const uint64_t cap = launch_log_cap(k, pl.block_dim, 1, 65536);
    if (cap >= (1ull << 31)) return SR_E_RANGE;
    d.log_cap = (uint32_t)cap;
    d.arena_off = 0;
    d.arena_words = prog->global_words;
    d.ir_bytes = sr::ir_smem_bytes(ncode);
    d.nrows = rm.nrows;
    const uint32_t nw = (pl.block_dim + 31) / 32;
    d.group_bytes = sr::group_layout(nw * 32, pl.shmem_words, ncode, rm.nrows, 0, 0).total;
    d.groups = 1;
    d.item_blocks = 1;
    d.check_group = sr::check_group_for(d.log_cap);
    d.check_item = (uint32_t)check_items;
    check_items += (d.grid + d.check_group - 1) / d.check_group;
    if (d.ir_bytes + d.group_bytes + 1024 > (uint32_t)optin) return SR_E_RANGE;
    nblocks += d.grid;
    L[l] = d;
  }
  const uint32_t nl = prog->nlaunches;

  // ---- scratch layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += up256(bytes ? bytes : 1);
    return o;
  };
  const size_t o_code = take((size_t)npacked * 8);
  const size_t o_launch = take((size_t)std::max(1u, nl) * sizeof(sr::LaunchDev));
  const size_t o_blocks = take((size_t)nblocks * sizeof(sr::BlockRes));
  const size_t o_status = take(4 + 4 * (size_t)std::max(1u, nl));   // status, per-launch stop marks
  const size_t o_counters = take(sizeof(sr::Counters));
  const size_t o_total = take(8);
  const size_t o_heads = take(kMaxWaves * 4 + 4);      // checker work heads + error flag
  const size_t o_offsets = take(((size_t)nblocks + 1) * 8);
  const size_t o_partials = take(sr::compact_partials_count((uint32_t)nblocks) * 8);
  const uint32_t cctas = std::min<uint32_t>(kCheckCtas, (uint32_t)sms);
  const size_t o_table = take((size_t)cctas * sr::kScratchWords * 16);
  if (off >= SR_NOALLOC_SCRATCH_BYTES) return SR_E_RANGE;
  const size_t o_log = off;
  const uint64_t log_records = (SR_NOALLOC_SCRATCH_BYTES - off) / 8;

  // waves: consecutive launches whose logs fit the remaining scratch together
  NoallocWave* waves = T.waves;
  uint32_t nwaves = 0;
  uint64_t used = 0;
  for (uint32_t l = 0; l < nl; ++l) {
    const uint64_t need = (uint64_t)L[l].grid * L[l].log_cap;
    if (need > log_records) return SR_E_RANGE;        // one launch alone does not fit
    if (nwaves == 0 || used + need > log_records) {
      if (nwaves == kMaxWaves) return SR_E_RANGE;
      waves[nwaves++] = NoallocWave{l, l, L[l].block_base, L[l].block_base};
      used = 0;
    }
    L[l].log_base = used;
    used += need;
    waves[nwaves - 1].li1 = l + 1;
    waves[nwaves - 1].gb1 = L[l].block_base + L[l].grid;
  }

  // ---- upload and reset (pageable sources are staged before the calls return)
#define NA_TRY(call)                                  \
  do {                                                \
    if ((call) != cudaSuccess) {                      \
      cudaGetLastError();                             \
      return SR_E_CUDA;                               \
    }                                                 \
  } while (0)
  NA_TRY(cudaMemcpyAsync(base + o_code, code, (size_t)npacked * 8, cudaMemcpyHostToDevice, s));
  if (nl) NA_TRY(cudaMemcpyAsync(base + o_launch, L, (size_t)nl * sizeof(sr::LaunchDev), cudaMemcpyHostToDevice, s));
  NA_TRY(cudaMemsetAsync(base + o_blocks, 0, (size_t)nblocks * sizeof(sr::BlockRes), s));
  NA_TRY(cudaMemsetAsync(base + o_status, 0, 4, s));
  NA_TRY(cudaMemsetAsync(base + o_status + 4, 0, 4 * (size_t)std::max(1u, nl), s));
  NA_TRY(cudaMemsetAsync(base + o_counters, 0, sizeof(sr::Counters), s));
  NA_TRY(cudaMemsetAsync(base + o_total, 0, 8, s));
  NA_TRY(cudaMemsetAsync(base + o_heads, 0, kMaxWaves * 4 + 4, s));

  sr::RunArgs ra{};
  ra.launches = reinterpret_cast<const sr::LaunchDev*>(base + o_launch);
  ra.nlaunches = nl;
  ra.budget = 1u << 24;
  ra.check_races = 1;
  ra.spin_limit = 1u << 26;
  ra.code = reinterpret_cast<const uint2*>(base + o_code);
  ra.arena = d_arena;
  ra.log = reinterpret_cast<unsigned long long*>(base + o_log);
  ra.blocks = reinterpret_cast<sr::BlockRes*>(base + o_blocks);
  ra.prog_status = reinterpret_cast<uint32_t*>(base + o_status);
  ra.launch_dead = reinterpret_cast<uint32_t*>(base + o_status + 4);
  ra.counters = reinterpret_cast<sr::Counters*>(base + o_counters);
  uint32_t* heads = reinterpret_cast<uint32_t*>(base + o_heads);
  for (uint32_t wi = 0; wi < nwaves; ++wi) {
    const NoallocWave& w = waves[wi];
    for (uint32_t li = w.li0; li < w.li1; ++li) NA_TRY(sr::launch_interp_plain(ra, li, L[li], 0, s));
    sr::CheckArgs ca{};
    ca.launches = ra.launches;
    ca.li0 = w.li0;
    ca.li1 = w.li1;
    ca.item0 = L[w.li0].check_item;
    ca.item1 = w.li1 < nl ? L[w.li1].check_item : (uint32_t)check_items;
    ca.log = ra.log;
    ca.blocks = ra.blocks;
    ca.scratch = reinterpret_cast<uint4*>(base + o_table);
    ca.work_head = heads + wi;
    ca.error_flag = heads + kMaxWaves;
    ca.spin_limit = ra.spin_limit;
    ca.table_words = sr::check_table_words(L, w.li0, w.li1, sr::check_table_cap(0));
    const uint32_t ctas = std::min<uint32_t>(cctas, ca.item1 - ca.item0);
    if (ctas) NA_TRY(sr::launch_check(ca, 0, ctas, s));
    sr::CompactArgs ka{};
    ka.launches = ra.launches;
    ka.nlaunches = nl;
    ka.gb0 = w.gb0;
    ka.gb1 = w.gb1;
    ka.total = reinterpret_cast<unsigned long long*>(base + o_total);
    ka.log = ra.log;
    ka.blocks = ra.blocks;
    ka.offsets = reinterpret_cast<unsigned long long*>(base + o_offsets);
    ka.partials = reinterpret_cast<unsigned long long*>(base + o_partials);
    ka.out = d_reports;
    ka.out_cap = report_cap;
    ka.counters = ra.counters;
    ka.error_flag = heads + kMaxWaves;
    NA_TRY(sr::launch_compact_scan(ka, s));
    NA_TRY(sr::launch_compact_emit(ka, s));
  }
  unsigned long long total = 0;
  uint32_t st = 0, err = 0;
  NA_TRY(cudaMemcpyAsync(&total, base + o_total, 8, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaMemcpyAsync(&st, base + o_status, 4, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaMemcpyAsync(&err, heads + kMaxWaves, 4, cudaMemcpyDeviceToHost, s));
  NA_TRY(cudaStreamSynchronize(s));
#undef NA_TRY
  *n_reports = total;
  *status = st;
  if (err & sr::kErrBounds) return SR_E_BOUNDS;
  if (err) return SR_E_TIMEOUT;
  return total > report_cap ? SR_E_RANGE : SR_OK;
}
