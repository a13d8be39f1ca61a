// runtime.cpp - host side of libsimtcheck: the C ABI of include/simtcheck.h.
//
// load_programs  validates and packs the programs (code with an EXIT sentinel, register
//                fields remapped so RZ and unused operands read the zero row), bounds
//                every launch's per-block access log statically, groups launches into
//                waves whose logs fit the log budget, and uploads everything.
// run_and_check  per wave: interpreter (one launch per (program, launch) in plain mode;
//                in batched mode one persistent launch, preceded with two CTAs per SM by
//                one grid of the programs that run one block per CTA), race check, report
//                scan and emission.  Everything is enqueued on the caller's stream.
// fetch_*        synchronise the stream and copy results to the host.
#include <algorithm>
#include <cstdarg>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "host_prep.h"
#include "sr_internal.h"

using sr::LaunchDev;
using namespace sr::host;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Wave {
  uint32_t li0, li1;      // launch index range
  uint32_t gb0, gb1;      // global block range
  uint32_t item0, item1;  // batched work items
  uint32_t bq0, bq1;      // batched mode, two CTAs per SM: entries of the block queue
  uint32_t bq_blocks;     // and the blocks (tickets) they hold
  uint64_t log_records;
  uint64_t glog_records;  // global-memory race check: records of the wave's global logs
  uint32_t addr_bits;     // and the bits of its largest global word address
};

}  // namespace

struct sr_ctx {
  sr_opts opts{};
  sr_allocator alloc{};
  bool custom_alloc = false;
  std::string err;
  int device = 0;
  int sms = 0;
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;
  cudaMemPool_t pool = nullptr;   // without a caller allocator: this context's own memory pool
};

struct sr_batch {
  uint32_t nprogs = 0;
  std::vector<LaunchDev> launches;
  std::vector<uint64_t> arena_off, arena_words;
  std::vector<uint2> items;
  std::vector<uint32_t> item_launch;       // race check: launch of every work item
  // batched mode, two CTAs per SM: the launches run one block per CTA (k_interp_blocks), per
  // wave in ticket order, and the first ticket of each
  std::vector<uint8_t> one_per_cta;        // per launch
  std::vector<uint32_t> bq_launch, bq_first;
  uint32_t blocks_smem = 0;
  uint64_t bq_blocks = 0;                  // blocks of all waves run one per CTA
  std::vector<Wave> waves;
  uint32_t nblocks = 0;
  uint32_t check_items = 0;                // race-check work items of all waves
  uint32_t max_key_bits = 1;
  uint32_t batched_smem = 0;
  uint64_t total_code = 0, total_arena = 0, log_records = 0;
  DevBuf code, launches_d, arena_init, arena_work, log, blocks, prog_status, launch_dead, counters, items_d,
      queue_head, launch_done, scratch, work_head, err_flag, offsets, partials, out, total, item_launch_d,
      bq_launch_d, bq_first_d, bq_head;
  uint64_t out_cap = 0;
  // global-memory race check (opts.check_global)
  DevBuf glog, glog_n, goff, gpartials, gtotal, sort_a, sort_b, hist, status, tile_ctr, ord_bits, entries_a, entries_b,
      gn, gcount, gstart, gn_sorted;
  std::vector<uint32_t> ord_bits_h;
  uint64_t glog_records = 0;               // largest wave's global-log records
  uint64_t entry_cap = 0;                  // report entries of one wave that fit
  cudaStream_t stream = nullptr;
  bool ran = false;
  uint32_t check_ctas = 0;
  // CUDA graph of run_and_check (batched mode with use_graph)
  cudaGraphExec_t graph = nullptr;
  cudaStream_t graph_stream = nullptr;
  // profiling
  std::vector<cudaEvent_t> events;
  uint32_t nevents_used = 0;
  uint32_t kernels = 0;                    // kernel launches enqueued by the last run
};

namespace {

thread_local std::string g_create_error;   // failures of sr_create (no context yet)

int fail(sr_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_error = buf;
  return code;
}
#define CUDA_TRY(c, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail((c), SR_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

void* dev_alloc(sr_ctx* c, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (c->custom_alloc) return c->alloc.alloc(c->alloc.user, bytes, s);
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, bytes, c->pool, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void dev_free(sr_ctx* c, DevBuf& b, cudaStream_t s) {
  if (!b.p) return;
  if (c->custom_alloc)
    c->alloc.release(c->alloc.user, b.p, b.bytes, s);
  else
    cudaFreeAsync(b.p, s);
  b.p = nullptr;
  b.bytes = 0;
}
int alloc_buf(sr_ctx* c, DevBuf& b, size_t bytes, cudaStream_t s, const char* what) {
  b.p = dev_alloc(c, bytes, s);
  b.bytes = bytes ? bytes : 16;
  if (!b.p) return fail(c, SR_E_NOMEM, "device allocation of %zu bytes for %s failed", bytes, what);
  return SR_OK;
}

void free_batch_buffers(sr_ctx* c, sr_batch* b, cudaStream_t s) {
  DevBuf* all[] = {&b->code, &b->launches_d, &b->arena_init, &b->arena_work, &b->log, &b->blocks,
                   &b->prog_status, &b->launch_dead, &b->counters, &b->items_d, &b->queue_head,
                   &b->launch_done, &b->scratch, &b->work_head, &b->err_flag, &b->offsets, &b->partials,
                   &b->out, &b->total, &b->item_launch_d, &b->glog, &b->glog_n, &b->goff, &b->gpartials,
                   &b->gtotal, &b->sort_a, &b->sort_b, &b->hist, &b->status, &b->tile_ctr, &b->ord_bits,
                   &b->entries_a, &b->entries_b, &b->gn, &b->gcount, &b->gstart, &b->gn_sorted,
                   &b->bq_launch_d, &b->bq_first_d, &b->bq_head};
  for (DevBuf* d : all) dev_free(c, *d, s);
}

cudaEvent_t next_event(sr_batch* b) {
  if (b->nevents_used == b->events.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    b->events.push_back(e);
  }
  return b->events[b->nevents_used++];
}

// Enqueue the whole pipeline for one run on stream s.
sr::CompactArgs compact_args(sr_batch* b, const Wave& w) {
  sr::CompactArgs ka{};
  ka.launches = (const LaunchDev*)b->launches_d.p;
  ka.nlaunches = (uint32_t)b->launches.size();
  ka.gb0 = w.gb0;
  ka.gb1 = w.gb1;
  ka.total = (unsigned long long*)b->total.p;
  ka.log = (const unsigned long long*)b->log.p;
  ka.blocks = (const sr::BlockRes*)b->blocks.p;
  ka.offsets = (unsigned long long*)b->offsets.p;
  ka.partials = (unsigned long long*)b->partials.p;
  ka.out = (sr_report*)b->out.p;
  ka.out_cap = b->out_cap;
  ka.counters = (sr::Counters*)b->counters.p;
  ka.error_flag = (uint32_t*)b->err_flag.p;
  if (w.glog_records) {
    ka.gcount = (const uint32_t*)b->gcount.p;
    ka.gstart = (const unsigned long long*)b->gstart.p;
    ka.gentries = (const uint4*)b->entries_a.p;
    ka.gcap = b->entry_cap;
  }
  return ka;
}

// The global-memory race check of wave wi (enqueued on s).
sr::GcheckArgs gcheck_args(sr_ctx* c, sr_batch* b, uint32_t wi) {
  const Wave& w = b->waves[wi];
  sr::GcheckArgs g{};
  g.launches = (const LaunchDev*)b->launches_d.p;
  g.li0 = w.li0;
  g.li1 = w.li1;
  g.gb0 = w.gb0;
  g.gb1 = w.gb1;
  g.glog = (const uint4*)b->glog.p;
  g.glog_n = (const uint32_t*)b->glog_n.p;
  g.goff = (unsigned long long*)b->goff.p;
  g.gtotal = (unsigned long long*)b->gtotal.p;
  g.partials = (unsigned long long*)b->gpartials.p;
  g.sort_a = (uint4*)b->sort_a.p;
  g.sort_b = (uint4*)b->sort_b.p;
  g.rec_cap = w.glog_records;
  g.addr_passes = std::max(1u, (w.addr_bits + 7) / 8);
  g.hist = (unsigned long long*)b->hist.p;
  g.status = (unsigned long long*)b->status.p;
  g.tile_ctr = (uint32_t*)b->tile_ctr.p;
  g.err = (uint32_t*)b->err_flag.p;
  g.spin_limit = c->opts.spin_limit;
  g.sms = (uint32_t)c->sms;
  g.ord_bits = (const uint32_t*)b->ord_bits.p;
  g.entries_a = (uint4*)b->entries_a.p;
  g.entries_b = (uint4*)b->entries_b.p;
  g.entry_cap = b->entry_cap;
  g.gn = (unsigned long long*)b->gn.p + wi;
  g.gcount = (uint32_t*)b->gcount.p;
  g.gstart = (unsigned long long*)b->gstart.p;
  g.gn_sorted = (unsigned long long*)b->gn_sorted.p;
  return g;
}

int enqueue_run(sr_ctx* c, sr_batch* b, cudaStream_t s, bool profile) {
  const sr_opts& o = c->opts;
  b->nevents_used = 0;
  b->kernels = 0;
  auto mark = [&]() -> cudaEvent_t {
    if (!profile) return nullptr;
    cudaEvent_t e = next_event(b);
    if (e) cudaEventRecord(e, s);
    return e;
  };
  mark();
  CUDA_TRY(c, cudaMemcpyAsync(b->arena_work.p, b->arena_init.p, b->total_arena * 4, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(c, cudaMemsetAsync(b->blocks.p, 0, (size_t)b->nblocks * sizeof(sr::BlockRes), s));
  CUDA_TRY(c, cudaMemsetAsync(b->prog_status.p, 0, (size_t)b->nprogs * 4, s));
  CUDA_TRY(c, cudaMemsetAsync(b->launch_dead.p, 0, std::max<size_t>(1, b->launches.size()) * 4, s));
  CUDA_TRY(c, cudaMemsetAsync(b->counters.p, 0, sizeof(sr::Counters), s));
  CUDA_TRY(c, cudaMemsetAsync(b->launch_done.p, 0, b->launches.size() * 4, s));
  CUDA_TRY(c, cudaMemsetAsync(b->total.p, 0, 8, s));
  CUDA_TRY(c, cudaMemsetAsync(b->err_flag.p, 0, 4, s));
  if (o.check_global) CUDA_TRY(c, cudaMemsetAsync(b->glog_n.p, 0, (size_t)b->nblocks * 4, s));
  mark();

  sr::RunArgs ra{};
  ra.launches = (const LaunchDev*)b->launches_d.p;
  ra.nlaunches = (uint32_t)b->launches.size();
  ra.budget = o.round_budget;
  ra.check_races = o.check_races;
  ra.spin_limit = o.spin_limit;
  ra.code = (const uint2*)b->code.p;
  ra.arena = (int32_t*)b->arena_work.p;
  ra.log = (unsigned long long*)b->log.p;
  ra.blocks = (sr::BlockRes*)b->blocks.p;
  ra.prog_status = (uint32_t*)b->prog_status.p;
  ra.launch_dead = (uint32_t*)b->launch_dead.p;
  ra.counters = (sr::Counters*)b->counters.p;
  ra.items = (const uint2*)b->items_d.p;
  ra.launch_done = (uint32_t*)b->launch_done.p;
  ra.glog = (uint4*)b->glog.p;
  ra.glog_n = (uint32_t*)b->glog_n.p;

  for (size_t wi = 0; wi < b->waves.size(); ++wi) {
    const Wave& w = b->waves[wi];
    if (o.mode == SR_MODE_BATCHED) {
      if (w.bq_blocks) {         // (two CTAs per SM) the wave's launches that run one block per CTA
        ra.bq_launch = (const uint32_t*)b->bq_launch_d.p + w.bq0;
        ra.bq_first = (const uint32_t*)b->bq_first_d.p + w.bq0;
        ra.bq_n = w.bq1 - w.bq0;
        ra.bq_head = (uint32_t*)b->bq_head.p + wi;
        CUDA_TRY(c, cudaMemsetAsync(ra.bq_head, 0, 4, s));
        CUDA_TRY(c, sr::launch_interp_blocks(ra, w.bq_blocks, b->blocks_smem, s));
        b->kernels += 1;
      }
      ra.items = (const uint2*)b->items_d.p + w.item0;
      ra.nitems = w.item1 - w.item0;
      ra.queue_head = (uint32_t*)b->queue_head.p + wi;
      CUDA_TRY(c, cudaMemsetAsync(ra.queue_head, 0, 4, s));
      const uint32_t ctas = std::min<uint32_t>(ra.nitems, (uint32_t)c->sms);
      if (ctas)
        CUDA_TRY(c, sr::launch_interp_batched(ra, ctas, b->batched_smem,
                                              o.fused_check && o.check_races && !o.check_global, o.check_global != 0,
                                              s));
      b->kernels += ctas ? 1 : 0;
    } else {
      for (uint32_t li = w.li0; li < w.li1; ++li)
        CUDA_TRY(c, sr::launch_interp_plain(ra, li, b->launches[li], o.interp_variant, s));
      b->kernels += w.li1 - w.li0;
    }
    mark();
    if (o.check_races) {
      sr::CheckArgs ca{};
      ca.launches = ra.launches;
      ca.li0 = w.li0;
      ca.li1 = w.li1;
      ca.item0 = b->launches[w.li0].check_item;
      ca.item1 = w.li1 < b->launches.size() ? b->launches[w.li1].check_item : b->check_items;
      ca.log = ra.log;
      ca.blocks = ra.blocks;
      ca.scratch = (uint4*)b->scratch.p;
      ca.work_head = (uint32_t*)b->work_head.p + wi;
      ca.error_flag = (uint32_t*)b->err_flag.p;
      ca.spin_limit = o.spin_limit;
      ca.table_words = sr::check_table_words(b->launches.data(), w.li0, w.li1, sr::check_table_cap(o.check_variant));
      ca.item_launch = (const uint32_t*)b->item_launch_d.p;
      CUDA_TRY(c, cudaMemsetAsync(ca.work_head, 0, 4, s));
      const uint32_t ctas = std::min<uint32_t>(b->check_ctas, ca.item1 - ca.item0);
      if (ctas) CUDA_TRY(c, sr::launch_check(ca, o.check_variant, ctas, s));
      b->kernels += ctas ? 1 : 0;
    }
    mark();
    if (w.glog_records) CUDA_TRY(c, sr::launch_gcheck(gcheck_args(c, b, (uint32_t)wi), b->kernels, s));
    mark();
    const sr::CompactArgs ka = compact_args(b, w);
    CUDA_TRY(c, sr::launch_compact_scan(ka, s));
    CUDA_TRY(c, sr::launch_compact_emit(ka, s));
    b->kernels += sr::compact_kernels(ka);
    mark();
  }
  return SR_OK;
}

}  // namespace

extern "C" {

int sr_create(sr_ctx** out, const sr_opts* opts) {
  if (!out) return fail(nullptr, SR_E_INVAL, "out is NULL");
  *out = nullptr;
  sr_ctx* c = new (std::nothrow) sr_ctx();
  if (!c) return fail(nullptr, SR_E_NOMEM, "host allocation failed");
  if (opts)
    c->opts = *opts;
  else
    c->opts.check_races = 1;
  sr_opts& o = c->opts;
  if (o.round_budget == 0) o.round_budget = 1u << 24;
  if (o.loop_log_records == 0) o.loop_log_records = 65536;
  if (o.ctas_per_sm == 0) o.ctas_per_sm = 1;
  if (o.spin_limit == 0) o.spin_limit = 1u << 26;
  if (o.round_budget > sr::kMaxBudget || o.mode > SR_MODE_BATCHED || o.interp_variant > 2 ||
      o.check_variant > SR_CHECK_VARIANTS) {
    delete c;
    return fail(nullptr, SR_E_INVAL, "round_budget above 2^26, or unknown mode or kernel variant");
  }
  if (o.allocator && o.allocator->alloc && o.allocator->release) {
    c->alloc = *o.allocator;
    c->custom_alloc = true;
  }
  o.allocator = nullptr;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->smem_optin = (size_t)optin;
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
  c->smem_per_sm = (size_t)per_sm;
  if (e == cudaSuccess) e = sr::init_kernel_attributes((uint32_t)optin);
  if (e == cudaSuccess && !c->custom_alloc) {
    // a pool of its own that keeps freed memory (batch after batch reuses it instead of
    // returning it to the driver at every synchronisation)
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = c->device;
    e = cudaMemPoolCreate(&c->pool, &pp);
    if (e == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    // memory freed on one stream is reused on that stream only: reuse across streams would
    // make batches on different streams wait for each other
    int no = 0;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowOpportunistic, &no);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
    return fail(nullptr, SR_E_CUDA, "device setup failed: %s", cudaGetErrorString(e));
  }
  *out = c;
  return SR_OK;
}

void sr_destroy(sr_ctx* c) {
  if (!c) return;
  if (c->pool) cudaMemPoolDestroy(c->pool);   // released once frees still in flight complete
  delete c;
}

const char* sr_last_error(sr_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

int sr_validate_program(const sr_program* prog, char* msg, size_t msg_len) {
  if (msg && msg_len) msg[0] = 0;
  return validate(prog, msg, msg_len);
}

int load_programs(sr_ctx* c, const sr_program* progs, uint32_t n, void* stream, sr_batch** out) {
  if (!c || !out || (n && !progs)) return fail(c, SR_E_INVAL, "null argument");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const sr_opts& o = c->opts;
  for (uint32_t i = 0; i < n; ++i) {
    char msg[256];
    if (validate(&progs[i], msg, sizeof msg) != SR_OK) return fail(c, SR_E_INVAL, "program %u: %s", i, msg);
  }
  sr_batch* b = new (std::nothrow) sr_batch();
  if (!b) return fail(c, SR_E_NOMEM, "host allocation failed");
  b->nprogs = n;
  b->stream = s;

  // ---- pack code and arenas, bound the logs
  std::vector<uint2> code;
  std::vector<uint32_t> code_off(n);
  b->arena_off.resize(n);
  b->arena_words.resize(n);
  uint64_t arena_total = 0;
  uint64_t nblocks = 0, check_items = 0;
  // shared memory of a CTA of the plain or the persistent batched kernel (one per SM)
  const uint32_t smem_budget =
      (uint32_t)std::min<size_t>(c->smem_optin ? c->smem_optin : 227 * 1024, 227 * 1024) - 1024;
  // batched mode with two CTAs per SM: a program whose every launch takes one group per
  // persistent CTA, and whose blocks fit two CTAs per SM, runs one block per CTA instead
  const bool hybrid = o.mode == SR_MODE_BATCHED && o.ctas_per_sm >= 2 && !o.fused_check && !o.check_global;
  const uint32_t blocks_cap =
      hybrid ? std::min<uint32_t>(smem_budget, sr::interp_blocks_smem_cap((uint32_t)c->smem_per_sm)) : 0u;
  for (uint32_t i = 0; i < n; ++i) {
    const sr_program& P = progs[i];
    code_off[i] = (uint32_t)code.size();
    const RegMap rm = map_registers(P);
    for (uint32_t pc = 0; pc < P.ncode; ++pc) code.push_back(pack(P.code[pc], rm));
    code.push_back(exit_sentinel(rm));
    set_run_lengths(code.data() + code_off[i], P.ncode + 1);
    if (code.size() & 1) code.push_back(exit_sentinel(rm));
    b->arena_off[i] = arena_total;
    b->arena_words[i] = P.global_words;
    arena_total += (P.global_words + 3) & ~3ull;
    std::vector<KernelBound> kb(P.nkernels);
    {
      std::vector<uint8_t> colour(P.ncode + 1);
      std::vector<uint32_t> acc(P.ncode + 1), bar(P.ncode + 1), spc(P.ncode + 1), snx(P.ncode + 1), gacc(P.ncode + 1);
      const BoundScratch ws{colour.data(), acc.data(), bar.data(), spc.data(), snx.data(), gacc.data()};
      for (uint32_t k = 0; k < P.nkernels; ++k) kb[k] = bound_kernel(P.code, P.ncode, P.kernel_entry[k], ws);
    }
    const uint32_t first_launch = (uint32_t)b->launches.size();   // the program's launches are contiguous
    bool one_all = P.nlaunches > 0;            // every launch of the program runs one block per CTA
    // the global-memory race check of a program whose launches are not all ordered needs its
    // launch-order matrix (and all its launches in one wave)
    uint32_t ord_off = sr::kNoDep;
    if (o.check_global && P.nlaunches > 1) {
      std::vector<uint32_t> bits;
      if (launch_order_bits(P.launches, P.nlaunches, bits)) {
        ord_off = (uint32_t)b->ord_bits_h.size();
        b->ord_bits_h.insert(b->ord_bits_h.end(), bits.begin(), bits.end());
      }
    }
    for (uint32_t l = 0; l < P.nlaunches; ++l) {
      const sr_launch& L = P.launches[l];
      LaunchDev d{};
      d.prog = i;
      d.launch = l;
      d.index = first_launch + l;
      launch_deps(P.launches, l, sr::kNoDep, d.dep_prev, d.dep_wait);
      if (d.dep_prev != sr::kNoDep) d.dep_prev += first_launch;
      if (d.dep_wait != sr::kNoDep) d.dep_wait += first_launch;
      d.entry = P.kernel_entry[L.kernel];
      d.ncode = P.ncode;
      d.code_off = code_off[i];
      d.grid = L.block_count ? L.block_count : L.grid;     // the blocks this batch runs
      d.gdim = L.grid;
      d.block_off = L.block_begin;
      d.bdim = L.block_dim;
      d.shw = L.shmem_words;
      d.nparams = L.nparams;
      for (uint32_t q = 0; q < 4; ++q) d.params[q] = q < L.nparams ? L.params[q] : 0;
      d.block_base = (uint32_t)nblocks;
      d.key_bits = key_bits_for(std::max(1u, L.shmem_words));
      const KernelBound& k = kb[L.kernel];
      const uint64_t cap = launch_log_cap(k, L.block_dim, o.check_races, o.loop_log_records);
      if (cap >= (1ull << 31)) {
        delete b;
        return fail(c, SR_E_INVAL, "program %u launch %u: access log bound too large", i, l);
      }
      d.log_cap = (uint32_t)cap;
      if (o.check_global) {
        const uint64_t gcap = launch_glog_cap(k, L.block_dim, o.loop_log_records);
        if (gcap >= (1ull << 31)) {
          delete b;
          return fail(c, SR_E_INVAL, "program %u launch %u: global log bound too large", i, l);
        }
        d.glog_cap = (uint32_t)gcap;
      }
      d.first_launch = first_launch;
      d.nl_prog = P.nlaunches;
      d.ord_off = ord_off;
      d.arena_off = b->arena_off[i];
      d.arena_words = P.global_words;
      d.ir_bytes = sr::ir_smem_bytes(P.ncode);
      d.nrows = rm.nrows;
      const uint32_t nw = (L.block_dim + 31) / 32;
      d.uninit = o.check_uninit ? 1u : 0u;
      // the fused race check where its summaries fit beside the block, else the access log
      d.fused = (o.fused_check && o.check_races && !o.check_global && L.shmem_words) ? 1u : 0u;
      d.group_bytes = sr::group_layout(nw * 32, L.shmem_words, P.ncode, rm.nrows, d.uninit, d.fused).total;
      if (d.fused && d.ir_bytes + d.group_bytes > smem_budget) {
        d.fused = 0;
        d.group_bytes = sr::group_layout(nw * 32, L.shmem_words, P.ncode, rm.nrows, d.uninit, 0).total;
      }
      if (d.ir_bytes + d.group_bytes > smem_budget) {
        delete b;
        return fail(c, SR_E_INVAL, "program %u launch %u: %u bytes of shared memory needed, %u available", i, l,
                    d.ir_bytes + d.group_bytes, smem_budget);
      }
      uint32_t g = std::min<uint32_t>(32 / nw, (smem_budget - d.ir_bytes) / d.group_bytes);
      one_all = one_all && hybrid && g == 1 && d.ir_bytes + d.group_bytes <= blocks_cap;
      if (nw >= 2) g = std::min<uint32_t>(g, 15);
      d.groups = std::max<uint32_t>(1, std::min<uint32_t>(g, d.grid));
      // blocks per work item: up to 8 rounds of `groups` while the launch still makes two
      // items per SM, so that a group that finishes early takes another block of the item
      // instead of waiting for the item's slowest block
      const uint32_t rounds = std::max<uint32_t>(1, std::min<uint32_t>(
          8, d.grid / std::max<uint32_t>(1, d.groups * 2u * (uint32_t)c->sms)));
      d.item_blocks = d.groups * rounds;
      d.check_group = sr::check_group_for(d.log_cap);
      d.check_item = (uint32_t)check_items;
      check_items += (d.grid + d.check_group - 1) / d.check_group;
      b->max_key_bits = std::max(b->max_key_bits, d.key_bits);
      nblocks += d.grid;
      if (nblocks >= (1ull << 31) || check_items >= (1ull << 31)) {
        delete b;
        return fail(c, SR_E_INVAL, "too many simulated blocks in one batch");
      }
      b->launches.push_back(d);
    }
    // (a program as a whole: the launches a launch follows are of its own program, and each of
    // the two kernels waits only on launches that it runs itself)
    b->one_per_cta.resize(b->launches.size(), one_all ? 1 : 0);
  }
  b->nblocks = (uint32_t)nblocks;
  b->check_items = (uint32_t)check_items;
  b->item_launch.resize(check_items);
  for (uint32_t li = 0; li < b->launches.size(); ++li) {
    const LaunchDev& d = b->launches[li];
    const uint32_t n = (d.grid + d.check_group - 1) / d.check_group;
    std::fill(b->item_launch.begin() + d.check_item, b->item_launch.begin() + d.check_item + n, li);
  }
  b->total_code = code.size();
  b->total_arena = arena_total;

  // ---- waves: consecutive launches whose logs fit the budget together
  size_t free_b = 0, tot_b = 0;
  cudaMemGetInfo(&free_b, &tot_b);
  const uint64_t budget_records =
      std::max<uint64_t>(1, (o.log_budget_mb ? (uint64_t)o.log_budget_mb << 20
                                             : std::min<uint64_t>(96ull << 30, (uint64_t)free_b / 2)) / 8);
  // (8-byte units per launch: its access logs, and with the global check its global logs,
  // 16 B per record, held three times: the per-block regions and the two sort buffers)
  uint64_t wave_max = 0, gwave_max = 0;
  {
    auto need_of = [&](const LaunchDev& d) {
      return (uint64_t)d.grid * d.log_cap + 6ull * d.grid * d.glog_cap;
    };
    Wave cur{0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t used = 0;
    for (uint32_t li = 0; li < b->launches.size(); ++li) {
      LaunchDev& d = b->launches[li];
      uint64_t need = need_of(d);
      // a program with unordered launches (global check) starts a wave only as a whole
      if (d.ord_off != sr::kNoDep && d.launch == 0)
        for (uint32_t m = li + 1; m < li + d.nl_prog; ++m) need += need_of(b->launches[m]);
      const bool split_ok = d.ord_off == sr::kNoDep || d.launch == 0;
      if (cur.li1 > cur.li0 && split_ok && used + need > budget_records) {
        b->waves.push_back(cur);
        wave_max = std::max(wave_max, cur.log_records);
        gwave_max = std::max(gwave_max, cur.glog_records);
        cur = Wave{li, li, d.block_base, d.block_base, 0, 0, 0, 0, 0};
        used = 0;
      }
      d.log_base = cur.log_records;
      d.glog_base = cur.glog_records;
      cur.log_records += (uint64_t)d.grid * d.log_cap;
      cur.glog_records += (uint64_t)d.grid * d.glog_cap;
      used += need_of(d);
      if (d.glog_cap) cur.addr_bits = std::max(cur.addr_bits, key_bits_for((uint32_t)std::min<uint64_t>(
                                                                 std::max<uint64_t>(1, d.arena_words), 1u << 31)));
      cur.li1 = li + 1;
      cur.gb1 = d.block_base + d.grid;
    }
    if (cur.li1 > cur.li0) {
      b->waves.push_back(cur);
      wave_max = std::max(wave_max, cur.log_records);
      gwave_max = std::max(gwave_max, cur.glog_records);
    }
  }
  b->log_records = wave_max;
  b->glog_records = gwave_max;
  b->entry_cap = std::max<uint64_t>(1024, std::min<uint64_t>(gwave_max, o.report_cap ? o.report_cap : 1u << 20));

  // ---- batched work items: per wave, launch-index order, blocks in chunks of `item_blocks`;
  // with two CTAs per SM the launches that run one block per CTA go to the wave's block queue
  // instead, in the same order
  b->batched_smem = 0;
  b->blocks_smem = 0;
  b->bq_blocks = 0;
  for (Wave& w : b->waves) {
    w.item0 = (uint32_t)b->items.size();
    w.bq0 = (uint32_t)b->bq_launch.size();
    w.bq_blocks = 0;
    uint32_t maxl = 0;
    for (uint32_t li = w.li0; li < w.li1; ++li) maxl = std::max(maxl, b->launches[li].launch);
    for (uint32_t lv = 0; lv <= maxl; ++lv)
      for (uint32_t li = w.li0; li < w.li1; ++li) {
        const LaunchDev& d = b->launches[li];
        if (d.launch != lv || d.grid == 0) continue;
        if (b->one_per_cta[li]) {
          b->bq_launch.push_back(li);
          b->bq_first.push_back(w.bq_blocks);
          w.bq_blocks += d.grid;
          b->blocks_smem = std::max(b->blocks_smem, d.ir_bytes + d.group_bytes);
          continue;
        }
        for (uint32_t blk = 0; blk < d.grid; blk += d.item_blocks) b->items.push_back(make_uint2(li, blk));
        b->batched_smem = std::max(b->batched_smem, d.ir_bytes + d.groups * d.group_bytes);
      }
    w.item1 = (uint32_t)b->items.size();
    w.bq1 = (uint32_t)b->bq_launch.size();
    b->bq_blocks += w.bq_blocks;
  }
  b->check_ctas = (uint32_t)c->sms * sr::check_ctas_per_sm(o.check_variant);

  // ---- device buffers
  int rc = SR_OK;
  const size_t nl = b->launches.size();
  const uint32_t nwaves = (uint32_t)b->waves.size();
  b->out_cap = o.report_cap ? o.report_cap : (1u << 20);
  struct A { DevBuf* buf; size_t bytes; const char* what; } allocs[] = {
      {&b->code, b->total_code * 8, "code"},
      {&b->launches_d, std::max<size_t>(1, nl) * sizeof(LaunchDev), "launch table"},
      {&b->arena_init, b->total_arena * 4, "initial arenas"},
      {&b->arena_work, b->total_arena * 4, "working arenas"},
      {&b->log, b->log_records * 8, "access log"},
      {&b->blocks, (size_t)b->nblocks * sizeof(sr::BlockRes), "block results"},
      {&b->prog_status, (size_t)n * 4, "status"},
      {&b->launch_dead, std::max<size_t>(1, b->launches.size()) * 4, "launch stop marks"},
      {&b->counters, sizeof(sr::Counters), "counters"},
      {&b->items_d, std::max<size_t>(1, b->items.size()) * 8, "work items"},
      {&b->queue_head, (size_t)nwaves * 4, "queue heads"},
      {&b->launch_done, std::max<size_t>(1, nl) * 4, "launch completion"},
      {&b->scratch, (size_t)b->check_ctas * sr::kScratchWords * 16, "checker scratch"},
      {&b->work_head, (size_t)nwaves * 4, "checker queue"},
      {&b->err_flag, 4, "error flag"},
      {&b->offsets, ((size_t)b->nblocks + 1) * 8, "report offsets"},
      {&b->partials, sr::compact_partials_count(b->nblocks) * 8, "scan partials"},
      {&b->out, b->out_cap * sizeof(sr_report), "reports"},
      {&b->total, 8, "report total"},
      {&b->item_launch_d, std::max<size_t>(1, b->item_launch.size()) * 4, "check item table"},
      {&b->bq_launch_d, std::max<size_t>(1, b->bq_launch.size()) * 4, "block queue launches"},
      {&b->bq_first_d, std::max<size_t>(1, b->bq_first.size()) * 4, "block queue tickets"},
      {&b->bq_head, (size_t)nwaves * 4, "block queue heads"},
      // global-memory race check (16-byte stand-ins when off)
      {&b->glog, (size_t)b->glog_records * 16, "global logs"},
      {&b->glog_n, o.check_global ? (size_t)b->nblocks * 4 : 0, "global log counts"},
      {&b->goff, o.check_global ? ((size_t)b->nblocks + 1) * 8 : 0, "global log offsets"},
      {&b->gpartials, o.check_global ? sr::gcheck_partials(b->nblocks) * 8 : 0, "global scan partials"},
      {&b->gtotal, 8, "global record total"},
      {&b->sort_a, (size_t)b->glog_records * 16, "global sort buffer"},
      {&b->sort_b, (size_t)b->glog_records * 16, "global sort buffer"},
      {&b->hist, o.check_global ? (size_t)12 * 256 * 8 : 0, "digit histograms"},
      {&b->status, o.check_global ? sr::gcheck_tiles(std::max(b->glog_records, b->entry_cap)) * 256 * 8 : 0,
       "sort tile states"},
      {&b->tile_ctr, 12 * 4, "sort tile counters"},
      {&b->ord_bits, std::max<size_t>(1, b->ord_bits_h.size()) * 4, "launch-order matrices"},
      {&b->entries_a, o.check_global ? (size_t)b->entry_cap * 32 : 0, "global race entries"},
      {&b->entries_b, o.check_global ? (size_t)b->entry_cap * 32 : 0, "global race entries"},
      {&b->gn, (size_t)nwaves * 8, "global entry counts"},
      {&b->gcount, o.check_global ? (size_t)b->nblocks * 4 : 0, "global entries per block"},
      {&b->gstart, o.check_global ? ((size_t)b->nblocks + 1) * 8 : 0, "global entry offsets"},
      {&b->gn_sorted, 8, "global entry total"},
  };
  for (auto& a : allocs) {
    rc = alloc_buf(c, *a.buf, a.bytes, s, a.what);
    if (rc) {
      free_batch_buffers(c, b, s);
      delete b;
      return rc;
    }
  }
  auto up = [&](DevBuf& d, const void* src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  cudaError_t e = up(b->code, code.data(), code.size() * 8);
  if (e == cudaSuccess) e = up(b->launches_d, b->launches.data(), nl * sizeof(LaunchDev));
  if (e == cudaSuccess) e = up(b->items_d, b->items.data(), b->items.size() * 8);
  if (e == cudaSuccess) e = up(b->item_launch_d, b->item_launch.data(), b->item_launch.size() * 4);
  if (e == cudaSuccess) e = up(b->bq_launch_d, b->bq_launch.data(), b->bq_launch.size() * 4);
  if (e == cudaSuccess) e = up(b->bq_first_d, b->bq_first.data(), b->bq_first.size() * 4);
  if (e == cudaSuccess) e = up(b->ord_bits, b->ord_bits_h.data(), b->ord_bits_h.size() * 4);
  // every arena starts on a 16-byte boundary; the up to three padding words after it are
  // zeroed by copies too, not by a memset: a memset is a kernel, which would wait for SMs that
  // other batches' kernels hold, and the synchronisation below would wait with it
  static const int32_t kZeros[4] = {0, 0, 0, 0};
  for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
    int32_t* dst = (int32_t*)b->arena_init.p + b->arena_off[i];
    if (progs[i].global_words)
      e = cudaMemcpyAsync(dst, progs[i].global_init, progs[i].global_words * 4, cudaMemcpyHostToDevice, s);
    const uint64_t pad = ((b->arena_words[i] + 3) & ~3ull) - b->arena_words[i];
    if (pad && e == cudaSuccess)
      e = cudaMemcpyAsync(dst + b->arena_words[i], kZeros, pad * 4, cudaMemcpyHostToDevice, s);
  }
  // host buffers are caller-owned: the copies must finish before we return
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_batch_buffers(c, b, s);
    delete b;
    return fail(c, SR_E_CUDA, "upload failed: %s", cudaGetErrorString(e));
  }
  *out = b;
  return SR_OK;
}

int run_and_check(sr_ctx* c, sr_batch* b, void* stream) {
  if (!c || !b) return fail(c, SR_E_INVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  b->stream = s;
  b->ran = true;
  const bool profile = c->opts.profile != 0;
  if (c->opts.use_graph && c->opts.mode == SR_MODE_BATCHED && !profile) {
    if (!b->graph || b->graph_stream != s) {
      if (b->graph) cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
      cudaStream_t cap;
      CUDA_TRY(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      CUDA_TRY(c, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue_run(c, b, cap, false);
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap, &g);
      cudaStreamDestroy(cap);
      if (rc) return rc;
      if (e != cudaSuccess) return fail(c, SR_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail(c, SR_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
      b->graph_stream = s;
    }
    CUDA_TRY(c, cudaGraphLaunch(b->graph, s));
    return SR_OK;
  }
  return enqueue_run(c, b, s, profile);
}

int fetch_reports(sr_ctx* c, sr_batch* b, sr_report* dst, uint64_t cap, uint64_t* n_total) {
  if (!c || !b) return fail(c, SR_E_INVAL, "null argument");
  if (!b->ran) return fail(c, SR_E_INVAL, "run_and_check has not been called");
  cudaStream_t s = b->stream;
  if (c->opts.check_global) {
    // a wave's global race entries outgrew their buffer: grow it and run again (runs are
    // deterministic; the entries of every wave then fit)
    std::vector<unsigned long long> gn(b->waves.size());
    CUDA_TRY(c, cudaMemcpyAsync(gn.data(), b->gn.p, gn.size() * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    const unsigned long long need = gn.empty() ? 0 : *std::max_element(gn.begin(), gn.end());
    if (need > b->entry_cap) {
      dev_free(c, b->entries_a, s);
      dev_free(c, b->entries_b, s);
      dev_free(c, b->status, s);
      b->entry_cap = need + need / 8 + 1024;
      int rc = alloc_buf(c, b->entries_a, b->entry_cap * 32, s, "global race entries");
      if (!rc) rc = alloc_buf(c, b->entries_b, b->entry_cap * 32, s, "global race entries");
      if (!rc)
        rc = alloc_buf(c, b->status, sr::gcheck_tiles(std::max(b->glog_records, b->entry_cap)) * 256 * 8, s,
                       "sort tile states");
      if (rc) return rc;
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      rc = run_and_check(c, b, s);
      if (rc) return rc;
    }
  }
  unsigned long long total = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&total, b->total.p, 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  if (total > b->out_cap) {
    // The report buffer was too small: grow it.  With one wave, that wave's logs, block
    // results and report offsets are all still on the device, so only the emission runs
    // again; with several, later waves reused the log pool and the whole run is repeated
    // (runs are deterministic).
    dev_free(c, b->out, s);
    b->out_cap = total + total / 8 + 1024;
    int rc = alloc_buf(c, b->out, b->out_cap * sizeof(sr_report), s, "reports");
    if (rc) return rc;
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    if (b->waves.size() == 1) {
      CUDA_TRY(c, sr::launch_compact_emit(compact_args(b, b->waves[0]), s));
    } else {
      rc = run_and_check(c, b, s);
      if (rc) return rc;
      CUDA_TRY(c, cudaMemcpyAsync(&total, b->total.p, 8, cudaMemcpyDeviceToHost, s));
      CUDA_TRY(c, cudaStreamSynchronize(s));
    }
  }
  uint32_t err = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&err, b->err_flag.p, 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  if (n_total) *n_total = total;
  if (err & sr::kErrBounds) return fail(c, SR_E_BOUNDS, "an internal index check failed (debug build)");
  if (err & sr::kErrCorrupt) return fail(c, SR_E_TIMEOUT, "the race checker found an access log out of order");
  if (err) return fail(c, SR_E_TIMEOUT, "a device-side wait of the checks gave up");
  if (!dst) return SR_OK;
  if (cap < total) return fail(c, SR_E_RANGE, "report buffer holds %llu, %llu needed", (unsigned long long)cap, total);
  if (total) CUDA_TRY(c, cudaMemcpyAsync(dst, b->out.p, total * sizeof(sr_report), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(c, cudaStreamSynchronize(s));
  return SR_OK;
}

int fetch_memory(sr_ctx* c, sr_batch* b, uint32_t prog, int32_t* dst, uint64_t cap_words, uint64_t* n_words) {
  if (!c || !b) return fail(c, SR_E_INVAL, "null argument");
  const bool all = prog == SR_ALL_PROGRAMS;
  if (!all && prog >= b->nprogs) return fail(c, SR_E_INVAL, "program %u out of range", prog);
  // arenas are laid out back to back in program order
  const uint64_t nw = all ? b->total_arena : b->arena_words[prog];
  const uint64_t off = all ? 0 : b->arena_off[prog];
  if (n_words) *n_words = nw;
  if (!dst) return SR_OK;
  if (cap_words < nw) return fail(c, SR_E_RANGE, "arena has %llu words", (unsigned long long)nw);
  const DevBuf& src = b->ran ? b->arena_work : b->arena_init;
  if (nw) CUDA_TRY(c, cudaMemcpyAsync(dst, (int32_t*)src.p + off, nw * 4, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(c, cudaStreamSynchronize(b->stream));
  return SR_OK;
}

int sr_batch_status(sr_ctx* c, sr_batch* b, uint32_t prog, uint32_t* status) {
  if (!c || !b || !status) return fail(c, SR_E_INVAL, "null argument");
  const bool all = prog == SR_ALL_PROGRAMS;
  if (!all && prog >= b->nprogs) return fail(c, SR_E_INVAL, "program %u out of range", prog);
  CUDA_TRY(c, cudaMemcpyAsync(status, (uint32_t*)b->prog_status.p + (all ? 0 : prog),
                              4 * (all ? b->nprogs : 1), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(c, cudaStreamSynchronize(b->stream));
  return SR_OK;
}

int sr_batch_stats(sr_ctx* c, sr_batch* b, sr_stats* out) {
  if (!c || !b || !out) return fail(c, SR_E_INVAL, "null argument");
  memset(out, 0, sizeof(*out));
  sr::Counters k{};
  CUDA_TRY(c, cudaMemcpyAsync(&k, b->counters.p, sizeof k, cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(c, cudaStreamSynchronize(b->stream));
  out->thread_instrs = k.thread_instrs;
  out->shared_accesses = k.shared_accesses;
  out->global_accesses = k.global_accesses;
  out->reports = k.total_reports;
  out->log_bytes = b->log_records * 8;
  out->blocks = b->nblocks;
  out->waves = (uint32_t)b->waves.size();
  out->kernels = b->kernels;
  out->one_per_cta_blocks = b->bq_blocks;
  out->global_records = k.global_records;
  if (c->opts.profile && b->nevents_used >= 2) {
    float ms = 0;
    cudaEventElapsedTime(&ms, b->events[0], b->events[1]);
    out->ms_reset = ms;
    for (uint32_t i = 1; i + 4 < b->nevents_used; i += 4) {   // per wave: interp, check, global, compact
      float t;
      cudaEventElapsedTime(&t, b->events[i], b->events[i + 1]);
      out->ms_interp += t;
      cudaEventElapsedTime(&t, b->events[i + 1], b->events[i + 2]);
      out->ms_check += t;
      cudaEventElapsedTime(&t, b->events[i + 2], b->events[i + 3]);
      out->ms_global += t;
      cudaEventElapsedTime(&t, b->events[i + 3], b->events[i + 4]);
      out->ms_compact += t;
    }
  }
  return SR_OK;
}

void sr_free_batch(sr_ctx* c, sr_batch* b) {
  if (!c || !b) return;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  free_batch_buffers(c, b, b->stream);
  cudaStreamSynchronize(b->stream);
  delete b;
}

}  // extern "C"
