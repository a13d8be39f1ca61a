/*
 * simtcheck.h - C ABI of the GB300 SIMT race and barrier checker (libsimtcheck.so).
 *
 * The library executes simulated CUDA-C kernels for many threads at once and checks
 * them the way the paper's cudak tool does (Hathhorn, Becchi, Harrison, Procter,
 * "Formal Semantics of Heterogeneous CUDA-C", SSV 2012):
 *   - every kernel launch creates grid x blockDim threads with a per-block dynamic
 *     shared array; launches of one program run in order over one global arena with
 *     the implicit grid-wide synchronisation at the end of each kernel call
 *     (Sec. 2; Sec. 3 "Threads and memory");
 *   - every shared-memory access is logged and each barrier interval is checked for
 *     races: two distinct threads, same location, no barrier in between, at least one
 *     write (Sec. 3.1, first paragraph);
 *   - every __syncthreads() is checked: threads of a block waiting at different barrier
 *     instructions (divergence), or waiting while other threads have exited (deadlock,
 *     Sec. 3.1, last paragraph; Sec. 3 "Barrier synchronization").
 * Programs are given in a small int32 register IR instead of C source.
 *
 * Conventions for every entry point
 *   - Return 0 on success or a negative SR_E_* code; the message of the last failure
 *     of a context is returned by sr_last_error().  On SR_E_INVAL nothing was enqueued.
 *   - Host buffers passed in are owned by the caller and only read (or, for fetch_*,
 *     written) during the call.  Device memory is owned by the library: it is obtained
 *     through the allocator given at sr_create (default: stream-ordered allocation from a
 *     memory pool owned by the context) and released by sr_free_batch / sr_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  run_and_check only
 *     enqueues work; fetch_* and sr_batch_status synchronise the batch's stream.
 *   - Races, deadlocks, divergent barriers, out-of-bounds accesses, division by zero and
 *     the round budget are *reports* about the simulated program, never error codes.
 *   - A context and its batches are not thread-safe: use one host thread per context.
 *
 * Instruction encoding (8 bytes): op_d_a_b = op | d << 8 | a << 16 | b << 24, imm.
 *   op bits 0..5 opcode, bit 7 SR_BIMM (second ALU operand is imm instead of register b).
 *   Registers r0..r15; 255 (SR_RZ) reads 0 and drops writes.  Word addresses.
 *   MOV d,B | ADD..SNE d,a,B | S2R d,#sreg | LDG d,[a+imm] | STG [a+imm],b
 *   LDS d,[a+imm] | STS [a+imm],b | ATOMS [a+imm],b (add, no return)
 *   BRA #t | BRZ a,#t | BRNZ a,#t (absolute pcs in 0..ncode) | BAR | EXIT
 *   BARAND d,a | BAROR d,a | BARPOPC d,a: __syncthreads_and/_or/_count (Sec. 3 feature
 *   list): a barrier like BAR whose thread contributes the predicate a != 0; when the
 *   barrier releases, d = 1 if every / some released thread's predicate holds, or the
 *   number that hold (threads released from a plain BAR contribute 0).
 *   At launch r0..r(nparams-1) hold the params, every other register 0; shared memory
 *   starts zeroed; running past the last instruction exits the thread.
 *
 * Execution model (the paper leaves the scheduler open, Sec. 3 "Threads and memory"
 * and Sec. 4; this library fixes one schedule so that results are reproducible):
 * warps of 32 consecutive tids advance in rounds; in each round every warp with a
 * runnable thread executes the lowest pc among its runnable threads for the threads at
 * that pc; all loads of a round see the state before the round, then stores apply in
 * ascending tid order, then atomic adds.  When no thread of a block can run the barrier
 * is resolved: no waiting threads -> the block is done; waiting and exited threads ->
 * DEADLOCK (the block stops and the program's later launches are skipped); waiting at
 * different barrier pcs -> DIVERGENCE, then release; otherwise release.
 */
#ifndef SIMTCHECK_H
#define SIMTCHECK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* opaque handles: a context (one CUDA device, options, allocator) and a loaded batch */
typedef struct sr_ctx sr_ctx;
typedef struct sr_batch sr_batch;

/* ---------------------------------------------------------------- return codes */
#define SR_OK 0
#define SR_E_INVAL (-1)    /* bad argument or program (validation failure) */
#define SR_E_NOMEM (-2)    /* device or host allocation failed */
#define SR_E_CUDA (-3)     /* a CUDA call failed; see sr_last_error */
#define SR_E_TIMEOUT (-4)  /* a device-side wait gave up (bounded spin) */
#define SR_E_RANGE (-5)    /* destination buffer too small (size returned) */
#define SR_E_BOUNDS (-6)   /* library built with SR_DEBUG_BOUNDS: an internal index check failed in a
                              kernel (the access was skipped); the results are invalid */

/* ---------------------------------------------------------------- IR opcodes */
enum {
  SR_OP_MOV = 1, SR_OP_ADD, SR_OP_SUB, SR_OP_MUL, SR_OP_DIV, SR_OP_REM, SR_OP_AND, SR_OP_OR,
  SR_OP_XOR, SR_OP_SHL, SR_OP_SHR, SR_OP_MIN, SR_OP_MAX, SR_OP_SLT, SR_OP_SLE, SR_OP_SEQ,
  SR_OP_SNE, SR_OP_S2R, SR_OP_LDG, SR_OP_STG, SR_OP_LDS, SR_OP_STS, SR_OP_ATOMS, SR_OP_BRA,
  SR_OP_BRZ, SR_OP_BRNZ, SR_OP_BAR, SR_OP_EXIT, SR_OP_BARAND, SR_OP_BAROR, SR_OP_BARPOPC
};
#define SR_BIMM 0x80u
#define SR_RZ 0xFFu
enum { SR_SREG_TID = 0, SR_SREG_BID, SR_SREG_BDIM, SR_SREG_GDIM, SR_SREG_WARPSIZE };

#define SR_MAX_CODE 4096u          /* instructions per program (pcs fit in 12 bits) */
#define SR_MAX_BLOCK_DIM 1024u     /* threads per block (tids fit in 10 bits) */
#define SR_MAX_SHMEM_WORDS 12288u  /* 48 KB of simulated shared memory per block */

/* ---------------------------------------------------------------- report records */
enum {
  SR_REP_RACE = 1,           /* a = word address, b = t1 << 16 | t2 (smallest conflicting
                                pair, t1 < t2), c = class << 24 | pc_lo << 12 | pc_hi over all
                                accesses to the word in the interval */
  SR_REP_DIVERGENCE = 2,     /* a = lowest, b = highest barrier pc waited at, c = nwait << 16 */
  SR_REP_DEADLOCK = 3,       /* a, b as above, c = nwait << 16 | nexited */
  SR_REP_STEP_LIMIT = 4,     /* a = rounds executed, b = runnable threads, c = their lowest pc */
  SR_REP_ERR_OOB_SHARED = 5, /* a = pc, b = lowest tid, c = thread executions in the interval */
  SR_REP_ERR_OOB_GLOBAL = 6, /* same fields */
  SR_REP_ERR_DIV0 = 7,       /* same fields */
  SR_REP_ERR_UNINIT_SHARED = 8, /* (with opts.check_uninit) a shared load of a word no thread of the
                                  block stored or added to in an earlier round; same fields */
  /* with opts.check_global (Sec. 3.1's race definition on global words): */
  SR_REP_GLOBAL_RACE = 9,    /* inside a barrier interval of a block: a = word of the program's
                                arena, b and c as for SR_REP_RACE (classes WW and WR) */
  SR_REP_GLOBAL_BLOCKS = 10, /* between blocks of one launch (nothing orders them before the kernel
                                call ends, Sec. 2): block = b1, epoch = 0, a = word, b = b2 (b1 < b2,
                                the smallest conflicting pair of blocks), c = class << 24 | pc_lo << 12
                                | pc_hi over the launch's accesses to the word */
  SR_REP_GLOBAL_LAUNCHES = 11 /* between launches that no stream order or event wait orders (Sec. 3,
                                streams and events): launch = l1, block = 0, epoch = 0, a = word,
                                b = l2 (l1 < l2, the smallest such conflicting pair), c = class << 24
                                over every such pair */
};
enum { SR_CLS_WW = 1, SR_CLS_WR = 2, SR_CLS_WA = 4, SR_CLS_AR = 8 };

/* per-program status bits (sr_batch_status) */
enum {
  SR_ST_DEADLOCK = 1,        /* a block deadlocked; later launches were skipped */
  SR_ST_STEP_LIMIT = 2,      /* a block ran out of rounds; later launches were skipped */
  SR_ST_LOG_OVERFLOW = 4,    /* a block's access log exceeded its region: race check incomplete */
  SR_ST_INTERNAL = 8,        /* a device-side wait timed out: results of the program are invalid */
  SR_ST_BOUNDS = 16          /* library built with SR_DEBUG_BOUNDS: an index check of the interpreter
                                failed for this program (the access was skipped); results invalid */
};

typedef struct { uint32_t op_d_a_b; int32_t imm; } sr_instr;

typedef struct {
  uint32_t kernel;           /* index into the program's kernel_entry */
  uint32_t grid;             /* blocks, >= 1 */
  uint32_t block_dim;        /* threads per block, 1..SR_MAX_BLOCK_DIM */
  uint32_t shmem_words;      /* dynamic shared words per block, 0..SR_MAX_SHMEM_WORDS */
  uint32_t nparams;          /* 0..4, loaded into r0.. */
  int32_t params[4];
  /* Sec. 2 and Sec. 3 "Streams and events": launches of one stream run in order, launches of
   * different streams may run at the same time.  `wait` = 1 + the index of an earlier launch
   * of the program that this one also waits for (an event recorded after that launch and
   * waited for by this launch's stream); 0 = none.  All zero: one in-order stream.  A launch
   * is skipped when the previous launch of its stream, or the one it waits for, stopped
   * (deadlock, step limit) or was skipped.  Launches that nothing orders must not share a
   * global word that one of them writes (the result would depend on timing; not checked). */
  uint32_t stream;
  uint32_t wait;             /* 0..index of this launch; SR_E_INVAL otherwise */
  /* Run only blocks [block_begin, block_begin + block_count) of the grid (a process's share
   * of a launch whose blocks are split across processes, Sec. 2: the blocks of a grid are
   * independent until the kernel call ends).  Block indices (S2R BID, reports) and GDIM keep
   * the whole grid's numbering.  block_count 0 = every block (block_begin must be 0). */
  uint32_t block_begin;
  uint32_t block_count;
} sr_launch;

typedef struct {
  const sr_instr* code; uint32_t ncode;           /* 1..SR_MAX_CODE instructions */
  const uint32_t* kernel_entry; uint32_t nkernels;
  const sr_launch* launches; uint32_t nlaunches;  /* run in stream order (sr_launch) */
  const int32_t* global_init; uint64_t global_words;  /* initial global arena (< 2^31 words) */
} sr_program;

/* one report; fetch_reports returns them sorted by (prog, launch, block, epoch, kind, a, b, c) */
typedef struct { uint32_t kind, prog, launch, block, epoch, a, b, c; } sr_report;

/* optional device allocator (e.g. a framework's caching allocator) */
typedef struct {
  void* (*alloc)(void* user, size_t bytes, void* stream);        /* NULL return = failure */
  void (*release)(void* user, void* ptr, size_t bytes, void* stream);
  void* user;
} sr_allocator;

enum { SR_MODE_PLAIN = 0,    /* one kernel launch per (program, launch) */
       SR_MODE_BATCHED = 1   /* one persistent launch over every block of every program */ };

typedef struct {
  uint32_t check_races;      /* 1 = log + race check (default), 0 = interpreter + barrier check only */
  uint32_t round_budget;     /* rounds per block before STEP_LIMIT; 0 = 1 << 24 (max 1 << 26) */
  uint32_t mode;             /* SR_MODE_* */
  uint32_t ctas_per_sm;      /* batched mode: 1 (0) = every launch in the persistent interpreter, one
                                1024-thread CTA per SM; 2 = the programs whose every launch would take
                                one group per persistent CTA (blocks of more than 512 threads, or
                                shared arrays that leave room for one) and whose blocks fit two CTAs
                                per SM run one simulated block per CTA, two CTAs per SM, all such
                                launches of a wave in one grid; the other programs stay persistent.
                                Without effect with fused_check or check_global */
  uint32_t loop_log_records; /* log region (records per block) for kernels with loops; 0 = 65536 */
  uint32_t interp_variant;   /* plain-mode interpreter: 1 = one 1024-thread CTA per SM budget,
                                2 = registers capped for two per SM, 0 = pick by occupancy */
  uint32_t use_graph;        /* batched mode: capture run_and_check once, replay as a CUDA graph */
  uint32_t profile;          /* record CUDA events between stages (sr_batch_stats) */
  uint32_t spin_limit;       /* device wait iterations before SR_ST_INTERNAL; 0 = 1 << 26 */
  uint32_t log_budget_mb;    /* device memory for access logs resident at once (launches are
                                processed in waves that fit); 0 = min(96 GB, half the free memory) */
  uint32_t report_cap;       /* initial report buffer (records); grown on demand; 0 = 1 << 20 */
  const sr_allocator* allocator;  /* NULL = stream-ordered allocation from a memory pool the
                                     context owns (freed memory is kept for reuse until
                                     sr_destroy) */
  uint32_t check_variant;    /* race-check kernel shape, 1..SR_CHECK_VARIANTS (consumer threads,
                                records per stage, staging, CTAs per SM, address-table size);
                                0 = the default */
  uint32_t check_uninit;     /* 1 = also report loads of shared words not yet written
                                (SR_REP_ERR_UNINIT_SHARED); 0 = off */
  uint32_t fused_check;      /* 1 = the interpreter keeps each shared word's access summary itself
                                (Sec. 3.1's per-location history, cleared at every barrier) and
                                writes no access log, for every launch whose summaries fit in
                                shared memory beside the block; same reports.  0 = access log +
                                race-check kernel */
  uint32_t check_global;     /* 1 = also check global memory for races (SR_REP_GLOBAL_*): every global
                                load and store is logged (16 B) and the logs are grouped by word with a
                                radix sort.  A program whose launches are not all ordered keeps its
                                launches in one wave; fused_check is ignored (the log path runs).
                                Programs racing on global memory have timing-dependent memory images:
                                the reports are exact, the racing words are not.  0 = off */
} sr_opts;

#define SR_CHECK_VARIANTS 7

typedef struct {
  uint64_t thread_instrs;    /* simulated thread-instructions executed */
  uint64_t shared_accesses;  /* logged shared accesses (records through the race check) */
  uint64_t global_accesses;  /* simulated LDG + STG thread executions */
  uint64_t reports;          /* reports produced */
  uint64_t log_bytes;        /* bytes of access-log capacity reserved on the device */
  uint64_t blocks;           /* simulated blocks in the batch */
  float ms_reset, ms_interp, ms_check, ms_compact;   /* last run, when opts.profile */
  uint32_t waves;            /* launch groups whose logs were resident together in the last run */
  uint32_t kernels;          /* kernel launches of the library enqueued by the last run */
  float ms_global;           /* last run, when opts.profile: the global-memory race check */
  uint64_t global_records;   /* global accesses logged for the global-memory race check (last run) */
  uint64_t one_per_cta_blocks; /* batched mode, ctas_per_sm 2: blocks run one per CTA in a run */
} sr_stats;

/* Create a context on the current CUDA device.  opts may be NULL (defaults). */
int sr_create(sr_ctx** out, const sr_opts* opts);
void sr_destroy(sr_ctx* ctx);

/* Host-only validation of one program (no CUDA call).  Writes a message on failure. */
int sr_validate_program(const sr_program* prog, char* msg, size_t msg_len);

/* Validate, pack and upload n programs (code, launch tables, initial arenas) into
 * device-resident arenas; returns a batch handle.  The initial arenas stay resident so
 * that run_and_check can be repeated.  Enqueued on `stream`.
 * Paper: Sec. 2 (the host allocates device memory, copies the inputs and configures each
 * kernel call <<<grid, block, shared bytes, stream>>>) and Fig. 1 lines 22-34 (the sum
 * program's host side); here the host program is replaced by the sr_program descriptor.
 *   progs   host array of n descriptors, read during the call only (copied to the device);
 *   stream  cudaStream_t for the uploads (the call waits for them before returning);
 *   out     receives the batch handle (NULL on failure).
 * Errors: SR_E_INVAL (a program fails validation; nothing is enqueued), SR_E_NOMEM,
 * SR_E_CUDA. */
int load_programs(sr_ctx* ctx, const sr_program* progs, uint32_t n, void* stream, sr_batch** out);

/* Reset every program's global arena to its initial image, run all launches of all
 * programs, check the access logs and barriers, and order the reports.  Asynchronous
 * on `stream`.
 * Paper: Sec. 3 "Threads and memory" (every thread of the grid runs the kernel; per-block
 * shared memory) and "Barrier synchronization" (__syncthreads); Sec. 3.1 (race detection:
 * two threads, one shared location, no barrier between, at least one write; the history
 * is cleared at each barrier; deadlock detection at a barrier some thread never reaches).
 * Errors: SR_E_INVAL (null handle), SR_E_CUDA (a launch failed).  Races, deadlocks and
 * the other findings about the simulated program are reports, not errors. */
int run_and_check(sr_ctx* ctx, sr_batch* batch, void* stream);

/* Copy the sorted reports to dst (capacity cap records) and the total into *n_total.
 * dst == NULL only queries the size.  SR_E_RANGE if cap < total (dst untouched).
 * Paper: Sec. 3.2 (cudak prints its diagnostics - a possible race on shared memory and
 * the source line, or a deadlock caused by a misplaced __syncthreads - beside the
 * program's output); here each diagnostic is one sr_report record.
 *   dst  host memory (pageable or page-locked) for cap records, owned by the caller.
 * Synchronises with the batch's stream.  SR_E_TIMEOUT if a device-side wait of the race
 * check gave up (the reports are then incomplete). */
int fetch_reports(sr_ctx* ctx, sr_batch* batch, sr_report* dst, uint64_t cap, uint64_t* n_total);

/* prog value of fetch_memory / sr_batch_status that addresses every program at once. */
#define SR_ALL_PROGRAMS 0xFFFFFFFFu

/* Paper: Sec. 3.2 (the program's own output, e.g. Fig. 1's OUTPUT 767, read back from
 * device memory by the host program).
 * Copy program `prog`'s final global arena (n_words = its size) to dst.  With
 * prog == SR_ALL_PROGRAMS every arena is copied in one copy, in program order, program k's
 * at word offset sum over i < k of round_up(global_words_i, 4) (each arena starts on a
 * 16-byte boundary; padding words are zero); n_words = that sum over all programs.  dst == NULL only queries the size;
 * SR_E_RANGE if cap_words < n_words.  Synchronises with the batch's stream; dst may be
 * pageable or page-locked host memory (page-locked copies run at link speed). */
int fetch_memory(sr_ctx* ctx, sr_batch* batch, uint32_t prog, int32_t* dst, uint64_t cap_words,
                 uint64_t* n_words);

/* SR_ST_* bits of program `prog` after the last run_and_check; with prog ==
 * SR_ALL_PROGRAMS, status points to an array of the batch's n programs' bits. */
int sr_batch_status(sr_ctx* ctx, sr_batch* batch, uint32_t prog, uint32_t* status);

/* Counters of the last run (synchronises). */
int sr_batch_stats(sr_ctx* ctx, sr_batch* batch, sr_stats* out);

void sr_free_batch(sr_ctx* ctx, sr_batch* batch);
const char* sr_last_error(sr_ctx* ctx);

/* ---------------------------------------------------------------- no-allocation entry point
 * The paper has no counterpart to this call: it serves callers that cannot allocate
 * device memory - frameworks that own every byte of the GPU through their own allocator
 * (a second allocator would fight theirs for memory), or processes that forbid cudaMalloc
 * after start-up (allocation can synchronise the device and stall other work).  It is
 * not for use while a CUDA graph is being captured: it copies from pageable host staging
 * memory and synchronises the stream, so on a capturing stream it returns SR_E_INVAL at once and
 * leaves the capture untouched.  It runs the whole check of one program (the same kernels
 * as load_programs + run_and_check + fetch_reports, plain mode, default options) and
 * allocates nothing: every intermediate buffer lives in one file-scope __device__ array
 * of SR_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the process
 * exits.
 *   prog       host descriptors of the program (prog->global_init is not read);
 *   d_arena    device memory, prog->global_words int32: the initial arena in, the final
 *              arena out (updated in place);
 *   d_reports  device memory for report_cap records: the sorted reports (at most report_cap);
 *   n_reports  host: total number of reports;  status: host, SR_ST_* bits of the program.
 * Synchronous on `stream`.  The host side keeps its staging arrays in thread-local storage
 * (about 150 KB per calling thread, allocated once by the C++ runtime, not per call).
 * Returns SR_E_RANGE when the program needs more scratch than
 * the array holds (more than 256 launches, or logs that do not fit even one launch at a
 * time) or when report_cap < *n_reports (extra reports dropped), SR_E_INVAL for an
 * invalid program or a stream that is being captured, SR_E_CUDA for a failed CUDA call.
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress and sets the kernels' shared-memory attributes (once per device,
 * also when several host threads make their first call at the same time).  All calls
 * share the one array and it keeps the last call's contents: calls that overlap on the GPU
 * (other streams, other host threads) race and corrupt each other's results.  The race
 * check runs on min(SMs, 8) CTAs here (each holds 256 KB of the array as staging), fewer
 * than the allocating path uses on a large GPU: results are the same, large programs are
 * checked more slowly. */
#define SR_NOALLOC_SCRATCH_BYTES (32u << 20)
int sr_check_program_noalloc(const sr_program* prog, int32_t* d_arena, sr_report* d_reports, uint64_t report_cap,
                             uint64_t* n_reports, uint32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif
