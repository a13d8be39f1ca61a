/*
 * simt_oracle.h - CPU oracle for the SIMT race/barrier checker.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code: it exists so that tests, the smoke check and the benchmark's CPU
 * baseline can compare the CUDA library against a plain, slow, obviously correct
 * restatement of the method.  It shares no header, constant table or helper with
 * the CUDA sources; the instruction encoding below is re-declared here on purpose.
 *
 * What it computes (paper: Hathhorn, Becchi, Harrison, Procter, "Formal Semantics of
 * Heterogeneous CUDA-C", SSV 2012):
 *   - execution of every thread of every block of every kernel launch of a program,
 *     launches in order over one global arena with the implicit grid-wide sync at the
 *     end of each kernel call (Sec. 2; Sec. 3 "Threads and memory");
 *   - per-block dynamic shared memory sized by the launch (Sec. 3 "Threads and memory");
 *   - __syncthreads() as a block-wide barrier (Sec. 3 "Barrier synchronization");
 *   - race detection: two distinct threads touch the same shared location with no
 *     barrier in between and at least one access writes; the access history is
 *     cleared at every barrier (Sec. 3.1, first paragraph);
 *   - deadlock detection: some thread of a block waits at a barrier that another
 *     thread of the block never reaches (Sec. 3.1, last paragraph).
 *
 * Readings where the paper is silent (each one is also listed in the design notes):
 *   - schedule: round-lockstep with warps of 32 consecutive tids and min-pc
 *     reconvergence; within a round all loads read the pre-round state, then stores
 *     apply in ascending tid order, then atomic adds;
 *   - arithmetic: int32 two's-complement wrap; DIV/REM truncate toward zero; x/0 and
 *     x%0 give 0 plus an ERR_DIV0 record; INT_MIN/-1 = INT_MIN, INT_MIN%-1 = 0; shift
 *     counts masked with 31, SHR arithmetic;
 *   - out-of-range shared/global accesses are suppressed (loads give 0) and recorded;
 *   - atomic-atomic pairs are not races;
 *   - global memory (optional, check_global): the same pair rule inside a block's barrier
 *     interval; any two blocks of one launch touching a word, one writing (blocks of a launch
 *     have no synchronisation point, Sec. 2); any two launches that no stream order or event
 *     wait orders touching a word, one writing (Sec. 3, streams and events);
 *   - a barrier whose waiting threads sit at different barrier instructions is
 *     reported as DIVERGENCE and then released; waiting plus exited threads is a
 *     DEADLOCK: the block stops and the program's later launches are skipped;
 *   - shared memory starts zeroed; running past the last instruction is an EXIT.
 */
#ifndef SIMT_ORACLE_H
#define SIMT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* instruction encoding (re-declared; see module docstring of the IR assembler) */
enum {
  ORC_MOV = 1, ORC_ADD, ORC_SUB, ORC_MUL, ORC_DIV, ORC_REM, ORC_AND, ORC_OR, ORC_XOR,
  ORC_SHL, ORC_SHR, ORC_MIN, ORC_MAX, ORC_SLT, ORC_SLE, ORC_SEQ, ORC_SNE,
  ORC_S2R, ORC_LDG, ORC_STG, ORC_LDS, ORC_STS, ORC_ATOMS, ORC_BRA, ORC_BRZ, ORC_BRNZ,
  ORC_BAR, ORC_EXIT, ORC_BARAND, ORC_BAROR, ORC_BARPOPC
};
#define ORC_BIMM 0x80u
#define ORC_RZ 0xFFu

/* report kinds (the library's public header defines the same numbers) */
enum {
  ORC_REP_RACE = 1, ORC_REP_DIVERGENCE = 2, ORC_REP_DEADLOCK = 3, ORC_REP_STEP_LIMIT = 4,
  ORC_REP_ERR_OOB_SHARED = 5, ORC_REP_ERR_OOB_GLOBAL = 6, ORC_REP_ERR_DIV0 = 7,
  ORC_REP_ERR_UNINIT_SHARED = 8,
  /* check_global: a = global word; b, c as for RACE (classes WW and WR only) */
  ORC_REP_GLOBAL_RACE = 9,
  /* check_global: block = b1, epoch = 0, a = word, b = b2 (b1 < b2, the smallest pair of
     blocks of the launch that conflict on the word), c = classes << 24 | pc range over every
     access of the launch to the word */
  ORC_REP_GLOBAL_BLOCKS = 10,
  /* check_global: launch = l1, block = 0, epoch = 0, a = word, b = l2 (l1 < l2, the smallest
     unordered pair of launches that conflict on the word), c = classes << 24 over every such
     pair */
  ORC_REP_GLOBAL_LAUNCHES = 11
};
/* race class bits (field c bits 24..27) */
enum { ORC_CLS_WW = 1, ORC_CLS_WR = 2, ORC_CLS_WA = 4, ORC_CLS_AR = 8 };
/* program status bits */
enum { ORC_ST_DEADLOCK = 1, ORC_ST_STEP_LIMIT = 2 };

typedef struct { uint32_t op_d_a_b; int32_t imm; } orc_instr;
/* Sec. 2 and Sec. 3 "Streams and events": launches of one stream run in order; launches of
 * different streams may run in parallel; a launch may also wait for an event recorded after an
 * earlier launch (wait = 1 + that launch's index, 0 = none).  A launch is skipped when the
 * launch before it in its stream, or the one it waits for, stopped or was skipped. */
typedef struct {
  uint32_t kernel, grid, block_dim, shmem_words, nparams;
  int32_t params[4];
  uint32_t stream, wait;
  /* run only blocks [block_begin, block_begin + block_count) of the grid, numbered as in the
     whole grid (count 0 = every block); Sec. 2: blocks of a grid are independent */
  uint32_t block_begin, block_count;
} orc_launch;
typedef struct {
  const orc_instr* code; uint32_t ncode;
  const uint32_t* kernel_entry; uint32_t nkernels;
  const orc_launch* launches; uint32_t nlaunches;
  int32_t* arena; uint64_t arena_words;      /* initial image in, final image out */
} orc_program;
typedef struct { uint32_t kind, prog, launch, block, epoch, a, b, c; } orc_report;

typedef struct {
  uint32_t round_budget;     /* rounds per block before STEP_LIMIT (0 = 1<<24) */
  uint32_t check_races;      /* 0 = skip the race check (plain interpreter) */
  uint32_t schedule;         /* 0 = round-lockstep (canonical), 1 = thread-sequential */
  uint32_t nthreads;         /* host threads over blocks of one launch (0/1 = serial) */
  uint32_t check_interblock; /* 1 = count global words that two blocks of one launch touch, one
                                writing (diagnostic; serial and threaded modes) */
  uint32_t max_blocks;       /* >0: run only blocks [0, max_blocks) of each launch (timing samples) */
  uint32_t check_uninit;     /* 1 = report shared loads of words no thread of the block wrote */
  uint32_t check_streams;    /* 1 = count global words that two launches no stream or event orders
                                both touch, one writing (serial mode only) */
  uint32_t check_global;     /* 1 = report global-memory races (kinds 9, 10, 11) */
} orc_opts;

typedef struct {
  orc_report* reports; uint64_t nreports;    /* sorted canonically; free with orc_free */
  uint32_t* status;                          /* per program */
  uint64_t thread_instrs;                    /* lane-instructions executed */
  uint64_t shared_accesses;                  /* shared accesses seen by the race check */
  uint64_t rounds;                           /* rounds executed, all blocks */
  uint64_t interblock_conflicts;             /* diagnostic (check_interblock): words, summed
                                                over launches */
  uint64_t stream_conflicts;                 /* diagnostic (check_streams) */
} orc_result;

/* returns 0, or a negative code for an invalid program (nothing is run) */
int orc_run(const orc_program* progs, uint32_t nprogs, const orc_opts* opts, orc_result* res);
void orc_free(orc_result* res);
const char* orc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
