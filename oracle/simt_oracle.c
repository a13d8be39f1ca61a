/*
 * simt_oracle.c - plain CPU oracle for the SIMT race/barrier checker.
 *
 * TEST INFRASTRUCTURE ONLY (see simt_oracle.h): used by tests, the smoke check and
 * the benchmark's CPU baseline; never by the product path.
 *
 * Structure mirrors the definitions, not any GPU design:
 *   run_program      - launches in order over one arena (Sec. 2: implicit sync at the
 *                      end of each kernel call; Fig. 1 lines 33-34)
 *   run_block        - one thread block: rounds, barrier resolution, step budget
 *   exec_one         - one instruction of one thread
 *   finish_epoch     - race check of the accesses since the last barrier (Sec. 3.1:
 *                      pairwise definition; the history is cleared at the barrier), of
 *                      shared words and, with check_global, of global words
 *   block_races      - with check_global: pairs of blocks of one launch that touch a
 *                      global word, one writing (no barrier orders blocks, Sec. 2)
 *   launch_races     - with check_global: pairs of launches that no stream order or event
 *                      wait orders and that touch a global word, one writing (Sec. 3,
 *                      streams and events)
 *   resolve          - barrier check at the point where no thread can run
 *                      (Sec. 3 "Barrier synchronization"; Sec. 3.1 deadlock paragraph),
 *                      and the results of __syncthreads_and/_or/_count at a release
 */
#include "simt_oracle.h"

#include <pthread.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_CODE 4096u
#define ORC_MAX_BDIM 1024u
#define ORC_MAX_SHMEM 12288u
#define ORC_DEFAULT_BUDGET (1u << 24)

enum { ST_RUN = 0, ST_WAIT = 1, ST_EXIT = 2 };
enum { K_R = 0, K_W = 1, K_A = 2 };

static char g_err[256];
const char* orc_last_error(void) { return g_err; }

/* ------------------------------------------------------------ growable arrays */
typedef struct { orc_report* v; uint64_t n, cap; } rep_vec;
typedef struct { uint32_t addr, tid, kind, pc; } access_t;
typedef struct { access_t* v; uint64_t n, cap; } acc_vec;
typedef struct { uint32_t addr, block, kind, pc; } gaccess_t;   /* a global access of a launch */
typedef struct { gaccess_t* v; uint64_t n, cap; } gacc_vec;
typedef struct { int32_t addr, val; } store_t;
typedef struct { store_t* v; uint64_t n, cap; } st_vec;

static void* xrealloc(void* p, size_t bytes) {
  void* q = realloc(p, bytes ? bytes : 1);
  if (!q) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
  return q;
}
static void rep_push(rep_vec* r, orc_report x) {
  if (r->n == r->cap) { r->cap = r->cap ? 2 * r->cap : 64; r->v = xrealloc(r->v, r->cap * sizeof(*r->v)); }
  r->v[r->n++] = x;
}
static void acc_push(acc_vec* r, access_t x) {
  if (r->n == r->cap) { r->cap = r->cap ? 2 * r->cap : 256; r->v = xrealloc(r->v, r->cap * sizeof(*r->v)); }
  r->v[r->n++] = x;
}
static void gacc_push(gacc_vec* r, gaccess_t x) {
  if (r->n == r->cap) { r->cap = r->cap ? 2 * r->cap : 256; r->v = xrealloc(r->v, r->cap * sizeof(*r->v)); }
  r->v[r->n++] = x;
}
static void st_push(st_vec* r, int32_t addr, int32_t val) {
  if (r->n == r->cap) { r->cap = r->cap ? 2 * r->cap : 256; r->v = xrealloc(r->v, r->cap * sizeof(*r->v)); }
  r->v[r->n].addr = addr; r->v[r->n].val = val; r->n++;
}

/* int32 two's-complement helpers (conversions written out, no signed overflow) */
static int32_t as_i32(uint32_t x) { return (x & 0x80000000u) ? -(int32_t)(~x) - 1 : (int32_t)x; }
static int32_t add32(int32_t a, int32_t b) { return as_i32((uint32_t)a + (uint32_t)b); }
static int32_t sub32(int32_t a, int32_t b) { return as_i32((uint32_t)a - (uint32_t)b); }
static int32_t mul32(int32_t a, int32_t b) { return as_i32((uint32_t)a * (uint32_t)b); }

/* ------------------------------------------------------------ one block */
typedef struct {
  const orc_program* P;
  uint32_t prog_idx, launch_idx;
  const orc_launch* L;
  const orc_opts* O;
  uint32_t budget;
  /* outputs (private to the host thread running the block) */
  rep_vec* reps;
  uint64_t thread_instrs, shared_accesses, rounds;
  uint32_t status;               /* ORC_ST_* seen in this launch */
  /* check_interblock: per global word of the launch, the block that wrote it and the block
     that read it (-1 none, -2 two or more distinct blocks); shared by the host threads of a
     launch and updated with atomic compare-and-swap, so the result is order-independent */
  int32_t* writer; int32_t* reader;
  /* check_streams: per global word of this launch, 1 = read, 2 = written (serial mode only) */
  uint8_t* acc;
  /* check_global: the global accesses of this host thread's blocks of the launch */
  gacc_vec* lacc;
} launch_ctx;

typedef struct {
  launch_ctx* C;
  uint32_t block, n, nwarps, shw;
  uint32_t* pc; uint8_t* st; uint32_t* wpc;
  uint8_t* bk; uint8_t* bp; uint8_t* bd;   /* waiting thread: barrier kind (0 plain, 1 and,
                                              2 or, 3 count), its predicate, destination */
  int32_t* regs;                 /* [n][16] */
  int32_t* sh;                   /* shared array of this block */
  uint32_t* err_cnt; uint32_t* err_min;   /* per pc, current epoch */
  uint8_t err_any;
  uint8_t* written;              /* shared words some thread of the block stored or added to */
  uint32_t* un_cnt; uint32_t* un_min;     /* loads of unwritten words, per pc, current epoch */
  acc_vec acc;                   /* shared accesses of the current epoch */
  acc_vec gacc;                  /* global accesses of the current epoch (check_global) */
  st_vec sst, gst, ats;          /* deferred shared stores, global stores, atomics (round) */
  uint32_t epoch;
  int deferred;                  /* 1 = lockstep rounds, 0 = immediate (sequential) */
} block_t;

static int32_t reg_read(block_t* B, uint32_t t, uint32_t r) {
  return r == ORC_RZ ? 0 : B->regs[t * 16 + r];
}
static void reg_write(block_t* B, uint32_t t, uint32_t r, int32_t v) {
  if (r != ORC_RZ) B->regs[t * 16 + r] = v;
}
static void note_err(block_t* B, uint32_t pc, uint32_t t) {
  B->err_cnt[pc]++;
  if (t < B->err_min[pc]) B->err_min[pc] = t;
  B->err_any = 1;
}
static void note_uninit(block_t* B, uint32_t pc, uint32_t t) {
  B->un_cnt[pc]++;
  if (t < B->un_min[pc]) B->un_min[pc] = t;
  B->err_any = 1;
}
/* one block's mark on a word: -1 (nobody) becomes the block; a second, different block
   makes it -2 (two or more); compare-and-swap so that host threads may share the array */
static void mark_block(int32_t* slot, int32_t me) {
  int32_t cur = __atomic_load_n(slot, __ATOMIC_RELAXED);
  for (;;) {
    if (cur == me || cur == -2) return;
    int32_t want = cur == -1 ? me : -2;
    if (__atomic_compare_exchange_n(slot, &cur, want, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) return;
  }
}
static void note_global(block_t* B, int32_t addr, uint32_t t, uint32_t pc, int is_write) {
  launch_ctx* C = B->C;
  if (C->acc) C->acc[addr] |= is_write ? 2u : 1u;
  if (C->writer) mark_block(is_write ? &C->writer[addr] : &C->reader[addr], (int32_t)B->block);
  if (C->lacc) {
    acc_push(&B->gacc, (access_t){(uint32_t)addr, t, is_write ? K_W : K_R, pc});
    gacc_push(C->lacc, (gaccess_t){(uint32_t)addr, B->block, is_write ? K_W : K_R, pc});
  }
}

static int32_t alu(block_t* B, uint32_t op, int32_t va, int32_t vb, uint32_t pc, uint32_t t) {
  switch (op) {
    case ORC_MOV: return vb;
    case ORC_ADD: return add32(va, vb);
    case ORC_SUB: return sub32(va, vb);
    case ORC_MUL: return mul32(va, vb);
    case ORC_DIV:
      if (vb == 0) { note_err(B, pc, t); return 0; }
      if (va == INT32_MIN && vb == -1) return INT32_MIN;
      return va / vb;                          /* C99: truncation toward zero */
    case ORC_REM:
      if (vb == 0) { note_err(B, pc, t); return 0; }
      if (va == INT32_MIN && vb == -1) return 0;
      return va % vb;                          /* sign follows the dividend */
    case ORC_AND: return va & vb;
    case ORC_OR:  return va | vb;
    case ORC_XOR: return va ^ vb;
    case ORC_SHL: return as_i32((uint32_t)va << ((uint32_t)vb & 31u));
    case ORC_SHR: {
      uint32_t s = (uint32_t)vb & 31u;
      return va < 0 ? ~((~va) >> s) : (va >> s);   /* arithmetic shift written out */
    }
    case ORC_MIN: return va < vb ? va : vb;
    case ORC_MAX: return va > vb ? va : vb;
    case ORC_SLT: return va < vb;
    case ORC_SLE: return va <= vb;
    case ORC_SEQ: return va == vb;
    case ORC_SNE: return va != vb;
  }
  return 0;
}

/* which operand fields an opcode reads (unused fields are never decoded) */
static int is_rbar(uint32_t b) { return b == ORC_BARAND || b == ORC_BAROR || b == ORC_BARPOPC; }
static int uses_d(uint32_t b) {
  return (b >= ORC_MOV && b <= ORC_SNE) || b == ORC_S2R || b == ORC_LDG || b == ORC_LDS || is_rbar(b);
}
static int uses_a(uint32_t b) {
  return (b >= ORC_ADD && b <= ORC_SNE) || b == ORC_LDG || b == ORC_STG || b == ORC_LDS ||
         b == ORC_STS || b == ORC_ATOMS || b == ORC_BRZ || b == ORC_BRNZ || is_rbar(b);
}
static int uses_b(uint32_t op) {
  uint32_t b = op & 0x7Fu;
  return ((b >= ORC_MOV && b <= ORC_SNE) && !(op & ORC_BIMM)) || b == ORC_STG || b == ORC_STS || b == ORC_ATOMS;
}

/* execute the instruction at pc for thread t (pc == ncode is the implicit EXIT) */
static void exec_one(block_t* B, uint32_t t, uint32_t pc) {
  const orc_program* P = B->C->P;
  const orc_launch* L = B->C->L;
  B->C->thread_instrs++;
  if (pc >= P->ncode) { B->st[t] = ST_EXIT; return; }
  uint32_t w = P->code[pc].op_d_a_b;
  int32_t imm = P->code[pc].imm;
  uint32_t op = w & 0xFFu, base = op & 0x7Fu;
  uint32_t d = (w >> 8) & 0xFFu, a = (w >> 16) & 0xFFu, b = (w >> 24) & 0xFFu;
  int32_t va = uses_a(base) ? reg_read(B, t, a) : 0;
  int32_t vb = (op & ORC_BIMM) ? imm : (uses_b(op) ? reg_read(B, t, b) : 0);
  uint32_t next = pc + 1;

  if (base >= ORC_MOV && base <= ORC_SNE) {
    reg_write(B, t, d, alu(B, base, va, vb, pc, t));
  } else switch (base) {
    case ORC_S2R: {
      int32_t v = 0;
      switch (imm) {
        case 0: v = (int32_t)t; break;
        case 1: v = (int32_t)B->block; break;
        case 2: v = (int32_t)L->block_dim; break;
        case 3: v = (int32_t)L->grid; break;
        case 4: v = 32; break;
      }
      reg_write(B, t, d, v);
      break;
    }
    case ORC_LDS: {
      int32_t addr = add32(va, imm), v = 0;
      if (addr < 0 || (uint32_t)addr >= B->shw) note_err(B, pc, t);
      else {
        v = B->sh[addr];                   /* deferred writes: pre-round value */
        acc_push(&B->acc, (access_t){(uint32_t)addr, t, K_R, pc});
        if (B->C->O->check_uninit && !B->written[addr]) note_uninit(B, pc, t);
      }
      reg_write(B, t, d, v);
      break;
    }
    case ORC_STS: case ORC_ATOMS: {
      int32_t addr = add32(va, imm);
      if (addr < 0 || (uint32_t)addr >= B->shw) { note_err(B, pc, t); break; }
      acc_push(&B->acc, (access_t){(uint32_t)addr, t, base == ORC_STS ? K_W : K_A, pc});
      if (base == ORC_STS) {
        if (B->deferred) st_push(&B->sst, addr, vb); else B->sh[addr] = vb;
      } else {
        if (B->deferred) st_push(&B->ats, addr, vb); else B->sh[addr] = add32(B->sh[addr], vb);
      }
      if (!B->deferred) B->written[addr] = 1;   /* in rounds: when the round's writes apply */
      break;
    }
    case ORC_LDG: {
      int32_t addr = add32(va, imm), v = 0;
      if (addr < 0 || (uint64_t)addr >= P->arena_words) note_err(B, pc, t);
      else { v = P->arena[addr]; note_global(B, addr, t, pc, 0); }
      reg_write(B, t, d, v);
      break;
    }
    case ORC_STG: {
      int32_t addr = add32(va, imm);
      if (addr < 0 || (uint64_t)addr >= P->arena_words) { note_err(B, pc, t); break; }
      note_global(B, addr, t, pc, 1);
      if (B->deferred) st_push(&B->gst, addr, vb); else P->arena[addr] = vb;
      break;
    }
    case ORC_BRA: next = (uint32_t)imm; break;
    case ORC_BRZ: if (va == 0) next = (uint32_t)imm; break;
    case ORC_BRNZ: if (va != 0) next = (uint32_t)imm; break;
    case ORC_BAR: case ORC_BARAND: case ORC_BAROR: case ORC_BARPOPC:
      /* __syncthreads and its reducing forms (Sec. 3 feature list): wait here; a
         reducing form also hands in its predicate and names where the result goes */
      B->st[t] = ST_WAIT; B->wpc[t] = pc;
      B->bk[t] = (uint8_t)(base == ORC_BAR ? 0 : base - ORC_BARAND + 1);
      B->bp[t] = base != ORC_BAR && va != 0;
      B->bd[t] = (uint8_t)d;
      break;
    case ORC_EXIT: B->st[t] = ST_EXIT; break;
  }
  B->pc[t] = next;
}

/* one lockstep round: every warp with a runnable thread issues its lowest pc */
static void exec_round(block_t* B) {
  B->sst.n = B->gst.n = B->ats.n = 0;
  for (uint32_t w = 0; w < B->nwarps; ++w) {
    uint32_t lo = 32 * w, hi = lo + 32 < B->n ? lo + 32 : B->n;
    uint32_t p = UINT32_MAX;
    for (uint32_t t = lo; t < hi; ++t)
      if (B->st[t] == ST_RUN && B->pc[t] < p) p = B->pc[t];
    if (p == UINT32_MAX) continue;
    for (uint32_t t = lo; t < hi; ++t)
      if (B->st[t] == ST_RUN && B->pc[t] == p) exec_one(B, t, p);
  }
  /* stores in ascending tid order (the lists were filled in that order), then atomics */
  for (uint64_t i = 0; i < B->sst.n; ++i) B->sh[B->sst.v[i].addr] = B->sst.v[i].val;
  for (uint64_t i = 0; i < B->gst.n; ++i) B->C->P->arena[B->gst.v[i].addr] = B->gst.v[i].val;
  for (uint64_t i = 0; i < B->ats.n; ++i)
    B->sh[B->ats.v[i].addr] = add32(B->sh[B->ats.v[i].addr], B->ats.v[i].val);
  /* the words this round stored to or added to count as written from the next round on */
  for (uint64_t i = 0; i < B->sst.n; ++i) B->written[B->sst.v[i].addr] = 1;
  for (uint64_t i = 0; i < B->ats.n; ++i) B->written[B->ats.v[i].addr] = 1;
}

static int cmp_access(const void* x, const void* y) {
  const access_t* p = x; const access_t* q = y;
  if (p->addr != q->addr) return p->addr < q->addr ? -1 : 1;
  if (p->tid != q->tid) return p->tid < q->tid ? -1 : 1;
  if (p->kind != q->kind) return p->kind < q->kind ? -1 : 1;
  if (p->pc != q->pc) return p->pc < q->pc ? -1 : 1;
  return 0;
}

static void emit(block_t* B, uint32_t kind, uint32_t a, uint32_t b, uint32_t c) {
  orc_report r = {kind, B->C->prog_idx, B->C->launch_idx, B->block, B->epoch, a, b, c};
  rep_push(B->C->reps, r);
}

/* the conflict class of two accesses by different threads (Sec. 3.1: at least one writes;
   reading: atomic adds commute with each other but not with reads or writes); 0 = none */
static uint32_t conflict_class(uint32_t k1, uint32_t k2) {
  if (k1 == K_W && k2 == K_W) return ORC_CLS_WW;
  if ((k1 == K_W && k2 == K_R) || (k1 == K_R && k2 == K_W)) return ORC_CLS_WR;
  if ((k1 == K_W && k2 == K_A) || (k1 == K_A && k2 == K_W)) return ORC_CLS_WA;
  if ((k1 == K_A && k2 == K_R) || (k1 == K_R && k2 == K_A)) return ORC_CLS_AR;
  return 0;                                     /* read-read, atomic-atomic */
}

/* race check of one interval's accesses to one memory: every pair of accesses to a word
   by distinct threads, one writing (Sec. 3.1); one record of kind `kind` per racy word */
static void interval_races(block_t* B, acc_vec* acc, uint32_t kind) {
  qsort(acc->v, acc->n, sizeof(access_t), cmp_access);
  uint64_t i = 0;
  while (i < acc->n) {
    uint64_t j = i;
    while (j < acc->n && acc->v[j].addr == acc->v[i].addr) ++j;
    uint32_t cls = 0, t1 = UINT32_MAX, t2 = UINT32_MAX, pclo = UINT32_MAX, pchi = 0;
    for (uint64_t x = i; x < j; ++x) {
      const access_t* p = &acc->v[x];
      if (p->pc < pclo) pclo = p->pc;
      if (p->pc > pchi) pchi = p->pc;
      for (uint64_t y = x + 1; y < j; ++y) {
        const access_t* q = &acc->v[y];
        if (p->tid == q->tid) continue;
        uint32_t bit = conflict_class(p->kind, q->kind);
        if (!bit) continue;
        cls |= bit;
        uint32_t lo = p->tid < q->tid ? p->tid : q->tid, hi = p->tid ^ q->tid ^ lo;
        if (lo < t1 || (lo == t1 && hi < t2)) { t1 = lo; t2 = hi; }
      }
    }
    if (cls) emit(B, kind, acc->v[i].addr, (t1 << 16) | t2, (cls << 24) | (pclo << 12) | pchi);
    i = j;
  }
}

/* race check of one barrier interval: the pairwise definition of Sec. 3.1 on shared words
 * (and, with check_global, on global words), then error records of the interval; the
 * access history is then cleared */
static void finish_epoch(block_t* B) {
  const orc_program* P = B->C->P;
  B->C->shared_accesses += B->acc.n;
  if (B->C->O->check_races && B->acc.n) interval_races(B, &B->acc, ORC_REP_RACE);
  B->acc.n = 0;
  if (B->gacc.n) interval_races(B, &B->gacc, ORC_REP_GLOBAL_RACE);
  B->gacc.n = 0;
  if (B->err_any) {
    for (uint32_t pc = 0; pc < P->ncode; ++pc) {
      if (!B->err_cnt[pc]) continue;
      uint32_t base = P->code[pc].op_d_a_b & 0x7Fu, kind;
      if (base == ORC_LDS || base == ORC_STS || base == ORC_ATOMS) kind = ORC_REP_ERR_OOB_SHARED;
      else if (base == ORC_LDG || base == ORC_STG) kind = ORC_REP_ERR_OOB_GLOBAL;
      else kind = ORC_REP_ERR_DIV0;
      emit(B, kind, pc, B->err_min[pc], B->err_cnt[pc]);
      B->err_cnt[pc] = 0; B->err_min[pc] = UINT32_MAX;
    }
    for (uint32_t pc = 0; pc < P->ncode; ++pc) {
      if (!B->un_cnt[pc]) continue;
      emit(B, ORC_REP_ERR_UNINIT_SHARED, pc, B->un_min[pc], B->un_cnt[pc]);
      B->un_cnt[pc] = 0; B->un_min[pc] = UINT32_MAX;
    }
    B->err_any = 0;
  }
}

/* returns 1 when the block is finished (done, deadlocked or out of budget) */
static int resolve(block_t* B) {
  uint32_t nW = 0, nX = 0, pmin = UINT32_MAX, pmax = 0;
  for (uint32_t t = 0; t < B->n; ++t) {
    if (B->st[t] == ST_WAIT) {
      ++nW;
      if (B->wpc[t] < pmin) pmin = B->wpc[t];
      if (B->wpc[t] > pmax) pmax = B->wpc[t];
    } else if (B->st[t] == ST_EXIT) ++nX;
  }
  if (nW == 0) { finish_epoch(B); return 1; }
  if (nX > 0) {            /* some thread will never reach the barrier the others wait at */
    emit(B, ORC_REP_DEADLOCK, pmin, pmax, (nW << 16) | nX);
    finish_epoch(B);
    B->C->status |= ORC_ST_DEADLOCK;
    return 1;
  }
  if (pmin != pmax)        /* all threads wait, but not at the same barrier instruction */
    emit(B, ORC_REP_DIVERGENCE, pmin, pmax, nW << 16);
  finish_epoch(B);
  B->epoch++;
  /* release: the reducing barriers' results, over every released thread's predicate
     (a thread released from a plain barrier contributes a false one) */
  uint32_t nP = 0;
  for (uint32_t t = 0; t < B->n; ++t) if (B->st[t] == ST_WAIT && B->bp[t]) ++nP;
  for (uint32_t t = 0; t < B->n; ++t) {
    if (B->st[t] != ST_WAIT) continue;
    if (B->bk[t] == 1) reg_write(B, t, B->bd[t], nP == nW);
    else if (B->bk[t] == 2) reg_write(B, t, B->bd[t], nP > 0);
    else if (B->bk[t] == 3) reg_write(B, t, B->bd[t], (int32_t)nP);
    B->st[t] = ST_RUN;
  }
  return 0;
}

static void run_block(launch_ctx* C, uint32_t block) {
  const orc_program* P = C->P;
  const orc_launch* L = C->L;
  block_t B;
  memset(&B, 0, sizeof(B));
  B.C = C; B.block = block; B.n = L->block_dim; B.nwarps = (L->block_dim + 31) / 32;
  B.shw = L->shmem_words;
  B.deferred = C->O->schedule == 0;
  B.pc = malloc(B.n * sizeof(uint32_t)); B.st = malloc(B.n); B.wpc = malloc(B.n * sizeof(uint32_t));
  B.bk = calloc(B.n, 1); B.bp = calloc(B.n, 1); B.bd = calloc(B.n, 1);
  B.regs = calloc((size_t)B.n * 16, sizeof(int32_t));
  B.sh = calloc(B.shw ? B.shw : 1, sizeof(int32_t));          /* shared memory starts at zero */
  B.err_cnt = calloc(P->ncode + 1, sizeof(uint32_t));
  B.err_min = malloc((P->ncode + 1) * sizeof(uint32_t));
  B.un_cnt = calloc(P->ncode + 1, sizeof(uint32_t));
  B.un_min = malloc((P->ncode + 1) * sizeof(uint32_t));
  for (uint32_t i = 0; i <= P->ncode; ++i) B.err_min[i] = B.un_min[i] = UINT32_MAX;
  B.written = calloc(B.shw ? B.shw : 1, 1);
  uint32_t entry = P->kernel_entry[L->kernel];
  for (uint32_t t = 0; t < B.n; ++t) {
    B.pc[t] = entry; B.st[t] = ST_RUN;
    for (uint32_t r = 0; r < L->nparams; ++r) B.regs[t * 16 + r] = L->params[r];
  }
  uint64_t rounds = 0;
  for (;;) {
    uint32_t nrun = 0, runpc = UINT32_MAX;
    for (uint32_t t = 0; t < B.n; ++t)
      if (B.st[t] == ST_RUN) { ++nrun; if (B.pc[t] < runpc) runpc = B.pc[t]; }
    if (nrun == 0) {
      if (resolve(&B)) break;
      continue;
    }
    if (rounds >= C->budget) {
      emit(&B, ORC_REP_STEP_LIMIT, (uint32_t)rounds, nrun, runpc);
      finish_epoch(&B);
      C->status |= ORC_ST_STEP_LIMIT;
      break;
    }
    if (B.deferred) {
      exec_round(&B);
      ++rounds;
    } else {
      /* thread-sequential: each thread alone until it waits or exits */
      for (uint32_t t = 0; t < B.n && rounds < C->budget; ++t)
        while (B.st[t] == ST_RUN && rounds < C->budget) { exec_one(&B, t, B.pc[t]); ++rounds; }
    }
  }
  C->rounds += rounds;
  free(B.pc); free(B.st); free(B.wpc); free(B.bk); free(B.bp); free(B.bd); free(B.regs); free(B.sh);
  free(B.err_cnt); free(B.err_min); free(B.un_cnt); free(B.un_min); free(B.written); free(B.acc.v); free(B.gacc.v);
  free(B.sst.v); free(B.gst.v); free(B.ats.v);
}

/* ------------------------------------------------------------ validation */
static int validate(const orc_program* P, uint32_t idx) {
  if (!P->code || P->ncode == 0 || P->ncode > ORC_MAX_CODE) {
    snprintf(g_err, sizeof g_err, "program %u: code size %u outside 1..%u", idx, P->ncode, ORC_MAX_CODE); return -1; }
  if (P->nkernels == 0 || !P->kernel_entry) { snprintf(g_err, sizeof g_err, "program %u: no kernels", idx); return -1; }
  for (uint32_t k = 0; k < P->nkernels; ++k)
    if (P->kernel_entry[k] >= P->ncode) { snprintf(g_err, sizeof g_err, "program %u: kernel %u entry out of range", idx, k); return -1; }
  for (uint32_t pc = 0; pc < P->ncode; ++pc) {
    uint32_t w = P->code[pc].op_d_a_b, op = w & 0xFFu, base = op & 0x7Fu;
    uint32_t d = (w >> 8) & 0xFFu, a = (w >> 16) & 0xFFu, b = (w >> 24) & 0xFFu;
    int32_t imm = P->code[pc].imm;
    int alu_op = base >= ORC_MOV && base <= ORC_SNE;
    if (base < ORC_MOV || base > ORC_BARPOPC || (op & 0x40u) || ((op & ORC_BIMM) && !alu_op)) {
      snprintf(g_err, sizeof g_err, "program %u pc %u: bad opcode 0x%x", idx, pc, op); return -1; }
    int need_b = uses_b(op);
    if ((uses_d(base) && d >= 16 && d != ORC_RZ) || (uses_a(base) && a >= 16 && a != ORC_RZ) ||
        (need_b && b >= 16 && b != ORC_RZ)) {
      snprintf(g_err, sizeof g_err, "program %u pc %u: bad register", idx, pc); return -1; }
    if ((base == ORC_BRA || base == ORC_BRZ || base == ORC_BRNZ) && (imm < 0 || (uint32_t)imm > P->ncode)) {
      snprintf(g_err, sizeof g_err, "program %u pc %u: branch target out of range", idx, pc); return -1; }
    if (base == ORC_S2R && (imm < 0 || imm > 4)) {
      snprintf(g_err, sizeof g_err, "program %u pc %u: bad special register", idx, pc); return -1; }
  }
  for (uint32_t l = 0; l < P->nlaunches; ++l) {
    const orc_launch* L = &P->launches[l];
    if (L->kernel >= P->nkernels || L->block_dim == 0 || L->block_dim > ORC_MAX_BDIM || L->grid == 0 ||
        L->shmem_words > ORC_MAX_SHMEM || L->nparams > 4) {
      snprintf(g_err, sizeof g_err, "program %u launch %u: bad configuration", idx, l); return -1; }
    if (L->wait > l) {
      snprintf(g_err, sizeof g_err, "program %u launch %u: waits for a launch that is not earlier", idx, l);
      return -1; }
    if ((L->block_count == 0 && L->block_begin != 0) || (uint64_t)L->block_begin + L->block_count > L->grid) {
      snprintf(g_err, sizeof g_err, "program %u launch %u: block range outside the grid", idx, l); return -1; }
  }
  if (P->arena_words > 0x7FFFFFFFull || (P->arena_words && !P->arena)) {
    snprintf(g_err, sizeof g_err, "program %u: bad arena", idx); return -1; }
  return 0;
}

/* ------------------------------------------------------------ global-memory races */
static int cmp_gaccess(const void* x, const void* y) {
  const gaccess_t* p = x; const gaccess_t* q = y;
  if (p->addr != q->addr) return p->addr < q->addr ? -1 : 1;
  if (p->block != q->block) return p->block < q->block ? -1 : 1;
  if (p->kind != q->kind) return p->kind < q->kind ? -1 : 1;
  if (p->pc != q->pc) return p->pc < q->pc ? -1 : 1;
  return 0;
}

/* Races between the blocks of one launch on global words: blocks of a grid run with no
 * synchronisation point between them (Sec. 2: only the end of the kernel call orders them),
 * so two accesses to a word by different blocks, one writing, race whatever the barrier
 * intervals.  Per word: the classes over all such pairs, the smallest pair of blocks, and
 * the pc range of every access of the launch to the word.  The accesses are sorted by
 * (word, block, kind, pc); repeated (block, kind) entries of a word add nothing to the pairs
 * and are compared once. */
static void block_races(gacc_vec* a, uint32_t prog, uint32_t launch, rep_vec* out) {
  qsort(a->v, a->n, sizeof(gaccess_t), cmp_gaccess);
  gacc_vec u = {0};                             /* the word's distinct (block, kind) entries */
  uint64_t i = 0;
  while (i < a->n) {
    uint64_t j = i;
    uint32_t pclo = UINT32_MAX, pchi = 0;
    u.n = 0;
    while (j < a->n && a->v[j].addr == a->v[i].addr) {
      const gaccess_t* x = &a->v[j];
      if (x->pc < pclo) pclo = x->pc;
      if (x->pc > pchi) pchi = x->pc;
      if (u.n == 0 || u.v[u.n - 1].block != x->block || u.v[u.n - 1].kind != x->kind) gacc_push(&u, *x);
      ++j;
    }
    uint32_t cls = 0, b1 = UINT32_MAX, b2 = UINT32_MAX;
    for (uint64_t x = 0; x < u.n; ++x)
      for (uint64_t y = x + 1; y < u.n; ++y) {
        const gaccess_t* p = &u.v[x]; const gaccess_t* q = &u.v[y];
        if (p->block == q->block) continue;
        uint32_t bit = conflict_class(p->kind, q->kind);
        if (!bit) continue;
        cls |= bit;
        uint32_t lo = p->block < q->block ? p->block : q->block, hi = p->block ^ q->block ^ lo;
        if (lo < b1 || (lo == b1 && hi < b2)) { b1 = lo; b2 = hi; }
      }
    if (cls) {
      orc_report r = {ORC_REP_GLOBAL_BLOCKS, prog, launch, b1, 0, a->v[i].addr, b2, (cls << 24) | (pclo << 12) | pchi};
      rep_push(out, r);
    }
    i = j;
  }
  free(u.v);
}

typedef struct { uint32_t addr, launch, kind; } laccess_t;   /* a launch touched a word */
typedef struct { laccess_t* v; uint64_t n, cap; } lacc_vec;
static void lacc_push(lacc_vec* r, laccess_t x) {
  if (r->n == r->cap) { r->cap = r->cap ? 2 * r->cap : 256; r->v = xrealloc(r->v, r->cap * sizeof(*r->v)); }
  r->v[r->n++] = x;
}
static int cmp_laccess(const void* x, const void* y) {
  const laccess_t* p = x; const laccess_t* q = y;
  if (p->addr != q->addr) return p->addr < q->addr ? -1 : 1;
  if (p->launch != q->launch) return p->launch < q->launch ? -1 : 1;
  if (p->kind != q->kind) return p->kind < q->kind ? -1 : 1;
  return 0;
}

/* before[l * nl + m] = 1 when launch m precedes launch l through a chain of stream order
 * (the previous launch of a stream) and event waits (Sec. 3, streams and events) */
static uint8_t* order_matrix(const int32_t* dep_prev, const int32_t* dep_wait, uint32_t nl) {
  uint8_t* before = calloc((size_t)(nl ? nl : 1) * (nl ? nl : 1), 1);
  for (uint32_t l = 0; l < nl; ++l) {
    int32_t d[2] = {dep_prev[l], dep_wait[l]};
    for (int k = 0; k < 2; ++k) {
      if (d[k] < 0) continue;
      before[(size_t)l * nl + (uint32_t)d[k]] = 1;
      for (uint32_t m = 0; m < nl; ++m)
        if (before[(size_t)(uint32_t)d[k] * nl + m]) before[(size_t)l * nl + m] = 1;
    }
  }
  return before;
}

/* Races between launches of one program on global words: two launches that nothing orders
 * may run at the same time (Sec. 3, streams and events), so a word both touch, one writing,
 * races.  Per word: the classes over all such pairs and the smallest pair (l1 < l2). */
static void launch_races(lacc_vec* a, uint32_t prog, const uint8_t* before, uint32_t nl, rep_vec* out) {
  qsort(a->v, a->n, sizeof(laccess_t), cmp_laccess);
  uint64_t i = 0;
  while (i < a->n) {
    uint64_t j = i;
    uint32_t writes = 0;
    while (j < a->n && a->v[j].addr == a->v[i].addr) writes += a->v[j++].kind == K_W;
    uint32_t cls = 0, l1 = UINT32_MAX, l2 = UINT32_MAX;
    for (uint64_t x = i; x < j && writes; ++x)
      for (uint64_t y = x + 1; y < j; ++y) {
        const laccess_t* p = &a->v[x]; const laccess_t* q = &a->v[y];
        if (p->launch == q->launch) continue;
        uint32_t m = p->launch < q->launch ? p->launch : q->launch, l = p->launch ^ q->launch ^ m;
        if (before[(size_t)l * nl + m]) continue;   /* ordered: m completes before l starts */
        uint32_t bit = conflict_class(p->kind, q->kind);
        if (!bit) continue;
        cls |= bit;
        if (m < l1 || (m == l1 && l < l2)) { l1 = m; l2 = l; }
      }
    if (cls) {
      orc_report r = {ORC_REP_GLOBAL_LAUNCHES, prog, l1, 0, 0, a->v[i].addr, l2, cls << 24};
      rep_push(out, r);
    }
    i = j;
  }
}

/* ------------------------------------------------------------ launches / programs */
typedef struct { launch_ctx* C; uint32_t b0, b1; } worker_arg;
static void* worker(void* p) {
  worker_arg* w = p;
  for (uint32_t b = w->b0; b < w->b1; ++b) run_block(w->C, b);
  return NULL;
}

static int cmp_report(const void* x, const void* y) {
  const uint32_t* p = x; const uint32_t* q = y;
  static const int order[8] = {1, 2, 3, 4, 0, 5, 6, 7};   /* prog, launch, block, epoch, kind, a, b, c */
  for (int i = 0; i < 8; ++i) {
    uint32_t u = p[order[i]], v = q[order[i]];
    if (u != v) return u < v ? -1 : 1;
  }
  return 0;
}

int orc_run(const orc_program* progs, uint32_t nprogs, const orc_opts* opts, orc_result* res) {
  memset(res, 0, sizeof(*res));
  g_err[0] = 0;
  for (uint32_t p = 0; p < nprogs; ++p) if (validate(&progs[p], p)) return -1;
  orc_opts O = *opts;
  uint32_t budget = O.round_budget ? O.round_budget : ORC_DEFAULT_BUDGET;
  uint32_t nth = O.nthreads ? O.nthreads : 1;
  res->status = calloc(nprogs ? nprogs : 1, sizeof(uint32_t));
  rep_vec all = {0};
  for (uint32_t p = 0; p < nprogs; ++p) {
    const orc_program* P = &progs[p];
    int32_t *writer = NULL, *reader = NULL;
    if (O.check_interblock && P->arena_words) {
      writer = malloc(P->arena_words * sizeof(int32_t));
      reader = malloc(P->arena_words * sizeof(int32_t));
    }
    lacc_vec prog_acc = {0};                   /* check_global: (word, launch, kind) */
    const uint32_t nl = P->nlaunches;
    /* the launches each launch follows: the previous one of its stream, the one it waits for */
    int32_t* dep_prev = malloc((nl ? nl : 1) * sizeof(int32_t));
    int32_t* dep_wait = malloc((nl ? nl : 1) * sizeof(int32_t));
    uint8_t* dead = calloc(nl ? nl : 1, 1);   /* stopped (deadlock, step limit) or skipped */
    uint8_t** acc = (O.check_streams && nth == 1 && P->arena_words) ? calloc(nl ? nl : 1, sizeof(uint8_t*)) : NULL;
    for (uint32_t l = 0; l < nl; ++l) {
      dep_prev[l] = -1;
      for (uint32_t m = l; m-- > 0;)
        if (P->launches[m].stream == P->launches[l].stream) { dep_prev[l] = (int32_t)m; break; }
      dep_wait[l] = P->launches[l].wait ? (int32_t)P->launches[l].wait - 1 : -1;
    }
    for (uint32_t l = 0; l < nl; ++l) {
      const orc_launch* L = &P->launches[l];
      if ((dep_prev[l] >= 0 && dead[dep_prev[l]]) || (dep_wait[l] >= 0 && dead[dep_wait[l]])) {
        dead[l] = 1;                                            /* skipped */
        continue;
      }
      /* the blocks run: [b_first, b_first + nblocks) of the grid */
      uint32_t b_first = L->block_count ? L->block_begin : 0;
      uint32_t nblocks = L->block_count ? L->block_count : L->grid;
      if (O.max_blocks && O.max_blocks < nblocks) nblocks = O.max_blocks;
      if (writer) {
        memset(writer, 0xFF, P->arena_words * sizeof(int32_t));
        memset(reader, 0xFF, P->arena_words * sizeof(int32_t));
      }
      uint32_t nw = nth < nblocks ? nth : nblocks;
      launch_ctx* ctx = calloc(nw, sizeof(launch_ctx));
      rep_vec* reps = calloc(nw, sizeof(rep_vec));
      gacc_vec* lacc = O.check_global ? calloc(nw, sizeof(gacc_vec)) : NULL;
      for (uint32_t i = 0; i < nw; ++i) {
        ctx[i].P = P; ctx[i].prog_idx = p; ctx[i].launch_idx = l; ctx[i].L = L; ctx[i].O = &O;
        ctx[i].budget = budget; ctx[i].reps = &reps[i]; ctx[i].writer = writer; ctx[i].reader = reader;
        ctx[i].lacc = lacc ? &lacc[i] : NULL;
      }
      if (acc) ctx[0].acc = acc[l] = calloc(P->arena_words, 1);
      if (nw == 1) {
        for (uint32_t b = 0; b < nblocks; ++b) run_block(&ctx[0], b_first + b);
      } else {
        pthread_t* th = malloc(nw * sizeof(pthread_t));
        worker_arg* wa = malloc(nw * sizeof(worker_arg));
        for (uint32_t i = 0; i < nw; ++i) {
          wa[i].C = &ctx[i];
          wa[i].b0 = b_first + (uint32_t)((uint64_t)nblocks * i / nw);
          wa[i].b1 = b_first + (uint32_t)((uint64_t)nblocks * (i + 1) / nw);
          pthread_create(&th[i], NULL, worker, &wa[i]);
        }
        for (uint32_t i = 0; i < nw; ++i) pthread_join(th[i], NULL);
        free(th); free(wa);
      }
      uint32_t st = 0;
      for (uint32_t i = 0; i < nw; ++i) {
        st |= ctx[i].status;
        res->thread_instrs += ctx[i].thread_instrs;
        res->shared_accesses += ctx[i].shared_accesses;
        res->rounds += ctx[i].rounds;
        for (uint64_t k = 0; k < reps[i].n; ++k) rep_push(&all, reps[i].v[k]);
        free(reps[i].v);
      }
      free(reps); free(ctx);
      if (writer) {
        /* words two blocks of the launch touched, one writing */
        for (uint64_t w = 0; w < P->arena_words; ++w)
          if (writer[w] == -2 || (writer[w] >= 0 && reader[w] != -1 && reader[w] != writer[w]))
            res->interblock_conflicts++;
      }
      if (lacc) {
        gacc_vec la = {0};
        for (uint32_t i = 0; i < nw; ++i) {
          for (uint64_t k = 0; k < lacc[i].n; ++k) gacc_push(&la, lacc[i].v[k]);
          free(lacc[i].v);
        }
        free(lacc);
        block_races(&la, p, l, &all);          /* sorts la by (word, block, kind, pc) */
        for (uint64_t k = 0; k < la.n;) {      /* per word: did the launch read it, write it */
          uint64_t e = k;
          int rd = 0, wr = 0;
          for (; e < la.n && la.v[e].addr == la.v[k].addr; ++e) {
            if (la.v[e].kind == K_W) wr = 1; else rd = 1;
          }
          if (rd) lacc_push(&prog_acc, (laccess_t){la.v[k].addr, l, K_R});
          if (wr) lacc_push(&prog_acc, (laccess_t){la.v[k].addr, l, K_W});
          k = e;
        }
        free(la.v);
      }
      res->status[p] |= st;
      if (st & (ORC_ST_DEADLOCK | ORC_ST_STEP_LIMIT)) dead[l] = 1;   /* launches after it are skipped */
    }
    if (O.check_global) {
      uint8_t* before = order_matrix(dep_prev, dep_wait, nl);
      launch_races(&prog_acc, p, before, nl, &all);
      free(before);
    }
    free(prog_acc.v);
    if (acc) {
      /* pairs of launches that no chain of stream order and event waits orders: any global
         word that both touch, one of them writing, makes the result depend on timing */
      uint8_t* before = order_matrix(dep_prev, dep_wait, nl);   /* before[l*nl+m]: m precedes l */
      for (uint32_t l = 0; l < nl; ++l)
        for (uint32_t m = 0; m < l; ++m) {
          if (before[(size_t)l * nl + m] || !acc[l] || !acc[m]) continue;
          for (uint64_t w = 0; w < P->arena_words; ++w)
            if (((acc[l][w] & 2u) && acc[m][w]) || ((acc[m][w] & 2u) && acc[l][w])) res->stream_conflicts++;
        }
      for (uint32_t l = 0; l < nl; ++l) free(acc[l]);
      free(acc); free(before);
    }
    free(dep_prev); free(dep_wait); free(dead);
    free(writer); free(reader);
  }
  qsort(all.v, all.n, sizeof(orc_report), cmp_report);
  res->reports = all.v;
  res->nreports = all.n;
  return 0;
}

void orc_free(orc_result* res) {
  free(res->reports); free(res->status);
  memset(res, 0, sizeof(*res));
}
