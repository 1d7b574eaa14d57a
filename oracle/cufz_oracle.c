/*
 * cufz oracle: a plain, slow, serial CPU interpreter of access-index programs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code with the device engine (its own decoder, its own hashing, its own
 * classification) and the engine never calls it.
 *
 * What it computes is the plain definition of one checked fuzz execution of
 * a kernel under test:
 *
 *   - Every thread of every block runs, blocks in linear order, threads in
 *     linear order inside a block.  This is the paper's collapsing transform
 *     (Sec. 4.1, Listings 1-2: a block becomes a CPU function, its threads
 *     iterations of a loop); running them one after another is a valid
 *     refinement of the GPU semantics (Sec. 4.1, "Correctness of
 *     Transformation").  Stores are checked but never performed, so there is
 *     no inter-thread data flow and barriers have no effect (Alg. 2,
 *     BarrierElimination).
 *   - The program is run UNPRUNED.
 *   - Every load and store is checked exactly against its buffer's bounds:
 *     byte_off = idx * width, a violation iff byte_off < 0 or
 *     byte_off + width > len (exact base and bounds, the detector the paper
 *     finds complete in Sec. 7.2, "No-Fat can detect all spatial memory
 *     errors").  Global memory buffers and per-block shared buffers are
 *     separate spaces (Sec. 4.1, memory remapping).  Redzones of R bytes
 *     give each violation a class (tripwire adjacency, Sec. 7.2): underflow
 *     redzone, overflow redzone, another allocation of the same space, wild.
 *   - Every branch evaluation (IF, and each loop-head decision) updates an
 *     AFL-style edge counter: e = (loc ^ prev) & 0xFFFF, count[e] += 1,
 *     prev = loc >> 1, with prev = 0 at each thread's start (Sec. 2.1: AFL's
 *     trampolines after branches feed a coverage payload).  Counts are then
 *     bucketed: 0,1,2 stay; 3->4; 4-7->8; 8-15->16; 16-31->32; 32-127->64;
 *     >=128->128.
 *   - LOOP ctr, n, max behaves as C's for (ctr = 0; ctr < trip; ctr++) with
 *     trip = clamp(n, 0, max) taken once at entry: the counter is 0 on
 *     entry, 1 more after each body, and equals trip after the exit.  Each
 *     head decision (ctr < trip) is a branch evaluation.
 *   - A per-thread back-edge budget stands in for the fuzzer's hang timeout
 *     (Sec. 7.1, 10 s per execution): a thread whose back-edge count exceeds
 *     it stops, and the input is flagged BUDGET.
 *   - Launch configurations that CUDA rejects are not run and get status
 *     INVALID_CONFIG (Sec. 2.3.1, cudaErrorInvalidConfiguration); a grid of
 *     zero blocks or threads is such a configuration (Sec. 7.3 reports the
 *     paper's own runtime dividing by a zero task count).
 *
 * Loaded values: a global buffer k of a program with content seed S holds
 * word j = fmix32(S ^ (k * 0x9E3779B9) ^ j) (fmix32: the MurmurHash3 32-bit
 * finalizer, written from its published definition).  A 1-byte load
 * returns byte (off & 3) of word off >> 2, zero-extended, little endian; a
 * 4-byte load the word; 8- and 16-byte loads the first word.  Shared
 * buffers read 0, and a load that violates reads 0.
 *
 * Per-input digest of all executed accesses (the pruning check, Sec. 5.2:
 * all memory accesses are preserved exactly):
 *   H  = block_lin * 0x9E3779B1 + thread_lin + 0x7F4A7C15 (32-bit), then for
 *        each access of the thread, in program order:
 *        H = H * K + idx  (32-bit), K = (site * 0xC2B2AE3D) | 3
 *   D  = sum over the input's test threads of H ^ (H >> 16), mod 2^64
 * idx is the access's int32 index; the site fixes buffer, kind and width.
 * K is odd, so each step is a bijection of H: a thread whose access sequence
 * differs in one index ends with a different H.  K - 1 is twice an odd
 * number, so one access more or fewer changes H unless H * (K - 1) + idx
 * happens to be 0 mod 2^32.  H ^ (H >> 16), a bijection that is not linear,
 * binds each thread's H to the thread before the sum: two threads that trade
 * their access sequences change D.
 * ordinal = the number of checked events (accesses and divisions) the
 * thread executed before this one.
 *
 * Division (the division-by-zero fault of the paper's kernel errors,
 * Sec. 2.3): DIV and REM are signed, truncating toward zero.  A zero divisor
 * is a fault: the result is 0 and the thread records a violation of kind 2
 * (division) at the division's site (the k-th DIV/REM in program order),
 * with class DIV_ZERO, buffer, width, space and byte offset 0.  INT_MIN / -1
 * is INT_MIN and INT_MIN % -1 is 0, without a fault.  A division is not an
 * access: it is not counted in n_accesses and does not enter the digest.
 *
 * Device heap (the temporal errors of Sec. 2.3: use after free, double
 * free, invalid free), per test thread.  HALLOC at allocation site s (the
 * s-th HALLOC) with size n >= 1 makes block s live with n bytes and returns
 * handle s + 1; with n <= 0 it returns 0 (NULL) and changes nothing.
 * HFREE h: h = 0 does nothing; a handle of no block this thread allocated
 * is an invalid free, a freed block a double free (both records of kind 3,
 * space 2, at the free's site); otherwise the block is freed.  HLD / HST at
 * index i of width w through handle h are accesses (counted, in the digest,
 * access sites shared with LD / ST) to heap space 2: a handle of no
 * allocated block is a wild access, a freed block a use after free, and
 * otherwise byte offset i * w is checked against the block's size as for
 * a buffer (redzone classes, no neighbours).  Heap loads read 0.  Every
 * HFREE, like every access and division, is a checked event for ordinals.
 *
 * Performed shared stores and barriers (the input of BarrierElimination,
 * Sec. 5.2, Alg. 2).  Header byte 11 bit 0 marks a program whose stores to
 * shared buffers are performed: each block's shared buffers start as zero
 * bytes; an in-bounds ST writes the value's little-endian bytes (width 1:
 * its low byte; widths 8 and 16: its four bytes, then zero bytes) and an
 * in-bounds LD reads them back (width 1: the byte, zero-extended; wider:
 * the int32 of the first four bytes); out-of-bounds accesses are checked as
 * always and store nothing.  BAR (0x55, top level only) splits the program
 * into phases; a block runs each phase for all of its threads, one thread
 * after another in thread_lin order, before the next phase: the serial
 * program that translation by loop fission gives (Sec. 5.2).  A thread
 * stopped by the budget runs no later phase.  Without the flag BAR does
 * nothing: stores are never performed and shared loads read 0.  Global
 * buffers are never written.
 *
 * first_key = min over violations of
 *   block_lin << 32 | thread_lin << 22 | min(ordinal, 2^22 - 1).
 *
 * The wire formats (program bytes, the 128-byte input record, the 32-byte
 * violation record) are restated here, not included from the engine.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAGIC 0x315A4643u
#define ORC_MAX_OPS 2048
#define ORC_MAX_BUFS 9
#define ORC_MAX_DEPTH 16

enum { ORC_ST_OK = 0, ORC_ST_VIOLATION = 1, ORC_ST_INVALID_CONFIG = 2, ORC_ST_LIMIT = 3 };
enum { ORC_FL_BUDGET = 1, ORC_FL_OVERFLOW = 2, ORC_FL_NEW_COV = 4 };
enum { ORC_CLS_NONE = 0, ORC_CLS_UNDERFLOW_RZ = 1, ORC_CLS_OVERFLOW_RZ = 2,
       ORC_CLS_OTHER_ALLOC = 3, ORC_CLS_WILD = 4, ORC_CLS_DIV_ZERO = 5,
       ORC_CLS_USE_AFTER_FREE = 6, ORC_CLS_DOUBLE_FREE = 7, ORC_CLS_INVALID_FREE = 8 };
enum { ORC_E_FORMAT = -1, ORC_E_OPERAND = -2, ORC_E_STRUCTURE = -3, ORC_E_LOOPCTR = -4,
       ORC_E_SITES = -5, ORC_E_NOMEM = -6 };

enum {
  OP_NOP = 0x00, OP_SREG = 0x01, OP_IMM = 0x02, OP_MOV = 0x03, OP_SEL = 0x04,
  OP_DIV = 0x05, OP_REM = 0x06, OP_HALLOC = 0x07, OP_HFREE = 0x08,
  OP_ADD = 0x10, OP_SUB, OP_MUL, OP_SHL, OP_SHR, OP_SHRU, OP_AND, OP_OR, OP_XOR,
  OP_MIN, OP_MAX, OP_SETLT, OP_SETLE, OP_SETEQ, OP_SETNE, OP_SETLTU,
  OP_LD = 0x40, OP_ST = 0x41, OP_HLD = 0x42, OP_HST = 0x43,
  OP_IF = 0x50, OP_ELSE = 0x51, OP_ENDIF = 0x52, OP_LOOP = 0x53, OP_ENDLOOP = 0x54,
  OP_BAR = 0x55
};
enum { ORC_PF_SHARED_STORES = 1 }; /* header byte 11 */

typedef struct {
  uint32_t program_id, grid[3], block[3];
  int32_t args[4];
  uint32_t pad;
  uint64_t buf_len[9];
  uint64_t user_tag;
} orc_input; /* 128 bytes */

typedef struct {
  uint32_t redzone;      /* R, bytes */
  uint32_t iter_budget;  /* back-edges per thread */
  uint64_t max_threads;  /* inputs with more threads get LIMIT */
} orc_opts;

typedef struct {
  int32_t status;
  uint32_t flags;
  uint64_t n_accesses, n_violations, first_key, digest, n_branch, n_threads;
  uint32_t n_records, n_edges;
  uint64_t n_ops; /* executed value ops, see exec_range */
} orc_result; /* 72 bytes */

typedef struct {
  uint32_t block_lin, thread_lin, ordinal;
  uint16_t site;
  uint8_t buf, kind, width, space, cls, pad0;
  uint32_t pad1;
  int64_t byte_off;
} orc_record; /* 32 bytes */

typedef struct {
  uint8_t opc, dst, a, b;
  int32_t imm;
  int32_t else_pc, end_pc; /* IF: ELSE (or -1) and ENDIF; LOOP: ENDLOOP */
  int32_t site;            /* branch site (IF/LOOP), access site (LD/ST) or
                              division site (DIV/REM) */
} orc_op;

typedef struct {
  int n_ops, n_regs, n_bufs, n_sites, n_access, n_div, n_alloc, n_free;
  uint32_t shared_mask, seed, flags;
  uint16_t loc[256][2];
  orc_op ops[ORC_MAX_OPS];
} orc_prog;

/* ---------------------------------------------------------------- hashing */

static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

uint32_t orc_fmix32(uint32_t h) { return fmix32(h); }

static uint8_t bucket(uint64_t n) {
  if (n == 0) return 0;
  if (n == 1) return 1;
  if (n == 2) return 2;
  if (n == 3) return 4;
  if (n <= 7) return 8;
  if (n <= 15) return 16;
  if (n <= 31) return 32;
  if (n <= 127) return 64;
  return 128;
}

uint8_t orc_bucket(uint64_t n) { return bucket(n); }

/* --------------------------------------------------------------- decoding */

static uint16_t rd16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static int writes_reg(const orc_op* o) {
  switch (o->opc) {
    case OP_SREG: case OP_IMM: case OP_MOV: case OP_SEL: case OP_LD: case OP_LOOP:
    case OP_DIV: case OP_REM: case OP_HALLOC: case OP_HLD: return 1;
    default: return (o->opc >= 0x10 && o->opc <= 0x1F) || (o->opc >= 0x30 && o->opc <= 0x3F);
  }
}

static int valid_width(int32_t w) { return w == 1 || w == 4 || w == 8 || w == 16; }

/* Decodes and validates a program image; returns 0 or a negative ORC_E_*. */
static int decode(const uint8_t* p, size_t n, orc_prog* P) {
  if (n < 32) return ORC_E_FORMAT;
  if (rd32(p) != ORC_MAGIC || rd16(p + 4) != 1) return ORC_E_FORMAT;
  P->n_ops = rd16(p + 6);
  P->n_regs = p[8];
  P->n_bufs = p[9];
  P->n_sites = p[10];
  P->shared_mask = rd16(p + 12);
  P->seed = rd32(p + 16);
  P->flags = p[11];
  if ((P->flags & ~(uint32_t)ORC_PF_SHARED_STORES) || rd16(p + 14) != 0 || rd32(p + 20) ||
      rd32(p + 24) || rd32(p + 28))
    return ORC_E_FORMAT;
  if (P->n_ops < 1 || P->n_ops > ORC_MAX_OPS || P->n_bufs > ORC_MAX_BUFS) return ORC_E_FORMAT;
  if (P->shared_mask >> P->n_bufs) return ORC_E_FORMAT;
  if (n != 32u + 4u * (size_t)P->n_sites + 8u * (size_t)P->n_ops) return ORC_E_FORMAT;
  for (int s = 0; s < P->n_sites; s++) {
    P->loc[s][0] = rd16(p + 32 + 4 * s);
    P->loc[s][1] = rd16(p + 34 + 4 * s);
  }
  const uint8_t* q = p + 32 + 4 * P->n_sites;
  int stack[ORC_MAX_DEPTH];
  int depth = 0, bsite = 0, asite = 0, dsite = 0, hsite = 0, fsite = 0;
  int R = P->n_regs;
  for (int pc = 0; pc < P->n_ops; pc++) {
    orc_op* o = &P->ops[pc];
    o->opc = q[8 * pc];
    o->dst = q[8 * pc + 1];
    o->a = q[8 * pc + 2];
    o->b = q[8 * pc + 3];
    o->imm = (int32_t)rd32(q + 8 * pc + 4);
    o->else_pc = -1;
    o->end_pc = -1;
    o->site = -1;
    int opc = o->opc;
    int ok;
    if (opc >= 0x10 && opc <= 0x1F) {
      ok = o->dst < R && o->a < R && o->b < R && o->imm == 0;
    } else if (opc >= 0x30 && opc <= 0x3F) {
      ok = o->dst < R && o->a < R && o->b == 0;
    } else {
      switch (opc) {
        case OP_NOP: ok = !o->dst && !o->a && !o->b && !o->imm; break;
        case OP_SREG: ok = o->dst < R && !o->a && !o->b && o->imm >= 0 && o->imm <= 15; break;
        case OP_IMM: ok = o->dst < R && !o->a && !o->b; break;
        case OP_MOV: ok = o->dst < R && o->a < R && !o->b && !o->imm; break;
        case OP_SEL: ok = o->dst < R && o->a < R && o->b < R && o->imm >= 0 && o->imm < R; break;
        case OP_DIV:
        case OP_REM:
          ok = o->dst < R && o->a < R && o->b < R && !o->imm;
          if (ok) o->site = dsite++;
          break;
        case OP_HALLOC:
          ok = o->dst < R && o->a < R && !o->b && !o->imm;
          if (ok) o->site = hsite++;
          break;
        case OP_HFREE:
          ok = !o->dst && o->a < R && !o->b && !o->imm;
          if (ok) o->site = fsite++;
          break;
        case OP_HLD:
        case OP_HST:
          ok = o->dst < R && o->a < R && o->b < R && valid_width(o->imm);
          if (ok) o->site = asite++;
          break;
        case OP_LD:
        case OP_ST:
          ok = o->dst < R && o->a < R && o->b < P->n_bufs && valid_width(o->imm);
          if (ok) o->site = asite++;
          break;
        case OP_IF:
          ok = !o->dst && o->a < R && !o->b && !o->imm;
          if (ok) {
            if (depth >= ORC_MAX_DEPTH) return ORC_E_STRUCTURE;
            o->site = bsite++;
            stack[depth++] = pc;
          }
          break;
        case OP_LOOP:
          ok = o->dst < R && o->a < R && !o->b && o->imm >= 0 && o->imm <= 65535;
          if (ok) {
            if (depth >= ORC_MAX_DEPTH) return ORC_E_STRUCTURE;
            o->site = bsite++;
            stack[depth++] = pc;
          }
          break;
        case OP_ELSE:
          ok = !o->dst && !o->a && !o->b && !o->imm;
          if (ok) {
            if (depth == 0) return ORC_E_STRUCTURE;
            orc_op* h = &P->ops[stack[depth - 1]];
            if (h->opc != OP_IF || h->else_pc >= 0) return ORC_E_STRUCTURE;
            h->else_pc = pc;
          }
          break;
        case OP_ENDIF:
          ok = !o->dst && !o->a && !o->b && !o->imm;
          if (ok) {
            if (depth == 0 || P->ops[stack[depth - 1]].opc != OP_IF) return ORC_E_STRUCTURE;
            P->ops[stack[--depth]].end_pc = pc;
          }
          break;
        case OP_ENDLOOP:
          ok = !o->dst && !o->a && !o->b && !o->imm;
          if (ok) {
            if (depth == 0 || P->ops[stack[depth - 1]].opc != OP_LOOP) return ORC_E_STRUCTURE;
            P->ops[stack[--depth]].end_pc = pc;
          }
          break;
        case OP_BAR: /* a block-wide barrier: outside every IF and LOOP */
          ok = !o->dst && !o->a && !o->b && !o->imm;
          if (ok && depth != 0) return ORC_E_STRUCTURE;
          break;
        default: return ORC_E_FORMAT;
      }
    }
    if (!ok) return ORC_E_OPERAND;
  }
  if (depth != 0) return ORC_E_STRUCTURE;
  if (bsite != P->n_sites) return ORC_E_SITES;
  P->n_access = asite;
  P->n_div = dsite;
  P->n_alloc = hsite;
  P->n_free = fsite;
  /* a loop counter is read-only inside its own body */
  for (int pc = 0; pc < P->n_ops; pc++) {
    const orc_op* o = &P->ops[pc];
    if (o->opc != OP_LOOP) continue;
    for (int j = pc + 1; j < o->end_pc; j++)
      if (writes_reg(&P->ops[j]) && P->ops[j].dst == o->dst) return ORC_E_LOOPCTR;
  }
  return 0;
}

void* orc_load(const uint8_t* bytes, size_t n, int* err) {
  orc_prog* P = (orc_prog*)calloc(1, sizeof(orc_prog));
  if (!P) {
    if (err) *err = ORC_E_NOMEM;
    return NULL;
  }
  int e = decode(bytes, n, P);
  if (err) *err = e;
  if (e) {
    free(P);
    return NULL;
  }
  return P;
}

void orc_free(void* h) { free(h); }

int orc_n_access_sites(const void* h) { return ((const orc_prog*)h)->n_access; }

/* ------------------------------------------------------------ interpreter */

/* The shared-buffer bytes one block has written (programs with performed
 * shared stores), keyed by (buffer, byte offset); a byte never written
 * reads 0.  Open addressing; the table doubles at half load. */
typedef struct {
  uint64_t* keys; /* 0 = empty, else ((buffer << 56) | offset) + 1 */
  uint8_t* vals;
  uint64_t cap, used;
} orc_smem;

static uint64_t smem_slot(const orc_smem* m, uint64_t key) {
  uint64_t i = (key * 0x9E3779B97F4A7C15ull) & (m->cap - 1);
  while (m->keys[i] && m->keys[i] != key) i = (i + 1) & (m->cap - 1);
  return i;
}

static int smem_put(orc_smem* m, int buf, int64_t off, uint8_t v) {
  if (2 * (m->used + 1) > m->cap) {
    orc_smem g;
    g.cap = m->cap ? 2 * m->cap : 1024;
    g.used = 0;
    g.keys = (uint64_t*)calloc(g.cap, sizeof(uint64_t));
    g.vals = (uint8_t*)calloc(g.cap, 1);
    if (!g.keys || !g.vals) {
      free(g.keys);
      free(g.vals);
      return 0;
    }
    for (uint64_t i = 0; i < m->cap; i++)
      if (m->keys[i]) {
        uint64_t j = smem_slot(&g, m->keys[i]);
        g.keys[j] = m->keys[i];
        g.vals[j] = m->vals[i];
        g.used++;
      }
    free(m->keys);
    free(m->vals);
    *m = g;
  }
  uint64_t key = (((uint64_t)buf << 56) | (uint64_t)off) + 1;
  uint64_t i = smem_slot(m, key);
  if (!m->keys[i]) {
    m->keys[i] = key;
    m->used++;
  }
  m->vals[i] = v;
  return 1;
}

static uint8_t smem_get(const orc_smem* m, int buf, int64_t off) {
  if (!m->cap) return 0;
  uint64_t i = smem_slot(m, (((uint64_t)buf << 56) | (uint64_t)off) + 1);
  return m->keys[i] ? m->vals[i] : 0;
}

typedef struct {
  const orc_prog* P;
  const orc_opts* o;
  orc_result* res;
  orc_record* recs;
  uint64_t rec_cap;
  uint64_t* counts;
  int64_t len[ORC_MAX_BUFS], base[ORC_MAX_BUFS];
  int32_t sreg[16];
  int32_t r[256];
  uint32_t block_lin, thread_lin, ordinal, prev_loc;
  uint32_t h; /* the thread's digest state H */
  uint64_t backedges;
  int stopped;
  int32_t hsize[ORC_MAX_OPS];  /* per allocation site: the block's size */
  uint8_t hstate[ORC_MAX_OPS]; /* 0 never allocated, 1 live, 2 freed */
  orc_smem* sm;                /* the block's shared bytes, or NULL when
                                  shared stores are not performed */
  int nomem;
} orc_ctx;

static void cover(orc_ctx* c, int site, int outcome) {
  uint32_t cur = c->P->loc[site][outcome];
  c->counts[(cur ^ c->prev_loc) & 0xFFFFu]++;
  c->prev_loc = cur >> 1;
  c->res->n_branch++;
}

static uint8_t classify(const orc_ctx* c, int buf, int64_t off, int w) {
  int64_t R = (int64_t)c->o->redzone;
  int64_t len = c->len[buf];
  if (off < 0 && off >= -R) return ORC_CLS_UNDERFLOW_RZ;
  if (off >= 0 && off < len + R) return ORC_CLS_OVERFLOW_RZ;
  uint32_t space = (c->P->shared_mask >> buf) & 1u;
  int64_t a = c->base[buf] + off;
  for (int j = 0; j < c->P->n_bufs; j++) {
    if (j == buf || ((c->P->shared_mask >> j) & 1u) != space || c->len[j] == 0) continue;
    if (a < c->base[j] + c->len[j] && a + w > c->base[j]) return ORC_CLS_OTHER_ALLOC;
  }
  return ORC_CLS_WILD;
}

/* A violation of the current thread at its current ordinal: counts it,
 * lowers the first key, keeps the record while there is room. */
static void violation(orc_ctx* c, const orc_record* proto) {
  orc_result* res = c->res;
  uint64_t ord = c->ordinal < 0x3FFFFFu ? c->ordinal : 0x3FFFFFu;
  uint64_t key = ((uint64_t)c->block_lin << 32) | ((uint64_t)c->thread_lin << 22) | ord;
  if (key < res->first_key) res->first_key = key;
  if (res->n_violations < c->rec_cap) {
    orc_record* rec = &c->recs[res->n_violations];
    *rec = *proto;
    rec->block_lin = c->block_lin;
    rec->thread_lin = c->thread_lin;
    rec->ordinal = c->ordinal;
  }
  res->n_violations++;
}

static int32_t do_access(orc_ctx* c, const orc_op* op, int is_store) {
  int32_t idx = c->r[op->a];
  int w = op->imm;
  int buf = op->b;
  int64_t off = (int64_t)idx * (int64_t)w;
  int viol = off < 0 || off + w > c->len[buf];
  orc_result* res = c->res;
  res->n_accesses++;
  uint32_t K = ((uint32_t)op->site * 0xC2B2AE3Du) | 3u;
  c->h = c->h * K + (uint32_t)idx;
  int32_t value = 0;
  if (viol) {
    orc_record proto;
    memset(&proto, 0, sizeof(proto));
    proto.site = (uint16_t)op->site;
    proto.buf = (uint8_t)buf;
    proto.kind = (uint8_t)is_store;
    proto.width = (uint8_t)w;
    proto.space = (uint8_t)((c->P->shared_mask >> buf) & 1u);
    proto.cls = classify(c, buf, off, w);
    proto.byte_off = off;
    violation(c, &proto);
  } else if (!((c->P->shared_mask >> buf) & 1u)) {
    if (!is_store) {
      uint32_t word = fmix32(c->P->seed ^ ((uint32_t)buf * 0x9E3779B9u) ^ (uint32_t)(off >> 2));
      value = (w == 1) ? (int32_t)((word >> (8 * (off & 3))) & 0xFFu) : (int32_t)word;
    }
  } else if (c->sm && is_store) { /* a performed shared store */
    uint32_t v = (uint32_t)c->r[op->dst];
    for (int k = 0; k < w; k++)
      if (!smem_put(c->sm, buf, off + k, k < 4 ? (uint8_t)(v >> (8 * k)) : 0)) c->nomem = 1;
  } else if (c->sm) { /* a shared load of what the block stored */
    uint32_t v = 0;
    for (int k = 0; k < (w == 1 ? 1 : 4); k++) v |= (uint32_t)smem_get(c->sm, buf, off + k) << (8 * k);
    value = (int32_t)v;
  }
  c->ordinal++;
  return value;
}

/* DIV / REM: signed, truncating; a zero divisor faults and gives 0. */
static int32_t do_divide(orc_ctx* c, const orc_op* op) {
  int32_t x = c->r[op->a], y = c->r[op->b];
  int32_t value;
  if (y == 0) {
    orc_record proto;
    memset(&proto, 0, sizeof(proto));
    proto.site = (uint16_t)op->site;
    proto.kind = 2;
    proto.cls = ORC_CLS_DIV_ZERO;
    violation(c, &proto);
    value = 0;
  } else if (x == INT32_MIN && y == -1) {
    value = op->opc == OP_DIV ? INT32_MIN : 0;
  } else {
    value = op->opc == OP_DIV ? x / y : x % y;
  }
  c->ordinal++;
  return value;
}

/* HALLOC: a live block of n >= 1 bytes at this site, handle site + 1. */
static int32_t do_alloc(orc_ctx* c, const orc_op* op) {
  int32_t n = c->r[op->a];
  if (n < 1) return 0;
  c->hstate[op->site] = 1;
  c->hsize[op->site] = n;
  return op->site + 1;
}

/* HFREE: NULL is a no-op; a handle of no allocated block is an invalid
 * free, a freed block a double free. */
static void do_free(orc_ctx* c, const orc_op* op) {
  int32_t h = c->r[op->a];
  if (h != 0) {
    int cls = 0;
    if (h < 1 || h > c->P->n_alloc || c->hstate[h - 1] == 0)
      cls = ORC_CLS_INVALID_FREE;
    else if (c->hstate[h - 1] == 2)
      cls = ORC_CLS_DOUBLE_FREE;
    else
      c->hstate[h - 1] = 2;
    if (cls) {
      orc_record proto;
      memset(&proto, 0, sizeof(proto));
      proto.site = (uint16_t)op->site;
      proto.kind = 3;
      proto.space = 2;
      proto.cls = (uint8_t)cls;
      violation(c, &proto);
    }
  }
  c->ordinal++;
}

/* HLD / HST: an access through a heap handle; heap loads read 0. */
static void do_heap_access(orc_ctx* c, const orc_op* op, int is_store) {
  int32_t idx = c->r[op->a];
  int32_t h = c->r[op->b];
  int w = op->imm;
  int64_t off = (int64_t)idx * (int64_t)w;
  c->res->n_accesses++;
  uint32_t K = ((uint32_t)op->site * 0xC2B2AE3Du) | 3u;
  c->h = c->h * K + (uint32_t)idx;
  int cls = 0, buf = 0;
  if (h < 1 || h > c->P->n_alloc || c->hstate[h - 1] == 0) {
    cls = ORC_CLS_WILD;
  } else {
    buf = h - 1;
    int64_t len = c->hsize[h - 1], R = (int64_t)c->o->redzone;
    if (c->hstate[h - 1] == 2)
      cls = ORC_CLS_USE_AFTER_FREE;
    else if (off < 0 || off + w > len)
      cls = (off < 0 && off >= -R) ? ORC_CLS_UNDERFLOW_RZ
            : (off >= 0 && off < len + R) ? ORC_CLS_OVERFLOW_RZ : ORC_CLS_WILD;
  }
  if (cls) {
    orc_record proto;
    memset(&proto, 0, sizeof(proto));
    proto.site = (uint16_t)op->site;
    proto.buf = (uint8_t)buf;
    proto.kind = (uint8_t)is_store;
    proto.width = (uint8_t)w;
    proto.space = 2;
    proto.cls = (uint8_t)cls;
    proto.byte_off = off;
    violation(c, &proto);
  }
  c->ordinal++;
}

static int32_t alu(int op, int32_t x, int32_t y) {
  uint32_t ux = (uint32_t)x, uy = (uint32_t)y;
  switch (op) {
    case OP_ADD: return (int32_t)(ux + uy);
    case OP_SUB: return (int32_t)(ux - uy);
    case OP_MUL: return (int32_t)(ux * uy);
    case OP_SHL: return (int32_t)(ux << (uy & 31u));
    case OP_SHR: { /* arithmetic shift written without relying on >> of negatives */
      uint32_t s = uy & 31u;
      uint32_t v = ux >> s;
      if ((ux & 0x80000000u) && s) v |= ~(0xFFFFFFFFu >> s);
      return (int32_t)v;
    }
    case OP_SHRU: return (int32_t)(ux >> (uy & 31u));
    case OP_AND: return (int32_t)(ux & uy);
    case OP_OR: return (int32_t)(ux | uy);
    case OP_XOR: return (int32_t)(ux ^ uy);
    case OP_MIN: return x < y ? x : y;
    case OP_MAX: return x > y ? x : y;
    case OP_SETLT: return x < y;
    case OP_SETLE: return x <= y;
    case OP_SETEQ: return x == y;
    case OP_SETNE: return x != y;
    case OP_SETLTU: return ux < uy;
  }
  return 0;
}

/* Runs ops [pc, end) of the current thread.  n_ops counts the executed ops
 * that compute a value or make a check other than an access: IMM, MOV, SEL,
 * the ALU ops, DIV / REM, HALLOC and HFREE.  SREG (reading a launch
 * coordinate or an argument) and NOP are not counted, nor are accesses,
 * branches and loop heads, which have counts of their own.  On a pruned
 * program this is the work left after MathElimination (Sec. 5.2). */
static void exec_range(orc_ctx* c, int pc, int end) {
  const orc_prog* P = c->P;
  int32_t* r = c->r;
  while (pc < end && !c->stopped) {
    const orc_op* o = &P->ops[pc];
    int opc = o->opc;
    if (opc >= 0x10 && opc <= 0x1F) {
      r[o->dst] = alu(opc, r[o->a], r[o->b]);
      c->res->n_ops++;
      pc++;
      continue;
    }
    if (opc >= 0x30 && opc <= 0x3F) {
      r[o->dst] = alu(opc - 0x20, r[o->a], o->imm);
      c->res->n_ops++;
      pc++;
      continue;
    }
    switch (opc) {
      case OP_NOP: pc++; break;
      case OP_SREG: r[o->dst] = c->sreg[o->imm]; pc++; break;
      case OP_IMM: r[o->dst] = o->imm; c->res->n_ops++; pc++; break;
      case OP_MOV: r[o->dst] = r[o->a]; c->res->n_ops++; pc++; break;
      case OP_SEL:
        r[o->dst] = r[o->a] != 0 ? r[o->b] : r[o->imm];
        c->res->n_ops++;
        pc++;
        break;
      case OP_LD: r[o->dst] = do_access(c, o, 0); pc++; break;
      case OP_DIV:
      case OP_REM: r[o->dst] = do_divide(c, o); c->res->n_ops++; pc++; break;
      case OP_HALLOC: r[o->dst] = do_alloc(c, o); c->res->n_ops++; pc++; break;
      case OP_HFREE: do_free(c, o); c->res->n_ops++; pc++; break;
      case OP_HLD: do_heap_access(c, o, 0); r[o->dst] = 0; pc++; break;
      case OP_HST: do_heap_access(c, o, 1); pc++; break;
      case OP_ST: (void)do_access(c, o, 1); pc++; break;
      case OP_IF: {
        int taken = r[o->a] != 0;
        cover(c, o->site, taken);
        if (taken)
          exec_range(c, pc + 1, o->else_pc >= 0 ? o->else_pc : o->end_pc);
        else if (o->else_pc >= 0)
          exec_range(c, o->else_pc + 1, o->end_pc);
        pc = o->end_pc + 1;
        break;
      }
      case OP_LOOP: {
        /* for (ctr = 0; ctr < trip; ctr++) body;  trip = clamp(n, 0, max) */
        int32_t n = r[o->a];
        int32_t trip = n < 0 ? 0 : (n > o->imm ? o->imm : n);
        r[o->dst] = 0;
        for (;;) {
          int cont = r[o->dst] < trip;
          cover(c, o->site, cont);
          if (!cont) break;
          exec_range(c, pc + 1, o->end_pc);
          if (c->stopped) return;
          c->backedges++;
          if (c->backedges > c->o->iter_budget) {
            c->stopped = 1;
            c->res->flags |= ORC_FL_BUDGET;
            return;
          }
          r[o->dst]++;
        }
        pc = o->end_pc + 1;
        break;
      }
      default: pc++; break; /* BAR: phases are split by the caller; ELSE/ENDIF/ENDLOOP
                               are never reached inside a range */
    }
  }
}

static int invalid_config(const orc_input* in) {
  const uint32_t* g = in->grid;
  const uint32_t* b = in->block;
  if (!g[0] || !g[1] || !g[2] || !b[0] || !b[1] || !b[2]) return 1;
  if (b[0] > 1024 || b[1] > 1024 || b[2] > 64) return 1;
  if ((uint64_t)b[0] * b[1] * b[2] > 1024) return 1;
  if (g[0] > 0x7FFFFFFFu || g[1] > 65535 || g[2] > 65535) return 1;
  return 0;
}

/* One thread's state between the phases of a block. */
typedef struct {
  int32_t r[256];
  uint32_t ordinal, prev_loc, h;
  uint64_t backedges;
  int stopped;
} orc_saved;

static void thread_start(orc_ctx* c, uint64_t bl, uint64_t tl, uint32_t bx, uint32_t by) {
  const orc_prog* P = c->P;
  c->sreg[0] = (int32_t)(tl % bx);
  c->sreg[1] = (int32_t)((tl / bx) % by);
  c->sreg[2] = (int32_t)(tl / ((uint64_t)bx * by));
  memset(c->r, 0, sizeof(int32_t) * (P->n_regs ? P->n_regs : 1));
  c->block_lin = (uint32_t)bl;
  c->thread_lin = (uint32_t)tl;
  c->ordinal = 0;
  c->prev_loc = 0;
  c->backedges = 0;
  c->stopped = 0;
  memset(c->hstate, 0, (size_t)P->n_alloc);
  c->h = (uint32_t)bl * 0x9E3779B1u + (uint32_t)tl + 0x7F4A7C15u;
}

static void thread_save(const orc_ctx* c, orc_saved* s, int32_t* hsize, uint8_t* hstate) {
  memcpy(s->r, c->r, sizeof(s->r));
  s->ordinal = c->ordinal;
  s->prev_loc = c->prev_loc;
  s->h = c->h;
  s->backedges = c->backedges;
  s->stopped = c->stopped;
  memcpy(hsize, c->hsize, sizeof(int32_t) * (size_t)c->P->n_alloc);
  memcpy(hstate, c->hstate, (size_t)c->P->n_alloc);
}

static void thread_load(orc_ctx* c, const orc_saved* s, const int32_t* hsize,
                        const uint8_t* hstate, uint64_t tl, uint32_t bx, uint32_t by) {
  c->sreg[0] = (int32_t)(tl % bx);
  c->sreg[1] = (int32_t)((tl / bx) % by);
  c->sreg[2] = (int32_t)(tl / ((uint64_t)bx * by));
  memcpy(c->r, s->r, sizeof(s->r));
  c->thread_lin = (uint32_t)tl;
  c->ordinal = s->ordinal;
  c->prev_loc = s->prev_loc;
  c->h = s->h;
  c->backedges = s->backedges;
  c->stopped = s->stopped;
  memcpy(c->hsize, hsize, sizeof(int32_t) * (size_t)c->P->n_alloc);
  memcpy(c->hstate, hstate, (size_t)c->P->n_alloc);
}

/* A block of a program with performed shared stores: phase by phase (the
 * top-level BARs split the ops), every thread in thread_lin order runs the
 * phase's ops, its state kept in between.  Returns 0 or ORC_E_NOMEM. */
static int run_block_phased(orc_ctx* c, uint64_t bl, uint64_t T, uint32_t bx, uint32_t by) {
  const orc_prog* P = c->P;
  size_t na = (size_t)(P->n_alloc ? P->n_alloc : 1);
  orc_saved* st = (orc_saved*)malloc(sizeof(orc_saved) * T);
  int32_t* hsize = (int32_t*)malloc(sizeof(int32_t) * na * T);
  uint8_t* hstate = (uint8_t*)malloc(na * T);
  if (!st || !hsize || !hstate) {
    free(st);
    free(hsize);
    free(hstate);
    return ORC_E_NOMEM;
  }
  if (c->sm->cap) memset(c->sm->keys, 0, sizeof(uint64_t) * c->sm->cap); /* shared bytes: 0 */
  c->sm->used = 0;
  for (uint64_t tl = 0; tl < T; tl++) {
    thread_start(c, bl, tl, bx, by);
    thread_save(c, &st[tl], hsize + na * tl, hstate + na * tl);
  }
  int begin = 0;
  for (;;) {
    int end = begin;
    while (end < P->n_ops && P->ops[end].opc != OP_BAR) end++;
    for (uint64_t tl = 0; tl < T; tl++) {
      thread_load(c, &st[tl], hsize + na * tl, hstate + na * tl, tl, bx, by);
      exec_range(c, begin, end);
      thread_save(c, &st[tl], hsize + na * tl, hstate + na * tl);
    }
    if (end >= P->n_ops) break;
    begin = end + 1;
  }
  for (uint64_t tl = 0; tl < T; tl++) c->res->digest += st[tl].h ^ (st[tl].h >> 16);
  free(st);
  free(hsize);
  free(hstate);
  return c->nomem ? ORC_E_NOMEM : 0;
}

/* Runs one input; records (up to rec_cap; in (block, thread, ordinal) order,
 * or for programs with performed shared stores (block, phase, thread,
 * ordinal) order) and the bucketed bitmap (may be NULL) are written to the
 * caller's buffers.
 * snapshot (may be NULL = empty) is the union bitmap NEW_COV compares with. */
int orc_run(const void* handle, const orc_input* in, const orc_opts* opts, orc_result* res,
            orc_record* recs, uint64_t rec_cap, uint8_t* bitmap, const uint8_t* snapshot) {
  const orc_prog* P = (const orc_prog*)handle;
  memset(res, 0, sizeof(*res));
  res->first_key = ~0ull;
  if (bitmap) memset(bitmap, 0, 65536);
  if (invalid_config(in)) {
    res->status = ORC_ST_INVALID_CONFIG;
    return 0;
  }
  uint64_t nthreads_blk = (uint64_t)in->block[0] * in->block[1] * in->block[2];
  uint64_t nblocks = (uint64_t)in->grid[0] * in->grid[1] * in->grid[2];
  int too_big = nblocks > opts->max_threads / nthreads_blk;
  for (int k = 0; k < P->n_bufs; k++)
    if (in->buf_len[k] >= (1ull << 48)) too_big = 1;
  if (too_big) {
    res->status = ORC_ST_LIMIT;
    return 0;
  }
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  uint64_t* counts = (uint64_t*)calloc(65536, sizeof(uint64_t));
  orc_smem sm;
  memset(&sm, 0, sizeof(sm));
  if (!c || !counts) {
    free(c);
    free(counts);
    return ORC_E_NOMEM;
  }
  if (P->flags & ORC_PF_SHARED_STORES) c->sm = &sm;
  c->P = P;
  c->o = opts;
  c->res = res;
  c->recs = recs;
  c->rec_cap = rec_cap;
  c->counts = counts;
  res->n_threads = nblocks * nthreads_blk;
  /* virtual layout per space: base_0 = R, base_{k+1} = align256(base_k + len_k + R) */
  int64_t R = opts->redzone;
  int64_t next[2] = {R, R};
  for (int k = 0; k < P->n_bufs; k++) {
    int sp = (P->shared_mask >> k) & 1;
    c->len[k] = (int64_t)in->buf_len[k];
    c->base[k] = next[sp];
    next[sp] = (next[sp] + c->len[k] + R + 255) & ~(int64_t)255;
  }
  uint32_t gx = in->grid[0], gy = in->grid[1];
  uint32_t bx = in->block[0], by = in->block[1];
  for (int k = 0; k < 3; k++) {
    c->sreg[3 + k] = (int32_t)in->block[k];
    c->sreg[9 + k] = (int32_t)in->grid[k];
  }
  for (int k = 0; k < 4; k++) c->sreg[12 + k] = in->args[k];
  for (uint64_t bl = 0; bl < nblocks; bl++) {
    c->sreg[6] = (int32_t)(bl % gx);
    c->sreg[7] = (int32_t)((bl / gx) % gy);
    c->sreg[8] = (int32_t)(bl / ((uint64_t)gx * gy));
    if (c->sm) {
      int rc = run_block_phased(c, bl, nthreads_blk, bx, by);
      if (rc) {
        free(sm.keys);
        free(sm.vals);
        free(counts);
        free(c);
        return rc;
      }
      continue;
    }
    for (uint64_t tl = 0; tl < nthreads_blk; tl++) {
      thread_start(c, bl, tl, bx, by);
      exec_range(c, 0, P->n_ops);
      res->digest += c->h ^ (c->h >> 16);
    }
  }
  free(sm.keys);
  free(sm.vals);
  res->n_records = (uint32_t)(res->n_violations < rec_cap ? res->n_violations : rec_cap);
  if (res->n_violations > rec_cap) res->flags |= ORC_FL_OVERFLOW;
  res->status = res->n_violations ? ORC_ST_VIOLATION : ORC_ST_OK;
  uint32_t edges = 0;
  int newcov = 0;
  for (uint32_t e = 0; e < 65536; e++) {
    uint8_t b = bucket(counts[e]);
    if (!b) continue;
    edges++;
    if (bitmap) bitmap[e] = b;
    if (b & (uint8_t)~(snapshot ? snapshot[e] : 0)) newcov = 1;
  }
  res->n_edges = edges;
  if (newcov) res->flags |= ORC_FL_NEW_COV;
  free(counts);
  free(c);
  return 0;
}

/* ------------------------------------------------- batch over host threads */

typedef struct {
  const void* const* handles;
  uint64_t n_handles;
  const orc_input* inputs;
  const orc_opts* opts;
  orc_result* results;
  orc_record* records;
  uint64_t rec_cap;
  uint8_t* bitmaps;
  const uint8_t* snapshot;
  uint64_t n;
  uint64_t next;
  pthread_mutex_t mu;
  int err;
} orc_batch;

static void* batch_worker(void* arg) {
  orc_batch* B = (orc_batch*)arg;
  for (;;) {
    pthread_mutex_lock(&B->mu);
    uint64_t i = B->next++;
    pthread_mutex_unlock(&B->mu);
    if (i >= B->n) break;
    const orc_input* in = &B->inputs[i];
    if (in->program_id >= B->n_handles || !B->handles[in->program_id]) {
      pthread_mutex_lock(&B->mu);
      B->err = ORC_E_FORMAT;
      pthread_mutex_unlock(&B->mu);
      continue;
    }
    int e = orc_run(B->handles[in->program_id], in, B->opts, &B->results[i],
                    B->records ? B->records + i * B->rec_cap : NULL, B->records ? B->rec_cap : 0,
                    B->bitmaps ? B->bitmaps + i * 65536ull : NULL, B->snapshot);
    if (e) {
      pthread_mutex_lock(&B->mu);
      B->err = e;
      pthread_mutex_unlock(&B->mu);
    }
  }
  return NULL;
}

/* Runs n inputs over n_threads host threads; input i uses
 * handles[inputs[i].program_id]; its records go to records + i * rec_cap and
 * its bitmap to bitmaps + i * 65536 (either may be NULL). */
int orc_run_batch(const void* const* handles, uint64_t n_handles, const orc_input* inputs, uint64_t n,
                  const orc_opts* opts, orc_result* results, orc_record* records,
                  uint64_t rec_cap, uint8_t* bitmaps, const uint8_t* snapshot, int n_threads) {
  orc_batch B;
  memset(&B, 0, sizeof(B));
  B.handles = handles;
  B.n_handles = n_handles;
  B.inputs = inputs;
  B.opts = opts;
  B.results = results;
  B.records = records;
  B.rec_cap = rec_cap;
  B.bitmaps = bitmaps;
  B.snapshot = snapshot;
  B.n = n;
  pthread_mutex_init(&B.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < n_threads; t++)
    if (pthread_create(&th[started], NULL, batch_worker, &B) == 0) started++;
  if (!started) batch_worker(&B);
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&B.mu);
  return B.err;
}
