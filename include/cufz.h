/*
 * cufz.h - C ABI of the GB300 checked-execution engine.
 *
 * The engine runs a kernel under test, given as an integer access-index
 * program, over its full grid once per fuzz input (or, with CUFZ_CF_PREX,
 * over the few threads that decide the verdict, Sec. 5.1); it checks
 * every load and store against its buffer's bounds and records AFL-style
 * edge coverage.
 * This is the work the paper moves to the CPU through IR translation and
 * AddressSanitizer (Sec. 4, Fig. 2: translate, instrument with ASan and AFL,
 * run every GPU thread of every block) and then reduces with AXIPrune
 * (Sec. 5.2, Alg. 2).  Here it runs on the GPU, in hand-written sm_103a
 * kernels.
 *
 * Conventions
 *   - Every entry point returns a cufz_status: 0 on success, a negative
 *     CUFZ_E_* code otherwise.  Nothing aborts, throws across the ABI or
 *     traps; all device waits are bounded and surface as CUFZ_E_TIMEOUT.
 *   - Device memory belongs to the caller: cufz_create receives an arena
 *     (a device pointer and its size) and the library sub-allocates from it;
 *     it never calls cudaMalloc.  It allocates pinned host memory for its
 *     staging and completion buffers and creates its own CUDA streams.
 *   - The library copies program bytes and input records before a call
 *     returns; the caller may reuse its buffers at once.
 *   - Results (records, bitmaps) stay owned by the library until
 *     cufz_release (or, with CUFZ_CF_AUTO_RELEASE, until polled).
 *   - A context may be used from several host threads; calls on one
 *     context are serialised by an internal lock.
 *
 * Program format (little endian; the Python package's bytecode.py encodes
 * it):
 *   header, 32 bytes: u32 magic 0x315A4643 ("CFZ1"), u16 version 1, u16
 *     n_ops (1..2048), u8 n_regs, u8 n_bufs (<= 9), u8 n_sites (IF and LOOP
 *     ops), u8 flags (bit 0: stores to shared buffers are performed, see
 *     BAR), u16 shared_mask (bit k: buffer k is per-block shared memory),
 *     u16 0, u32 seed (content of the global buffers), u32 0 x 3;
 *   LOC table: n_sites x {u16 LOC not taken / exit, u16 LOC taken};
 *   ops, 8 bytes each: u8 opcode, u8 dst, u8 a, u8 b, i32 imm (unused
 *     fields 0).  The size is exactly 32 + 4 n_sites + 8 n_ops.
 * Opcodes: 0x01 SREG dst = special register imm (0-2 tid.xyz, 3-5
 * ntid.xyz, 6-8 ctaid.xyz, 9-11 nctaid.xyz, 12-15 scalar args 0-3); 0x02 IMM
 * dst = imm; 0x03 MOV dst = a; 0x04 SEL dst = a != 0 ? b : register imm;
 * 0x05 DIV and 0x06 REM dst = a / b and a % b, signed and truncating: a zero
 * divisor is a fault (a violation of kind 2, result 0), INT_MIN / -1 is
 * INT_MIN and INT_MIN % -1 is 0;
 * 0x07 HALLOC dst = a heap block of a bytes (the device heap of Sec. 2.3,
 * per test thread): the k-th HALLOC's block, handle k + 1, live with a
 * bytes, or 0 (NULL, nothing changes) when a <= 0; 0x08 HFREE frees the
 * block of handle a: 0 is a no-op, a handle of no block this thread
 * allocated is an invalid free and a freed block a double free (both
 * violations of kind 3, space 2, the block stays as it was); 0x42 HLD dst
 * = heap block of handle b at index a, width imm (reads 0), and 0x43 HST
 * (register dst, never performed): accesses to space 2, a handle of no
 * allocated block a wild access, a freed block a use after free, otherwise
 * checked against the block's size like a buffer of the redzone classes
 * (no neighbours);
 * 0x10-0x1F ALU dst = a op b and 0x30-0x3F the same with b = imm, op in
 * order add, sub, mul, shl, shr (arithmetic), shru, and, or, xor, min, max
 * (signed), setlt, setle, seteq, setne (signed, 0 or 1), setltu (unsigned),
 * all on int32 with wrap-around and shift counts taken mod 32; 0x40 LD dst =
 * buffer b at index a, width imm (1, 4, 8 or 16 bytes); 0x41 ST register
 * dst to buffer b at index a, width imm (checked, never performed); 0x50 IF
 * a, 0x51 ELSE, 0x52 ENDIF; 0x53 LOOP with counter dst and trip count
 * clamp(a, 0, imm), 0x54 ENDLOOP; 0x55 BAR, a block-wide barrier outside
 * every IF and LOOP.  With flags bit 0 each block's shared buffers start
 * as zero bytes, an in-bounds ST to one writes the value's little-endian
 * bytes (width 1: the low byte; widths 8 and 16: the four bytes, then
 * zeros) and an in-bounds LD reads them back (width 1: the byte; wider: the
 * int32 of the first four bytes); the BARs split the program into phases
 * that every thread of a block finishes, in thread order, before the next
 * phase.  The engine runs such a program only when BarrierElimination
 * (Sec. 5.2, Alg. 2) applies: no value loaded from a shared buffer reaches
 * an index, a branch, a loop trip, a divisor or a heap operand.  The
 * stores then change no check, and it runs the program without them and
 * without its barriers; any other such program loads as
 * CUFZ_E_UNSUPPORTED.  Without the flag, stores are never performed,
 * shared loads read 0 and BAR does nothing.
 * Control flow is structured, at most 16 deep; a loop counter is read-only
 * in its body.  The k-th LD/ST/HLD/HST in program order is access site k,
 * the k-th IF/LOOP branch site k, the k-th DIV/REM division site k, the
 * k-th HFREE free site k.  The program's registers and one register per
 * HALLOC must fit the interpreter's 128 per thread: a program above that
 * loads as CUFZ_E_INVALID_PROGRAM.
 *
 * Input, result and violation records are the fixed-layout structs below.
 */
#ifndef CUFZ_H
#define CUFZ_H

#if !defined(__CUDACC_RTC__)
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cufz_ctx cufz_ctx;
typedef int32_t cufz_status;

/* ---------------------------------------------------------------- status */
#define CUFZ_OK 0
#define CUFZ_E_INVALID_ARG (-1)     /* NULL pointer, bad size, bad config field */
#define CUFZ_E_INVALID_PROGRAM (-2) /* program bytes rejected by the validator */
#define CUFZ_E_NOMEM (-3)           /* arena too small, or a table is full */
#define CUFZ_E_BUSY (-4)            /* no free slot: poll, release, resubmit */
#define CUFZ_E_TIMEOUT (-5)         /* a bounded wait gave up */
#define CUFZ_E_CUDA (-6)            /* a CUDA runtime call failed */
#define CUFZ_E_NOT_FOUND (-7)       /* unknown ticket or program id */
#define CUFZ_E_NO_DEVICE (-8)       /* no usable CUDA device */
#define CUFZ_E_DEVICE_FAULT (-9)    /* the device reported an internal error word */
#define CUFZ_E_IO (-10)             /* the autotune cache file could not be written */
#define CUFZ_E_UNSUPPORTED (-11)    /* a valid program the engine does not run: a value
                                       loaded from a shared buffer whose stores are
                                       performed reaches an index, a branch, a loop
                                       trip, a divisor or a heap operand */

/* per-input status (cufz_result.status) */
#define CUFZ_ST_OK 0
#define CUFZ_ST_VIOLATION 1      /* at least one out-of-bounds access */
#define CUFZ_ST_INVALID_CONFIG 2 /* CUDA would reject the launch (Sec. 2.3.1) */
#define CUFZ_ST_LIMIT 3          /* beyond the engine's limits (max_threads, len >= 2^48) */
#define CUFZ_ST_BAD_PROGRAM 4    /* program_id names no loaded program */

/* per-input flags (cufz_result.flags) */
#define CUFZ_FL_BUDGET 1   /* some thread exceeded the back-edge budget (hang analog) */
#define CUFZ_FL_OVERFLOW 2 /* more violations than record_cap; counts stay exact */
#define CUFZ_FL_NEW_COV 4  /* bitmap has a bucket bit the epoch's union lacks */
#define CUFZ_FL_PARTIAL 8  /* CUFZ_CF_PREX ran only the planned threads: the status
                              (violation or not) is the full grid's; counts,
                              records, digest and bitmap cover those threads */

/* violation classes (cufz_violation.cls) */
#define CUFZ_CLS_UNDERFLOW_RZ 1 /* byte_off in [-R, 0) */
#define CUFZ_CLS_OVERFLOW_RZ 2  /* access overlaps [len, len + R) */
#define CUFZ_CLS_OTHER_ALLOC 3  /* lands in another buffer of the same space */
#define CUFZ_CLS_WILD 4         /* anything else */
#define CUFZ_CLS_DIV_ZERO 5     /* a division (record kind 2) by zero */
#define CUFZ_CLS_USE_AFTER_FREE 6 /* a heap access to a freed block */
#define CUFZ_CLS_DOUBLE_FREE 7    /* HFREE (record kind 3) of a freed block */
#define CUFZ_CLS_INVALID_FREE 8   /* HFREE of a handle of no allocated block */

/* configuration flags (cufz_config.flags) */
#define CUFZ_CF_KEEP_BITMAPS 1 /* keep each input's 64 KiB bitmap until released */
#define CUFZ_CF_PLAIN_LAUNCH 2 /* baseline path: one kernel launch per input */
#define CUFZ_CF_NO_PRUNE 4     /* run programs unpruned (the pruning check) */
#define CUFZ_CF_AUTO_RELEASE 8 /* release a slot as soon as its result is polled */
#define CUFZ_CF_NO_GRAPH 16    /* launch batches directly, not through a CUDA graph */
#define CUFZ_CF_NO_DIGEST 32   /* skip the per-access digest */
#define CUFZ_CF_JIT 64         /* run programs compiled to sm_103a code at load time
                                  instead of through the bytecode interpreter */
#define CUFZ_CF_JIT_FAST_COMPILE 128 /* compile faster, run slower (compiled path) */
#define CUFZ_CF_PREX 256       /* partial representative execution (Sec. 5.1): an input
                                  with a plan (cufz_prex_plan) of at most
                                  CUFZ_PREX_MAX_PLAN threads runs only those threads,
                                  flagged CUFZ_FL_PARTIAL */

#define CUFZ_PREX_MAX_PLAN 4096 /* larger plans run the full grid */

/* Engine configuration.  cufz_config_default fills every field; a zero in
 * max_slots, item_threads or cta_threads means "choose automatically". */
typedef struct {
  int32_t device;        /* CUDA device ordinal */
  uint32_t flags;        /* CUFZ_CF_* */
  void* stream;          /* caller's cudaStream_t: the arena is first touched on it */
  void* arena;           /* device memory owned by the caller, 256-byte aligned */
  uint64_t arena_bytes;  /* its size */
  uint32_t max_slots;    /* inputs resident at once (admission limit) */
  uint32_t record_cap;   /* violation records kept per input */
  uint32_t redzone;      /* R, bytes, for classification (default 256) */
  uint32_t iter_budget;  /* back-edges per test thread before it stops (default 4096) */
  uint64_t max_threads;  /* test threads per input beyond which LIMIT (<= 2^31) */
  uint32_t item_threads; /* test threads per work item (multiple of 32) */
  uint32_t cta_threads;  /* threads per CTA of the persistent kernel (64..1024) */
  uint32_t n_lanes;      /* batches that may overlap on the device (1..8) */
  uint32_t ctas_per_sm;  /* persistent CTAs per SM (0 = from occupancy) */
  uint32_t jit_min_ctas; /* compiled path: CTAs per SM its registers must allow (0 = 3) */
  uint32_t lane_items;   /* work items a batch's staging memory holds (0 = 2^20); the
                            arena grows with it (cufz_arena_bytes) and admission stops
                            where a batch's items would exceed it */
  const char* autotune_cache; /* NULL, or a file that keeps the autotuner's
                                 per-program choices across contexts and
                                 processes (read at create, applied at load,
                                 rewritten by cufz_autotune) */
} cufz_config;

/* One fuzz input, 128 bytes.  grid/block are the launch shape of the kernel
 * under test; args its four scalar arguments; buf_len[k] the byte length of
 * buffer k (for a shared buffer: its size per block). */
typedef struct {
  uint32_t program_id;
  uint32_t grid[3];
  uint32_t block[3];
  int32_t args[4];
  uint32_t reserved;
  uint64_t buf_len[9];
  uint64_t user_tag; /* returned unchanged in the result */
} cufz_input;

/* Result summary of one input, 96 bytes. */
typedef struct {
  uint64_t ticket;
  uint64_t user_tag;
  int32_t status;        /* CUFZ_ST_* */
  uint32_t flags;        /* CUFZ_FL_* */
  uint64_t n_accesses;   /* executed loads + stores (checked thread-accesses) */
  uint64_t n_violations; /* exact, even when records overflowed */
  uint64_t first_key;    /* min of block_lin<<32 | thread_lin<<22 | min(ordinal, 2^22-1) */
  uint64_t digest;       /* sum over test threads of a hash of the thread's
                            (site, index) access sequence, mod 2^64
                            (pruning check) */
  uint64_t n_branch;     /* branch evaluations (coverage events) */
  uint64_t n_threads;    /* test threads run */
  uint64_t n_ops;        /* executed program ops, summed over test threads */
  uint32_t n_records;    /* records stored (<= record_cap) */
  uint32_t n_edges;      /* nonzero bitmap entries */
  uint64_t n_branch_folded; /* of n_branch: loop-head evaluations whose edge
                               update the compiled path made in closed form,
                               as part of one add for a loop's repeated head
                               edge (0 on the interpreter) */
} cufz_result;

/* One violation record, 32 bytes; ids are linear:
 * block_lin = bx + by*gx + bz*gx*gy, thread_lin = tx + ty*Bx + tz*Bx*By. */
typedef struct {
  uint32_t block_lin;
  uint32_t thread_lin;
  uint32_t ordinal; /* checked events (accesses, divisions, frees) of this
                       thread before this one */
  uint16_t site;    /* kind 0/1: access site (LD/ST/HLD/HST in order);
                       kind 2: index of the DIV/REM among its DIV/REMs;
                       kind 3: index of the HFREE among its HFREEs */
  uint8_t buf;      /* the buffer; space 2: the block's allocation site (0
                       for a handle of no block); kinds 2 and 3: 0 */
  uint8_t kind;     /* 0 load, 1 store, 2 division by zero, 3 bad free */
  uint8_t width;    /* bytes (kinds 2 and 3: 0) */
  uint8_t space;    /* 0 global, 1 shared, 2 device heap (kind 2: 0) */
  uint8_t cls;      /* CUFZ_CLS_* */
  uint8_t pad0;
  uint32_t pad1;
  int64_t byte_off; /* index * width (kinds 2 and 3: 0) */
} cufz_violation;

#if !defined(__CUDACC_RTC__)
/* Statistics of a context since creation (or the last reset). */
typedef struct {
  uint64_t inputs_submitted;
  uint64_t inputs_completed;
  uint64_t kernel_launches;   /* engine kernels launched */
  uint64_t graph_launches;    /* of which through CUDA graphs */
  uint64_t batches;
  double kernel_ms;           /* device time of engine kernels (CUDA events) */
  uint32_t cta_threads;       /* launch shape in use */
  uint32_t ctas_per_sm;
  uint32_t item_threads;
  uint32_t n_sms;
  uint32_t max_slots;
  uint32_t smem_bytes;
  uint32_t graph_failures;    /* batches that fell back to direct launches */
  int32_t last_cuda_error;    /* last CUDA error code seen by the runtime (0 = none) */
  /* overlap of batches on the device (from their CUDA events, among the
     last 256 retired batches): pairs whose device intervals intersect, and
     the most batches running at one moment */
  uint64_t overlapping_batch_pairs;
  uint32_t max_concurrent_batches;
  uint32_t reserved;
} cufz_stats;

/* ------------------------------------------------ device fuzzing campaign
 * AFL++'s coverage-guided loop (Sec. 2.1, Fig. 1; the harness of Sec. 4)
 * with its queue, corpus and bug buckets resident on the device.  A round
 * takes `batch` parents from the corpus, favoured entries first (those that
 * brought new coverage and have not been picked since), least picked first,
 * then the lowest index, round robin; mutates a copy of each (cufz_mutate_children's streams, round r,
 * child j); runs the children on the context's compiled kernel; adds the
 * children flagged CUFZ_FL_NEW_COV to the corpus as favoured entries, in
 * child order; files every violating child under the key (program_id,
 * site, cls) of its first stored violation record (the least block, thread
 * and ordinal); keeps the children flagged CUFZ_FL_BUDGET and NEW_COV as
 * unique hangs; and renews the union's epoch snapshot.  Every step is a
 * kernel; a round is one launch of a CUDA graph, and no round waits for the
 * host.  (The host campaign in the Python package, fuzz.Campaign, follows
 * the same rules, one device batch per round.) */
typedef struct cufz_campaign cufz_campaign;

typedef struct {
  uint32_t batch;        /* children per round, 1..8192 (the context needs as
                            many free slots) */
  uint32_t corpus_cap;   /* corpus entries kept, 1..16384; later entries with
                            new coverage are counted as dropped */
  uint32_t bucket_cap;   /* bug bucket table size, a power of two, 16..2^20 */
  uint32_t hang_cap;     /* unique hangs kept, 1..2^20 */
  uint32_t item_threads; /* work-item size (0: the context's configured or
                            autotuned size, else 64 x its CTA threads) */
  uint32_t max_items;    /* work items per round, <= 2^24 (0: 64 per child); a child
                            whose items would pass it, counting the children
                            admitted before it in child order, completes as
                            CUFZ_ST_LIMIT */
  uint64_t seed;         /* of the children's mutation streams */
} cufz_campaign_config;

typedef struct {
  uint64_t key;      /* program_id << 32 | site << 8 | cls of the first
                        stored violation (site 0xFFFF, cls 0xFF: none stored);
                        for a child whose violations overflowed the record
                        area, which records were stored, and so the key, can
                        depend on the order its threads finished */
  uint64_t first;    /* round << 32 | child index of its first child */
  uint32_t hits;     /* violating children filed under it */
  uint32_t pad;
  cufz_input input;  /* that first child */
} cufz_bucket;

typedef struct {
  uint64_t rounds, executed, violating, hang_execs, new_coverage;
  uint32_t corpus, buckets, hangs;
  uint32_t corpus_dropped, buckets_dropped, hangs_dropped;
  uint32_t limit_children; /* children refused by max_items */
  uint32_t cycles_done;    /* least pick count in the corpus (queue cycles) */
} cufz_campaign_stats;

/* Device bytes a campaign of this configuration needs (0 for an invalid
 * configuration). */
uint64_t cufz_campaign_bytes(const cufz_campaign_config* cfg);

/* Creates a campaign over a context created with CUFZ_CF_JIT (not
 * CUFZ_CF_PLAIN_LAUNCH), in caller-owned device memory dev_mem (256-byte
 * aligned, cufz_campaign_bytes large; the caller frees it after
 * cufz_campaign_destroy).  Runs the n_seeds seeds once through the context
 * (AFL's dry run: the union then holds their coverage) and starts a new
 * epoch; the seeds become the corpus, favoured, picked 0 times.  Then
 * reserves `batch` of the context's slots and sets every loaded program to
 * the compiled path.  While a campaign exists the context's compiled module
 * stays as it is: loading or unloading programs or changing their paths or
 * lane mappings makes submits that would rebuild it, and cufz_destroy,
 * return CUFZ_E_BUSY.  The context may run other inputs meanwhile (on its
 * other slots); they share its union, and each campaign round renews the
 * union's epoch snapshot.  CUFZ_E_INVALID_ARG for a bad configuration, memory
 * or seed count (1..corpus_cap), checked before anything runs; CUFZ_E_BUSY
 * without batch free slots; CUFZ_E_UNSUPPORTED for a context without the
 * compiled path.  These last two are found after the dry run, so the
 * context's union then holds the seeds' coverage. */
cufz_status cufz_campaign_create(cufz_ctx* ctx, const cufz_campaign_config* cfg, void* dev_mem,
                                 uint64_t dev_bytes, const cufz_input* seeds, uint32_t n_seeds,
                                 cufz_campaign** out);

/* Enqueues `rounds` rounds on the campaign's stream and returns; they run
 * one after another with no host involvement.  CUFZ_E_BUSY if the
 * context's module changed since the campaign was created. */
cufz_status cufz_campaign_run(cufz_campaign* camp, uint32_t rounds);

/* Waits for the enqueued rounds (timeout_us < 0: up to 120 s);
 * CUFZ_E_TIMEOUT if they are still running. */
cufz_status cufz_campaign_sync(cufz_campaign* camp, int32_t timeout_us);

/* Counters of the campaign (after its enqueued rounds). */
cufz_status cufz_campaign_get_stats(cufz_campaign* camp, cufz_campaign_stats* out);

/* The corpus in entry order: up to cap inputs (out may be NULL), their
 * favoured flags and pick counts (either may be NULL); *n = corpus size. */
cufz_status cufz_campaign_corpus(cufz_campaign* camp, cufz_input* out, uint8_t* favoured,
                                 uint32_t* picks, uint32_t cap, uint32_t* n);

/* The bug buckets, sorted by key: up to cap of them; *n = their number. */
cufz_status cufz_campaign_buckets(cufz_campaign* camp, cufz_bucket* out, uint32_t cap, uint32_t* n);

/* The unique hangs in the order they were found, with their rounds. */
cufz_status cufz_campaign_hangs(cufz_campaign* camp, cufz_input* out, uint64_t* rounds, uint32_t cap,
                                uint32_t* n);

/* Restores a saved campaign into one just created with the saved corpus as
 * its seeds (whose dry run rebuilt the union): the entries' favoured flags
 * and pick counts (n_corpus = the corpus size), the buckets, the unique
 * hangs and the counters (rounds, executed, violating, hang_execs,
 * new_coverage and the dropped and refused counts).  Afterwards the
 * campaign continues as the saved one would have.  CUFZ_E_INVALID_ARG when
 * n_corpus is not the corpus size, or for more hangs than hang_cap or more
 * buckets than half of bucket_cap (the table keeps room to probe). */
cufz_status cufz_campaign_restore(cufz_campaign* camp, const uint8_t* favoured, const uint32_t* picks,
                                  uint32_t n_corpus, const cufz_bucket* buckets, uint32_t n_buckets,
                                  const cufz_input* hangs, const uint64_t* hang_rounds, uint32_t n_hangs,
                                  const cufz_campaign_stats* counters);

/* Waits for the enqueued rounds, returns the slots to the context and frees
 * the campaign's host resources (not dev_mem). */
cufz_status cufz_campaign_destroy(cufz_campaign* camp);

/* Statistics of a loaded (or pruned) program. */
typedef struct {
  uint32_t n_ops_in;     /* ops of the program as given */
  uint32_t n_ops_kept;   /* ops left after pruning */
  uint32_t n_regs_in;
  uint32_t n_regs_alloc; /* device registers after allocation */
  uint32_t n_access_sites;
  uint32_t n_branch_sites;
  uint32_t n_loads_value_dead; /* loads kept as checks whose value is unused */
  uint32_t reserved;
} cufz_prog_stats;

/* ------------------------------------------------------------ host-only
 * These need no GPU. */

/* Fills a configuration with defaults (device 0, no arena). */
void cufz_config_default(cufz_config* cfg);

/* Bytes of arena needed for n_slots resident inputs under cfg's
 * record_cap and flags (plus the fixed tables). */
uint64_t cufz_arena_bytes(const cufz_config* cfg, uint32_t n_slots);

/* Validates program bytes (format, operands, nesting <= 16, loop counters
 * read-only in their body).  Returns CUFZ_OK or CUFZ_E_INVALID_PROGRAM. */
cufz_status cufz_validate_program(const void* bytes, size_t nbytes);

/* AXIPrune (Sec. 5.2, Alg. 2) on the program format: BarrierElimination
 * drops every BAR (CUFZ_E_UNSUPPORTED for a program with performed shared
 * stores whose barriers cannot go: a loaded shared value reaches a check;
 * the flag itself stays), and MathElimination drops every op whose result
 * reaches no access index, branch condition or loop trip count (stored
 * values are dropped; loads stay as checked accesses), then renumbers
 * registers.  Writes the pruned program in the
 * same format to out (capacity out_cap bytes; *out_bytes gets its size;
 * CUFZ_E_NOMEM if out_cap is smaller, so out = NULL, out_cap = 0 asks for
 * the size).  stats (may be NULL) receives the op and register counts.
 * Every access and branch decision of every thread is unchanged. */
cufz_status cufz_prune_program(const void* bytes, size_t nbytes, void* out, size_t out_cap,
                               size_t* out_bytes, cufz_prog_stats* stats);

/* The CUDA source the compiled path (CUFZ_CF_JIT) generates for one program
 * (pruned unless flags has CUFZ_CF_NO_PRUNE): a __device__ function running
 * a work item of that program, NUL-terminated.  *out_bytes receives the size
 * needed; CUFZ_E_NOMEM if out_cap is smaller. */
cufz_status cufz_program_cuda(const void* bytes, size_t nbytes, uint32_t flags, char* out,
                              size_t out_cap, size_t* out_bytes);

/* Generates and runtime-compiles the module for n programs for sm_103a
 * without loading it (no device needed): CUFZ_OK, or CUFZ_E_INVALID_PROGRAM
 * with the compiler's log in log. */
cufz_status cufz_compile_check(const void* const* progs, const size_t* sizes, uint32_t n,
                               uint32_t flags, char* log, uint32_t log_cap, size_t* cubin_bytes);

/* PREX check (Sec. 5.1): *eligible = 1 when the corner threads of `in`
 * (every thread and block coordinate first or last: at most 64) decide
 * whether any thread of its grid violates.  That holds (the theorem of
 * Sec. 5.1.1) when, executing the program once with thread-invariant
 * values, every branch condition and loop trip count is the same for all
 * threads, every access index is thread-invariant or an affine function of
 * the thread and block indices with thread-invariant coefficients, and no
 * such affine value can leave the int32 range in the launch box (the device
 * computes in wrapping 32-bit arithmetic).  Programs with thread-dependent
 * guards (the paper's Alg. 1 case, a heuristic) are not eligible, nor are
 * programs with divisions or heap ops, programs the engine does not load
 * (CUFZ_E_UNSUPPORTED), and launches it does not run (invalid shapes, more
 * than 2^31 threads).
 * iter_budget: the context's back-edge budget (0 = 4096). */
cufz_status cufz_prex_check(const void* bytes, size_t nbytes, const cufz_input* in,
                            uint32_t iter_budget, uint32_t* eligible);

/* PREX plan (Sec. 5.1): the test threads whose execution decides whether any
 * thread of `in`'s grid violates, as sorted linear ids g = block_lin * T +
 * thread_lin (T = threads per block), written to threads[0 .. *n_threads).
 * Two rules give a plan:
 *   - corners: cufz_prex_check's rule; the plan is the corner threads;
 *   - guarded grids (the guarded kernels of Sec. 5.1's Alg. 1, decided
 *     exactly rather than heuristically): each launch dimension is one axis,
 *     its global coordinate ctaid * ntid + tid, or two, tid and ctaid.  The
 *     program's values must be thread-invariant, affine in the thread and
 *     block indices, or piecewise affine: one of a few affine functions in
 *     each cell (min/max of affine values, a register the two sides of a
 *     guard set differently), all without int32 wrap in the launch box.  Its
 *     branch conditions must be guards or combinations of guards.  A guard compares
 *     values affine in one dimension's coordinates (<, <=, ==, !=, or an
 *     affine value against zero), so its truth changes only at a few cuts
 *     of that dimension's axes.  The cuts split the launch box into cells in
 *     which every condition is constant and every access index is affine.
 *     An affine index violates somewhere in a cell iff it does at one of the
 *     cell's corners.  The plan is the threads whose every axis coordinate
 *     is an end of its axis or lies next to a cut.  Both sides of each guard
 *     are explored, loop trips must be thread-invariant, and iter_budget
 *     bounds the abstract back-edges (0 = 4096).
 * *n_threads = 0 when neither rule applies (run the full grid), and for
 * launches the engine does not run (invalid shapes, more than 2^31 threads)
 * and for programs with divisions.  CUFZ_E_NOMEM when the plan has more than
 * cap threads (*n_threads gives the size).
 * Host-only; no device needed. */
cufz_status cufz_prex_plan(const void* bytes, size_t nbytes, const cufz_input* in,
                           uint32_t iter_budget, uint32_t* threads, uint32_t cap,
                           uint32_t* n_threads);

/* The fuzzing campaign's mutator (host-only, no device needed): mutates n
 * input records in place.  Each input gets one to three mutations of a
 * scalar argument or of the length of one of its program's buffers
 * (buffers 0 .. n_bufs[program_id] - 1).  A mutation flips one bit (of the
 * low 24 for a length), adds or subtracts 1..35 (a length stops at 0), or
 * substitutes a boundary value: 0, +-1, 2^k, 2^k +- 1 or -2^k for an
 * argument, and one of 29 lengths from 0 to 65536.  These are AFL's
 * deterministic-stage kinds drawn at random (Sec. 2.1).  Launch shapes are
 * left alone.  The draws come from a SplitMix64 stream whose 64-bit state
 * *rng_state is read and advanced, so a campaign resumes exactly from a
 * saved state.  CUFZ_E_INVALID_ARG for a program_id >= n_programs or an
 * n_bufs entry above 9 (and then nothing is changed). */
cufz_status cufz_mutate_inputs(cufz_input* inputs, uint32_t n, const uint8_t* n_bufs,
                               uint32_t n_programs, uint64_t* rng_state);

/* The mutator of the device fuzzing campaign below, on the host: mutates
 * inputs[j] with the draws of cufz_mutate_inputs from the SplitMix64 state
 * seed + ((round << 32) | j) * 0xD1B54A32D192ED03, one stream per child, so
 * the children of a round are mutated independently of one another (the
 * campaign's kernel mutates them in parallel from the same states).  The
 * host campaign uses it to follow the device campaign exactly.
 * CUFZ_E_INVALID_ARG as for cufz_mutate_inputs.  Host-only. */
cufz_status cufz_mutate_children(cufz_input* inputs, uint32_t n, const uint8_t* n_bufs,
                                 uint32_t n_programs, uint64_t seed, uint64_t round);

/* Human-readable name of a status code (the error classes of Sec. 2.3.1 and
 * Sec. 2.3.2 that the engine reports, and the context's own errors). */
const char* cufz_status_str(cufz_status s);

/* ------------------------------------------------------------- context */

/* Creates an engine on cfg->device over cfg->arena.  Clears the arena's
 * tables on cfg->stream and waits for that.  *out is NULL on failure.
 * Stands in for the runtime libraries of Sec. 4 (CPU-side cudaMalloc /
 * cudaMemcpy emulation and the thread pool over blocks): here the caller's
 * arena and stream are the device memory and the engine is the pool. */
cufz_status cufz_create(const cufz_config* cfg, cufz_ctx** out);

/* Waits (bounded) for in-flight work, then frees host-side resources.  The
 * arena is left to the caller.  (The end of a Sec. 4 runtime's process; no
 * separate counterpart in the paper.) */
cufz_status cufz_destroy(cufz_ctx* ctx);

/* The kernel translator of Sec. 4 (cuf-cc's AXIPrune pass, Sec. 5.2, Alg. 2,
 * then code generation) for one kernel-under-test given as a program.
 * Validates, prunes (unless the context's config has CUFZ_CF_NO_PRUNE:
 * pruning is chosen per context, not per call, so the call takes no flags),
 * allocates registers and uploads one program;
 * *program_id receives its id: the lowest id freed by
 * cufz_unload_program, else the next new one (0, 1, ...).  Programs stay
 * resident until unloaded or the context is destroyed.  Up to 256 loaded at
 * a time, 8 MiB of loaded program blobs (CUFZ_E_NOMEM beyond).
 * CUFZ_E_INVALID_PROGRAM for bytes the format rejects, CUFZ_E_UNSUPPORTED
 * for a program with performed shared stores whose barriers BarrierElimination
 * cannot remove. */
cufz_status cufz_load_program(cufz_ctx* ctx, const void* bytes, size_t nbytes,
                              uint32_t* program_id, cufz_prog_stats* stats);

/* Unloads a program: its device blob's space and its id become free for
 * later loads, and inputs that name it complete with CUFZ_ST_BAD_PROGRAM.
 * CUFZ_E_BUSY while inputs of the program are in flight, i.e. submitted and
 * not yet collected by cufz_poll_results or cufz_sync (collect, then retry);
 * CUFZ_E_NOT_FOUND for an id that is not loaded.  Results already completed
 * stay readable until released.  (Program loading and unloading are the
 * harness's job in the paper, Sec. 4; the call has no counterpart there.) */
cufz_status cufz_unload_program(cufz_ctx* ctx, uint32_t program_id);

/* The pruning check (Sec. 5.2: AXIPrune drops only instructions that feed no
 * memory address or branch, so every access is kept exactly).  Runs the n
 * inputs (their program_id is ignored) on loaded program `program_id` and
 * on the same program loaded unpruned (interpreted, a temporary id unloaded
 * afterwards), and counts in *n_mismatch the inputs whose outcomes differ
 * in anything pruning must keep: status, budget and overflow flags, access,
 * violation, branch and thread counts, first-violation key, access digest,
 * record count, edge count, bitmap (if kept) and, when not overflowing, the
 * record set.  Needs an idle context (CUFZ_E_BUSY otherwise); both runs
 * update the coverage union like any other inputs. */
cufz_status cufz_verify_prune(cufz_ctx* ctx, uint32_t program_id, const cufz_input* inputs,
                              uint32_t n, uint32_t* n_mismatch);

/* One fuzz execution per input (Sec. 4: the translated program run on a
 * fuzzer-provided input; Sec. 4.1: every thread of every block, here on
 * the GPU), with every access checked (the ASan checks of Sec. 4) and
 * edges counted (Sec. 2.1, the AFL trampolines after branches).
 * Admits a prefix of in[0..n) while slots are free and while the batch's
 * staging memory holds the admitted inputs' work items (admission by
 * memory: a large grid takes more of it); each admitted input gets ticket
 * first_ticket + i.  Inputs with an invalid launch configuration, beyond
 * the limits (an input whose work items exceed a batch's staging memory on
 * their own included) or naming no program are admitted and complete at
 * once with their status, without device work.  Returns CUFZ_E_BUSY (with
 * *n_accepted < n) when it ran out of slots or staging memory; the caller
 * polls and resubmits the rest.  The admitted inputs run as one batch: one persistent launch
 * (through a CUDA graph unless CUFZ_CF_NO_GRAPH), or one launch per input
 * with CUFZ_CF_PLAIN_LAUNCH.  Batches of successive calls overlap on the
 * device. */
cufz_status cufz_submit_inputs(cufz_ctx* ctx, const cufz_input* in, uint32_t n,
                               uint32_t* n_accepted, uint64_t* first_ticket);

/* What afl-fuzz reads back from a finished child (Sec. 2.1): the crash or
 * not (status, violation counts, first-violation key in place of ASan's
 * abort at the first error) and the coverage summary.
 * Copies up to max completed results (in completion order) to out and sets
 * *n_out.  Waits up to timeout_us microseconds for the first one when none
 * is ready (0: do not wait; <0: wait until all submitted inputs are done,
 * bounded by an internal limit). */
cufz_status cufz_poll_results(cufz_ctx* ctx, cufz_result* out, uint32_t max, uint32_t* n_out,
                              int32_t timeout_us);

/* Copies the stored violation records of a completed, unreleased ticket
 * (in device write order; *n receives min(n_records, cap)).  The records are
 * what ASan reports per error (Sec. 2.1, Sec. 4), kept for every violating
 * access up to the record cap instead of only the first. */
cufz_status cufz_get_records(cufz_ctx* ctx, uint64_t ticket, cufz_violation* out, uint32_t cap,
                             uint32_t* n);

/* Copies the 64 KiB bucketed edge bitmap of a completed, unreleased ticket
 * (needs CUFZ_CF_KEEP_BITMAPS): the AFL coverage map of one execution
 * (Sec. 2.1, the payload's hit counts, bucketed as AFL classifies them). */
cufz_status cufz_get_bitmap(cufz_ctx* ctx, uint64_t ticket, uint8_t* out65536);

/* Copies the device union bitmap (OR of every completed input's bitmap):
 * the fuzzer's record of coverage seen so far, which decides whether an
 * input found new paths (Sec. 2.1, the fitness of AFL's genetic loop). */
cufz_status cufz_get_union(cufz_ctx* ctx, uint8_t* out65536);

/* Waits for all in-flight inputs, then snapshots the union: NEW_COV of later
 * inputs is measured against this snapshot, which keeps it independent of
 * completion order.  The first epoch's snapshot is empty.  (AFL compares
 * each execution with the coverage seen before it, Sec. 2.1; a batch of
 * concurrent executions compares with the state at its epoch's start.) */
cufz_status cufz_new_epoch(cufz_ctx* ctx);

/* Frees the slot of a completed ticket (records and bitmap go with it).
 * No counterpart in the paper (each execution there is a forked child
 * whose memory goes when it exits, Sec. 2.1). */
cufz_status cufz_release(cufz_ctx* ctx, uint64_t ticket);

/* Waits until every submitted input has completed (bounded).  No
 * counterpart in the paper (its runtime runs each execution to completion,
 * Sec. 4). */
cufz_status cufz_sync(cufz_ctx* ctx, int32_t timeout_us);

/* Compiles every loaded program to sm_103a code with the runtime compiler
 * (one module; programs become straight-line functions with their registers
 * in hardware registers) and loads it.  Used by CUFZ_CF_JIT; runs by itself
 * at the next submit when programs were loaded since the last compile.  The
 * compiler's log is copied to log (capacity log_cap, may be NULL). */
cufz_status cufz_compile_programs(cufz_ctx* ctx, char* log, uint32_t log_cap);

/* Chooses how a program runs when CUFZ_CF_JIT is set: compiled (1) or by the
 * bytecode interpreter (0).  A batch runs its compiled programs' work items
 * and its interpreted programs' work items as two persistent launches.
 * The default at load is compiled. */
cufz_status cufz_set_program_path(cufz_ctx* ctx, uint32_t program_id, uint32_t compiled);
cufz_status cufz_get_program_path(cufz_ctx* ctx, uint32_t program_id, uint32_t* compiled);

/* Lane mapping of a compiled program: the test threads each CUDA thread of
 * the persistent kernel runs per iteration of the program's work-item loop
 * (1, 2 or 4; consecutive iterations of a lane take test threads one CTA
 * apart, so the mapping only interleaves their instructions).  Results do
 * not depend on it.  The default is 1, or the autotune cache's choice; a
 * change recompiles the module at the next submit.  CUFZ_E_INVALID_ARG for
 * other values.  (The paper's runtime maps each GPU thread to one iteration
 * of a loop over the block, Sec. 4.1, Listing 2; this is the GPU-side
 * counterpart of unrolling that loop.) */
cufz_status cufz_set_program_lanes(cufz_ctx* ctx, uint32_t program_id, uint32_t lanes);
cufz_status cufz_get_program_lanes(cufz_ctx* ctx, uint32_t program_id, uint32_t* lanes);

/* Autotuner: for every program in the sample, times the sample's inputs of
 * that program run compiled and interpreted (best of three each; the sample
 * is repeated up to 2^24 test threads, at most 2048 inputs, so that the
 * timing measures throughput rather than launch costs) and moves
 * the program off its load-time path only if the other is at least 25%
 * faster.  Then, for compiled programs of at most 24 kept ops, it times the
 * lane mappings 2 and 4 the same way and keeps the fastest (a wider mapping
 * must win by 3%).  Last, unless the config fixes item_threads, it times
 * the whole sample (an equal share of each program's, at most 4096 inputs)
 * with work items of the size heuristic's choice and of 4096, 16384, 65536
 * and 262144 test threads, and keeps the fastest (3% margin) for the set of
 * programs loaded (reported in cufz_stats.item_threads once a batch ran).
 * The choices go to the autotune cache, if the config names one.  Needs an idle context; the sample's results are discarded.
 * *n_compiled receives the number of programs left on the compiled path. */
cufz_status cufz_autotune(cufz_ctx* ctx, const cufz_input* sample, uint32_t n,
                          uint32_t* n_compiled);

cufz_status cufz_get_stats(cufz_ctx* ctx, cufz_stats* out);
cufz_status cufz_reset_stats(cufz_ctx* ctx);

/* Checked execution of one input without any device allocation, for callers
 * that cannot allocate device memory: plugins whose host framework owns
 * every device allocation and hands out only the buffers of a call, and
 * services that must not grow their device footprint after start-up.  The
 * paper has no counterpart (its runtime is a CPU process).
 *
 * Runs `input` of the program (bytes, nbytes) on the current device with
 * the bytecode interpreter, exactly as a context would (pruned unless flags
 * has CUFZ_CF_NO_PRUNE; CUFZ_CF_NO_DIGEST honoured; redzone R and back-edge
 * budget as given), and writes: up to record_cap violation records to
 * `records` (device memory, may be NULL with record_cap 0), the 64 KiB
 * bucketed bitmap to `bitmap` (device memory, may be NULL), and the result
 * summary to `result` (device or host memory).  NEW_COV is measured against
 * an empty union.  Work is queued on `stream` (NULL: the legacy default
 * stream) and the call returns after it has completed.
 *
 * Scratch memory is a fixed 2 MiB array inside this library, held by every
 * GPU that loads it until the process exits; nothing is allocated.  The
 * first call on a device looks up the array's device address; make that
 * first call before any stream capture.  Programs whose loaded form
 * exceeds 64 KiB are rejected with CUFZ_E_NOMEM (every valid program's
 * loaded form is smaller: at most about 34 KB for 2,048 ops).  Every call shares the
 * array (what must start at zero is cleared per call): calls that overlap
 * on the GPU -- from several host threads or streams -- race and must be
 * serialised by the caller. */
cufz_status cufz_run_noalloc(const void* program, size_t nbytes, const cufz_input* input,
                             uint32_t flags, uint32_t redzone, uint32_t iter_budget,
                             cufz_violation* records, uint32_t record_cap, uint8_t* bitmap,
                             cufz_result* result, void* stream);

/* Measures the INT32 issue rate of device `device` with a kernel of
 * independent integer add/logic chains on the caller's stream; writes lane
 * operations per second. */
cufz_status cufz_int32_peak(int32_t device, void* stream, double* lane_ops_per_s);

#endif /* !__CUDACC_RTC__ */

#ifdef __cplusplus
}
#endif

#endif /* CUFZ_H */
