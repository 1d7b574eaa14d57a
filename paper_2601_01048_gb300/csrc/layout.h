// Fixed layouts shared by the host runtime, the loader, the interpreter
// kernel and the programs compiled at load time (this header is also handed
// to the runtime compiler, so it uses no host headers there).
#pragma once

#if defined(__CUDACC_RTC__)
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
#else
#include <stddef.h>
#include <stdint.h>
#endif

#include "../../include/cufz.h"

namespace cufz {

constexpr int kMaxBufs = 9;
constexpr int kMaxDepth = 16;
constexpr int kMaxOps = 2048;       // ops of a program as given
constexpr int kMaxDevOps = 4096;    // device ops (kept ops + END)
constexpr int kMaxPhysRegs = 128;   // device registers per test thread
constexpr int kMaxPrograms = 256;
// Block-serial programs (performed shared stores whose barriers stay): one
// CUDA thread runs a whole test block, so a block's threads, their state
// between phases and its shared bytes live in that thread's local memory.
constexpr uint32_t kBlkMaxThreads = 64;   // threads per block
constexpr uint32_t kBlkSharedBytes = 1024; // bytes of all shared buffers of a block
constexpr uint32_t kBlkMaxSaved = 32;     // registers live across a barrier

constexpr int kBitmapBytes = 65536;
constexpr int kEdgeCount = 65536;
constexpr int kHashSlots = 2048;    // per-CTA edge hash table (power of two)
constexpr int kHashProbes = 8;
constexpr int kSatWords = kEdgeCount / 32;  // per-CTA bitmap of edges whose count reached 128
constexpr int kEdgeSmemBytes = (kHashSlots + kSatWords) * 4;  // hash table, then the bitmap
constexpr uint32_t kLaneBytes = 4;  // one i32 per lane per register
constexpr uint32_t kRegStride = 32 * kLaneBytes;  // register r of a warp: r * 128 + lane * 4

// Device opcodes (dense, so the dispatch switch is a jump table).
enum DevOpcode : uint8_t {
  D_MOV = 0,
  D_IMM,
  D_SEL,
  D_ALU0,              // 16 register-form ALU ops: D_ALU0 + (bytecode op - 0x10)
  D_ALUI0 = D_ALU0 + 16,  // 16 immediate forms
  D_LD = D_ALUI0 + 16, // load, value used
  D_LDX,               // load kept only as a checked access (value dead)
  D_ST,
  D_IF,
  D_ELSE,
  D_ENDIF,
  D_LOOP,
  D_ENDLOOP,
  D_END,
  D_NUM_OPCODES
};

// ALU order matches the program format's 0x10..0x1F.
enum AluOp : uint8_t {
  A_ADD = 0, A_SUB, A_MUL, A_SHL, A_SHR, A_SHRU, A_AND, A_OR, A_XOR, A_MIN, A_MAX,
  A_SETLT, A_SETLE, A_SETEQ, A_SETNE, A_SETLTU
};

// One device op, 16 bytes.  Register operands are byte offsets into the
// warp's register file (register r -> r * 128).
//   ALU/ALUI/MOV/IMM/SEL: d = dst, a, b (SEL: a cond, b x, imm = y offset);
//                         MOV: x = 1 for a special-register read (not
//                         counted in n_ops)
//   LD/LDX/ST:            d = dst (LD), a = index, b = buffer, x = log2 width,
//                         imm = access site
//   IF:                   a = cond, x = branch site, j0 = pc when no lane enters
//   ELSE:                 j0 = pc of ENDIF
//   LOOP/ENDLOOP:         d = counter, a = trip expression (LOOP), b = hidden
//                         trip register, imm = max trip (LOOP), x = branch site,
//                         j0 = exit pc, j1 = body pc
struct DevOp {
  uint8_t opc;
  uint8_t x;
  uint16_t d;
  uint16_t a;
  uint16_t b;
  int32_t imm;
  uint16_t j0;
  uint16_t j1;
};
static_assert(sizeof(DevOp) == 16, "DevOp is 16 bytes");

// Loaded program blob: header, ops, LOC table (u32: loc0 | loc1 << 16),
// zero list (u16 register offsets to clear at each test thread's start).
struct DevProgHdr {
  uint32_t n_ops;
  uint32_t n_regs;
  uint32_t n_bufs;
  uint32_t shared_mask;
  uint32_t seed;
  uint32_t n_sites;
  uint32_t sreg_mask;   // special registers materialised at thread start
  uint32_t n_zero;
  uint8_t sreg_reg[16]; // register index of each materialised special register
  uint32_t ops_off;     // byte offsets from the start of the blob
  uint32_t loc_off;
  uint32_t zero_off;
  uint32_t bytes;       // total blob size (multiple of 16)
  uint32_t n_loops;
  uint32_t reserved[3];
};
static_assert(sizeof(DevProgHdr) == 80, "DevProgHdr size");

// Everything a kernel needs about one admitted input, 576 bytes.
struct DevInput {
  uint32_t slot;
  uint32_t prog;          // program index
  uint32_t grid[3];
  uint32_t block[3];
  int32_t args[4];
  uint32_t T;             // threads per block
  uint32_t n_items;       // work items of this input
  uint64_t n_threads;     // grid * block threads
  // magic numbers for unsigned division by T, Bx, Bx*By, gx, gx*gy:
  // q = high 64 bits of m * n for n < 2^32, m = ceil(2^64 / d) for d >= 2;
  // d == 1 is encoded as m == 0.
  uint64_t mT, mBx, mBxy, mGx, mGxy;
  uint32_t Bx, Bxy, gx, gxy;
  int64_t len[kMaxBufs];
  int64_t base[kMaxBufs]; // virtual base in its space, for classification
  uint32_t prog_off;      // byte offset of the program blob in the program area
  uint32_t prog_bytes;
  uint64_t ticket;
  uint64_t user_tag;
  uint32_t seq;           // completion sequence number for the host
  uint32_t shared_mask;   // of the input's program: bit k = buffer k is shared
  uint32_t n_bufs;
  uint32_t pad[5];
  // in-bounds index count of buffer k for width 2^lw: min(len[k] >> lw, 2^31)
  uint32_t lim[kMaxBufs * 5];
  uint32_t pad2[19];
};
static_assert(sizeof(DevInput) == 576, "DevInput size");

// A contiguous range of linear test threads g = block_lin * T + thread_lin.
struct WorkItem {
  uint32_t input;   // index into the batch's DevInput array
  uint32_t g0;      // first linear thread
  uint32_t count;   // threads in this item
  uint32_t pad;
};

// Header of a batch in device memory, followed by DevInput[n_inputs] and
// WorkItem[n_items].
struct BatchHdr {
  uint32_t n_inputs;
  uint32_t n_items;
  uint32_t next_item;   // work counter (persistent CTAs pull from it)
  uint32_t epoch;
  uint64_t inputs_off;  // byte offsets from the header
  uint64_t items_off;
  uint32_t error;       // device-side error word (0 = none)
  uint32_t pad[7];
};
static_assert(sizeof(BatchHdr) == 64, "BatchHdr size");

// Per-slot accumulators in device memory; all zero at rest (first_key ~0).
struct SlotState {
  unsigned long long n_accesses;
  unsigned long long n_violations;
  unsigned long long digest;
  unsigned long long n_branch;
  unsigned long long n_ops;
  unsigned long long first_key;
  uint32_t rec_reserved;
  uint32_t n_touched;
  uint32_t items_done;
  uint32_t flags;
  uint32_t rec_listed;  // compiled path: violations of threads listed for records
  uint32_t pad;
  unsigned long long n_branch_folded;
};
static_assert(sizeof(SlotState) == 80, "SlotState size");

// Completion record in pinned host memory (one per slot).  The device writes
// the result, fences, then stores seq; the host reads seq first.
struct HostDone {
  cufz_result res;
  volatile uint32_t seq;
  uint32_t pad[7];
};
static_assert(sizeof(HostDone) == 128, "HostDone size");

// Device pointers of the arena tables, passed to every kernel.
struct EngineTables {
  uint8_t* progs;          // program blobs
  SlotState* slots;
  cufz_violation* records; // slot s: records + s * record_cap
  uint8_t* bitmaps;        // slot s: bitmaps + s * 65536 (if kept)
  uint32_t* counts;        // slot s: counts + s * 65536
  uint16_t* touched;       // slot s: touched + s * 65536
  uint32_t* union_map;     // 16384 words
  uint32_t* union_snap;    // 16384 words
  HostDone* done;          // pinned, mapped: done[slot]
  uint32_t record_cap;
  uint32_t redzone;
  uint32_t iter_budget;
  uint32_t flags;          // CUFZ_CF_*
};

}  // namespace cufz
