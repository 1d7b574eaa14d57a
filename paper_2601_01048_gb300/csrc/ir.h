// Internal program representation shared by the loader (decode, prune,
// register allocation, code generation) and the PREX analysis: the decoded
// program format (opcodes, structured control flow, sites).  Host-only.
#pragma once

#include <stdint.h>

#include <vector>

#include "engine.h"

namespace cufz {

enum : uint8_t {
  B_NOP = 0x00, B_SREG = 0x01, B_IMM = 0x02, B_MOV = 0x03, B_SEL = 0x04, B_DIV = 0x05, B_REM = 0x06,
  B_HALLOC = 0x07, B_HFREE = 0x08, B_LD = 0x40, B_ST = 0x41, B_HLD = 0x42, B_HST = 0x43,
  B_IF = 0x50, B_ELSE = 0x51, B_ENDIF = 0x52, B_LOOP = 0x53, B_ENDLOOP = 0x54, B_BAR = 0x55
};
constexpr uint32_t kMagic = 0x315A4643u;
// header byte 11: stores to shared buffers are performed (BARs order them)
constexpr uint32_t kPfSharedStores = 1;

inline bool is_alu_reg(uint8_t o) { return o >= 0x10 && o <= 0x1F; }
inline bool is_alu_imm(uint8_t o) { return o >= 0x30 && o <= 0x3F; }
inline bool is_heap_op(uint8_t o) { return o == B_HALLOC || o == B_HFREE || o == B_HLD || o == B_HST; }

// Virtual registers: 0..255 program registers, 256..271 special registers
// (materialised at thread start), 272.. hidden loop-trip registers.
constexpr int kSregBase = 256;
constexpr int kTripBase = 272;

struct IrOp {
  uint8_t opc = 0;     // program-format opcode
  int dst = -1, a = -1, b = -1, c = -1;
  int32_t imm = 0;
  int else_pc = -1, end_pc = -1, head_pc = -1;  // structure (head_pc: the IF/LOOP of an ELSE/ENDIF/ENDLOOP)
  int site = -1;       // branch site (IF/LOOP), access site (LD/ST/HLD/HST),
                       // division, allocation or free site
  int depth = 0;       // nesting depth of the op itself
  int trip = -1;       // hidden trip vreg (LOOP, ENDLOOP)
  bool kept = true;
  bool value_dead = false;
  bool value_live = false;  // ST of a block-serial program to a shared buffer: the
                            // stored value (register b) is performed, so a use
  int sreg = -1;       // SREG id (format level)
  int buf = -1;
  int width = 0;
};

struct Ir {
  int n_regs = 0, n_bufs = 0, n_sites = 0, n_access = 0, n_loops = 0, n_div = 0;
  int n_alloc = 0, n_free = 0;  // HALLOC and HFREE sites
  uint32_t shared_mask = 0, seed = 0, flags = 0;
  std::vector<uint16_t> loc0, loc1;
  std::vector<IrOp> ops;
  int nv = 0;  // vreg count (kTripBase + loops)
  // performed shared stores whose barriers must stay: each test block's
  // threads run in order, phase by phase (see prepare_barriers)
  bool block_serial = false;
};

// Decodes and validates program bytes; false on any violation of the format.
bool decode(const uint8_t* p, size_t n, Ir* ir);

// BarrierElimination (Sec. 5.2, Alg. 2): whether no value loaded from a
// shared buffer reaches an access index, a branch, a loop trip, a divisor or
// a heap operand.  Then a program's performed shared stores and its
// barriers change no check, edge or count, and it runs as if its stores
// were not performed and its barriers were gone.  True for programs whose
// shared stores are not performed.
bool barriers_eliminable(const Ir& ir);

// BarrierElimination where it applies; otherwise the program runs in the
// block-serial form (the compiled path's block functions: one CUDA thread
// runs a test block's threads in thread order, phase by phase between the
// BARs, with its shared stores performed; Sec. 4.1's collapsing transform,
// where a block becomes a loop over its threads that barriers split, run per
// GPU lane).  Sets ir->block_serial and marks the shared stores whose value
// is a use.  False for such programs with divisions or heap operations,
// which no engine runs that way.
bool prepare_barriers(Ir* ir);

// A program's decoded form as given (unpruned) for PREX, which looks at
// every access.
struct PrexInfo {
  Ir ir;
};

}  // namespace cufz
