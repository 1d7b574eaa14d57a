// Device opcodes of the checked operations beyond loads and stores:
// division (DIV / REM) and the device heap (HALLOC, HFREE, HLD / HST),
// numbered after the shared layout's opcodes.  The loader emits them and the
// bytecode interpreter executes them; programs compiled at load time carry
// these operations as emitted code.
#pragma once

#include "layout.h"

namespace cufz {

// DIV / REM.  d = quotient or remainder register, a = dividend, b = divisor,
// imm = division site, x = 1 for REM | 2 when the result is live.
constexpr uint8_t D_DIVREM = D_NUM_OPCODES;

// Heap ops.  The thread's heap state sits in registers after the program's
// own: register j0 + s holds allocation site s's block (0 never allocated,
// its size n >= 1 while live, -1 once freed), for the j1 sites.
//   HALLOC: d = handle register, a = size register, imm = allocation site.
//   HFREE:  a = handle register, imm = free site.
//   HACC:   d = loaded value register, a = index, b = handle register,
//           imm = access site, x = log2(width) | 8 for a store | 16 when a
//           load's value is live.
constexpr uint8_t D_HALLOC = D_NUM_OPCODES + 1;
constexpr uint8_t D_HFREE = D_NUM_OPCODES + 2;
constexpr uint8_t D_HACC = D_NUM_OPCODES + 3;

}  // namespace cufz
